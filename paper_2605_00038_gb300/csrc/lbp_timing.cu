// Optional per-kernel timing: CUDA event pairs recorded around the kernels
// that lbp_decode launches, summed on request (see lbp_timing_* in lbp.h).
#include <mutex>
#include <vector>

#include "internal.h"
#include "timing.h"

namespace {

struct Pair {
    cudaEvent_t a, b;
    int kind;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Pair> g_pairs;

void drop_all() {
    for (auto &p : g_pairs) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pairs.clear();
}

}  // namespace

namespace lbp {

bool timing_on() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_on;
}

void *timing_begin(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return nullptr;
    Pair p{};
    if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaEventRecord(p.a, s);
    g_pairs.push_back(p);
    return reinterpret_cast<void *>(g_pairs.size());
}

void timing_end(void *tok, cudaStream_t s, int kind) {
    if (!tok) return;
    std::lock_guard<std::mutex> lk(g_mu);
    const size_t i = reinterpret_cast<size_t>(tok) - 1;
    if (i >= g_pairs.size()) return;
    g_pairs[i].kind = kind;
    cudaEventRecord(g_pairs[i].b, s);
}

}  // namespace lbp

extern "C" int lbp_timing_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    drop_all();
    g_on = on != 0;
    return LBP_OK;
}

extern "C" int lbp_timing_read(double *bp_ms, int64_t *bp_launches, double *osd_ms, int64_t *osd_launches) {
    std::lock_guard<std::mutex> lk(g_mu);
    double t[2] = {0.0, 0.0};
    int64_t c[2] = {0, 0};
    int rc = LBP_OK;
    for (auto &p : g_pairs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
            cudaGetLastError();
            rc = LBP_ECUDA;
            continue;
        }
        const int k = p.kind == lbp::kTimeOsd ? 1 : 0;
        t[k] += ms;
        c[k] += 1;
    }
    drop_all();
    if (bp_ms) *bp_ms = t[0];
    if (bp_launches) *bp_launches = c[0];
    if (osd_ms) *osd_ms = t[1];
    if (osd_launches) *osd_launches = c[1];
    return rc;
}
