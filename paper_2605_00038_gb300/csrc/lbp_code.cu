// Host side of lbp_load_code / lbp_free_code and the small helpers of lbp.h.
//
// lbp_load_code validates H (CSR), derives the variable-major (CSC) view the
// LLR update walks, computes the prior LLR mu_v = ln((1 - p_v) / p_v) of
// Alg. 1 in binary64 and rounds it to binary32, and uploads a compact 16-bit
// image of the whole Tanner graph that the decode kernels stage into shared
// memory once per CTA.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace {

uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// Order in which the index-image kernel's lanes take the check pairs.  In
// the check phase, lane l of a warp's j-th step takes pair 32 j + l; each of
// its DC slots then gathers the posteriors of its two checks' columns, and a
// warp's 32 gathers cost as many shared-memory wavefronts as the most
// distinct columns that fall in one of the 32 banks (column mod 32).  The
// table keeps pair p at lane p mod 32, so the pair-indexed accesses (indices,
// messages, syndrome words) stay conflict-free, and chooses which pairs of a
// residue share a step so that the columns spread over the banks: simulated
// annealing over swaps within a residue, with a fixed seed (deterministic),
// minimising the summed wavefronts of the full steps.  Every pair is still
// processed exactly once, so results do not depend on the table.
std::vector<uint16_t> pair_table(const std::vector<uint8_t> &img, uint32_t off_cidx, int DC, int32_t Mp) {
    const int mp = Mp / 2, steps = mp / 32;
    std::vector<uint16_t> tab(static_cast<size_t>(mp));
    for (int p = 0; p < mp; ++p) tab[p] = static_cast<uint16_t>(p);
    if (steps < 2) return tab;
    const uint16_t *cidx = reinterpret_cast<const uint16_t *>(img.data() + off_cidx);
    auto step_cost = [&](int j) {
        int total = 0;
        for (int k = 0; k < DC; ++k) {
            for (int h = 0; h < 2; ++h) {
                uint16_t ids[32];
                int cnt[32] = {0};
                int worst = 0;
                for (int l = 0; l < 32; ++l) {
                    const uint16_t id = cidx[static_cast<size_t>(k) * Mp + 2 * tab[32 * j + l] + h];
                    bool dup = false;
                    for (int q = 0; q < l && !dup; ++q) dup = ids[q] == id;
                    ids[l] = id;
                    if (!dup && ++cnt[id & 31] > worst) worst = cnt[id & 31];
                }
                total += worst;
            }
        }
        return total;
    };
    std::vector<int> cost(static_cast<size_t>(steps));
    for (int j = 0; j < steps; ++j) cost[j] = step_cost(j);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;
        return st;
    };
    const long iters = std::min<long>(60000, 200L * mp);
    for (long it = 0; it < iters; ++it) {
        const double temp = 0.5 * (1.0 - static_cast<double>(it) / iters) + 0.01;
        const int l = static_cast<int>(next() % 32);
        const int j1 = static_cast<int>(next() % steps), j2 = static_cast<int>(next() % steps);
        if (j1 == j2) continue;
        std::swap(tab[32 * j1 + l], tab[32 * j2 + l]);
        const int c1 = step_cost(j1), c2 = step_cost(j2);
        const int d = c1 + c2 - cost[j1] - cost[j2];
        const double u = static_cast<double>(next() >> 11) * (1.0 / 9007199254740992.0);
        if (d <= 0 || std::exp(-d / temp) > u) {
            cost[j1] = c1;
            cost[j2] = c2;
        } else {
            std::swap(tab[32 * j1 + l], tab[32 * j2 + l]);
        }
    }
    return tab;
}

void release(lbp_code *c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaFree(c->d_image);
    cudaFree(c->d_ell);
    cudaFree(c->d_mu_pad);
    cudaFree(c->d_round);
    cudaFree(c->d_row_ptr);
    cudaFree(c->d_col_idx);
    cudaFree(c->d_mu);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

uint32_t magic(uint32_t x) { return static_cast<uint32_t>((1ull << 32) / x + 1); }

// Columns of check j of round t of the unrotated surface-code space-time
// matrix, by the formulas of Table III (VN0..VN3 data, VN4 / VN5 measurement
// blocks t-1 and t); absent neighbours are skipped.  Returns the count.
int surface_row(const lbp::SurfaceDesc &s, uint32_t t, uint32_t j, uint32_t out[6]) {
    int k = 0;
    const uint32_t d = static_cast<uint32_t>(s.d), bd = t * s.nr;
    if (s.type == 0) {
        const uint32_t r = j / d, cc = j % d;
        out[k++] = bd + j;
        out[k++] = bd + j + d;
        const uint32_t h = bd + s.d2 + r * (d - 1) + cc;
        if (cc != 0) out[k++] = h - 1;
        if (cc != d - 1) out[k++] = h;
    } else {
        const uint32_t r = j / (d - 1), cc = j % (d - 1);
        out[k++] = bd + r * d + cc;
        out[k++] = bd + r * d + cc + 1;
        const uint32_t h = bd + s.d2 + r * (d - 1) + cc;
        if (r != 0) out[k++] = h - (d - 1);
        if (r != d - 1) out[k++] = h;
    }
    const uint32_t M0 = static_cast<uint32_t>(s.T) * s.nr;
    int b4 = static_cast<int>(t) - 1;
    if (b4 < 0 && s.cyclic) b4 = s.T - 1;
    if (b4 >= 0 && b4 < s.nb) out[k++] = M0 + static_cast<uint32_t>(b4) * s.mr + j;
    if (static_cast<int>(t) < s.nb) out[k++] = M0 + t * s.mr + j;
    return k;
}

// Recognise H as the space-time matrix of Eq. 1 built from the H_X or H_Z
// rows of Table III (open or cyclic time boundary, d >= 3) by regenerating
// every row and comparing.  Fills *out and returns true on a match.
bool detect_surface(int32_t m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                    const std::vector<float> &mu, lbp::SurfaceDesc *out) {
    for (int64_t d = 3; d * (d - 1) <= m; ++d) {
        const int64_t mr = d * (d - 1), nr = d * d + (d - 1) * (d - 1);
        if (m % mr) continue;
        const int64_t T = m / mr;
        for (int cyclic = 0; cyclic < 2; ++cyclic) {
            if (cyclic && T < 2) continue;
            const int64_t nb = cyclic ? T : T - 1;
            if (T * nr + nb * mr != n) continue;
            // Exact multiply-high division for every dividend the kernel divides.
            if (static_cast<uint64_t>(n) * nr >= (1ull << 32) || static_cast<uint64_t>(m) * mr >= (1ull << 32))
                continue;
            for (int type = 0; type < 2; ++type) {
                lbp::SurfaceDesc s;
                std::memset(&s, 0, sizeof(s));
                s.d = static_cast<int32_t>(d); s.T = static_cast<int32_t>(T); s.nb = static_cast<int32_t>(nb);
                s.type = type; s.cyclic = cyclic;
                s.nr = static_cast<uint32_t>(nr); s.mr = static_cast<uint32_t>(mr);
                s.d2 = static_cast<uint32_t>(d * d);
                bool ok = true;
                uint32_t cols[6];
                for (int32_t c = 0; c < m && ok; ++c) {
                    const uint32_t t = static_cast<uint32_t>(c / mr), j = static_cast<uint32_t>(c % mr);
                    const int k = surface_row(s, t, j, cols);
                    std::sort(cols, cols + k);
                    const int32_t a = row_ptr[c];
                    if (row_ptr[c + 1] - a != k) { ok = false; break; }
                    for (int i = 0; i < k; ++i)
                        if (static_cast<uint32_t>(col_idx[a + i]) != cols[i]) { ok = false; break; }
                }
                if (!ok) continue;
                s.mg_d = magic(static_cast<uint32_t>(d));
                s.mg_d1 = magic(static_cast<uint32_t>(d - 1));
                s.mg_nr = magic(s.nr);
                s.mg_mr = magic(s.mr);
                const int64_t M0 = T * nr;
                s.mu_uniform = 1;
                s.mu_data = n > 0 ? mu[0] : 0.0f;
                s.mu_meas = nb > 0 ? mu[M0] : 0.0f;
                for (int64_t v = 0; v < n && s.mu_uniform; ++v)
                    if (mu[v] != (v < M0 ? s.mu_data : s.mu_meas)) s.mu_uniform = 0;
                *out = s;
                return true;
            }
        }
    }
    return false;
}

// Recognise H as the space-time matrix of Eq. 1 of some round matrix H_r
// (T >= 2 rounds, open or cyclic time boundary): row t m_r + j must hold H_r's
// row j (read from round 0) shifted by t n_r, then the measurement columns of
// blocks t - 1 and t that exist.  H_r's rows may have at most DC - 2 columns
// and its columns at most DV rows.  On a match fills *out and the round image.
bool detect_round(int32_t m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                  const std::vector<float> &mu, int DC, int DV, int32_t Mp, lbp::RoundDesc *out,
                  std::vector<uint8_t> *image) {
    for (int64_t T = 2; T <= m; ++T) {
        if (m % T) continue;
        const int64_t mr = m / T;
        for (int cyclic = 0; cyclic < 2; ++cyclic) {
            const int64_t nb = cyclic ? T : T - 1;
            const int64_t rest = static_cast<int64_t>(n) - nb * mr;
            if (rest <= 0 || rest % T) continue;
            const int64_t nr = rest / T, M0 = T * nr;
            const uint64_t big = static_cast<uint64_t>(n > m ? n : m), div = static_cast<uint64_t>(nr > mr ? nr : mr);
            if (nr >= 65535 || big * div >= (1ull << 32)) continue;    // exact multiply-high divisions
            bool ok = true;
            for (int64_t c = 0; c < m && ok; ++c) {
                const int64_t t = c / mr, j = c % mr;
                const int32_t a = row_ptr[c], e = row_ptr[c + 1];
                const int32_t a0 = row_ptr[j], e0 = row_ptr[j + 1];
                int32_t nd = 0;                       // round columns of row (t, j)
                while (a + nd < e && col_idx[a + nd] < M0) ++nd;
                int32_t nd0 = 0;
                while (a0 + nd0 < e0 && col_idx[a0 + nd0] < M0) ++nd0;
                if (nd != nd0 || nd > DC - 2) { ok = false; break; }
                for (int32_t k = 0; k < nd; ++k) {
                    if (col_idx[a0 + k] >= nr || col_idx[a + k] != col_idx[a0 + k] + t * nr) { ok = false; break; }
                }
                if (!ok) break;
                int64_t want[2];
                int nw = 0;
                for (int64_t b = t - 1; b <= t; ++b) {
                    int64_t bb = b;
                    if (cyclic) bb = (b + T) % T;
                    if (bb >= 0 && bb < nb) want[nw++] = M0 + bb * mr + j;
                }
                if (nw == 2 && want[0] > want[1]) std::swap(want[0], want[1]);
                if (nw == 2 && want[0] == want[1]) { ok = false; break; }
                if (e - (a + nd) != nw) { ok = false; break; }
                for (int k = 0; k < nw; ++k)
                    if (col_idx[a + nd + k] != want[k]) { ok = false; break; }
            }
            if (!ok) continue;
            // Round columns' checks (ascending) and their slots.
            std::vector<int32_t> deg(nr, 0);
            for (int64_t j = 0; j < mr; ++j)
                for (int32_t e = row_ptr[j]; e < row_ptr[j + 1] && col_idx[e] < M0; ++e) deg[col_idx[e]]++;
            int maxdeg = 0;
            for (int64_t q = 0; q < nr; ++q) maxdeg = deg[q] > maxdeg ? deg[q] : maxdeg;
            if (maxdeg > DV) continue;
            lbp::RoundDesc d;
            std::memset(&d, 0, sizeof(d));
            d.T = static_cast<int32_t>(T); d.nb = static_cast<int32_t>(nb); d.cyclic = cyclic;
            d.mr = static_cast<uint32_t>(mr); d.nr = static_cast<uint32_t>(nr);
            d.mg_mr = magic(d.mr); d.mg_nr = magic(d.nr);
            d.off_rcidx = 0;
            d.off_rvent = align16(2u * (DC - 2) * d.mr);
            d.bytes = align16(d.off_rvent + 4u * DV * d.nr);
            image->assign(d.bytes, 0);
            uint16_t *rcidx = reinterpret_cast<uint16_t *>(image->data() + d.off_rcidx);
            uint32_t *rvent = reinterpret_cast<uint32_t *>(image->data() + d.off_rvent);
            const uint32_t R = static_cast<uint32_t>(Mp) + 2u;
            for (size_t i = 0; i < static_cast<size_t>(DC - 2) * mr; ++i) rcidx[i] = static_cast<uint16_t>(nr);
            for (size_t i = 0; i < static_cast<size_t>(DV) * nr; ++i) rvent[i] = 0xffffffffu;
            std::vector<int32_t> fill(nr, 0);
            for (int64_t j = 0; j < mr; ++j) {
                int k = 0;
                for (int32_t e = row_ptr[j]; e < row_ptr[j + 1] && col_idx[e] < M0; ++e, ++k) {
                    const int32_t q = col_idx[e];
                    rcidx[static_cast<size_t>(k) * mr + j] = static_cast<uint16_t>(q);
                    rvent[static_cast<size_t>(fill[q]++) * nr + q] = static_cast<uint32_t>(k) * R + static_cast<uint32_t>(j);
                }
            }
            d.mu_uniform = 1;
            d.mu_data = mu[0];
            d.mu_meas = nb > 0 ? mu[M0] : 0.0f;
            for (int64_t v = 0; v < n && d.mu_uniform; ++v)
                if (mu[v] != (v < M0 ? d.mu_data : d.mu_meas)) d.mu_uniform = 0;
            *out = d;
            return true;
        }
    }
    return false;
}

}  // namespace

extern "C" void lbp_params_default(lbp_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->max_iter = 100;
    p->scale_mode = LBP_SCALE_ADAPTIVE;
    p->scale_const = 0.625f;
    p->lottery = 1;
    p->lottery_skip = 6;
    p->osd = 0;
    p->msg = LBP_MSG_F32;
    p->rule = LBP_RULE_MIN_SUM;
}

extern "C" const char *lbp_strerror(int code) {
    switch (code) {
        case LBP_OK: return "success";
        case LBP_EINVAL: return "invalid argument (malformed H, priors, parameters or sizes)";
        case LBP_ENOMEM: return "out of device memory or workspace too small";
        case LBP_ENOSYS: return "code / precision combination not supported";
        case LBP_ECUDA: return "CUDA runtime error";
        case LBP_E2BIG: return "request needs more scratch than the fixed no-allocation area holds";
        default: return "unknown error";
    }
}

namespace {

// The experiment switches of lbp_code, read once here (see internal.h).
void read_env_switches(lbp_code *c) {
    c->env_graph = 0;
    if (const char *g = std::getenv("LBP_GRAPH")) {
        if (!std::strcmp(g, "table")) c->env_graph = 1;
        else if (!std::strcmp(g, "implicit")) c->env_graph = 2;
        else if (!std::strcmp(g, "round")) c->env_graph = 3;
    }
    c->env_S = c->env_G = 0;
    if (const char *sh = std::getenv("LBP_BP_SHAPE")) {
        int S = 0, G = 0;
        if (std::sscanf(sh, "%d,%d", &S, &G) == 2 && S > 0 && G > 0) {
            c->env_S = S;
            c->env_G = G;
        }
    }
    c->env_pool_rows = 0;
    if (const char *pr = std::getenv("LBP_OSD_POOL_ROWS")) {
        const int v = std::atoi(pr);
        if (v > 0) c->env_pool_rows = v;
    }
    const char *lat = std::getenv("LBP_OSD_LAT");
    c->env_osd_lat = (lat && !std::strcmp(lat, "0")) ? 0 : 1;
    const char *dn = std::getenv("LBP_OSD_DENSE");
    c->env_osd_dense = (dn && !std::strcmp(dn, "0")) ? 0 : 1;
    const char *bl = std::getenv("LBP_BANK_LAYOUT");
    c->env_bank_layout = (bl && !std::strcmp(bl, "0")) ? 0 : 1;
}

// Rank of H over GF(2) (rows as packed 64-bit words, forward elimination).
int32_t gf2_rank(int32_t m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx) {
    const int32_t wn = (n + 63) / 64;
    std::vector<uint64_t> a(static_cast<size_t>(m) * wn, 0ull);
    for (int32_t r = 0; r < m; ++r)
        for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
            a[static_cast<size_t>(r) * wn + col_idx[e] / 64] |= 1ull << (col_idx[e] % 64);
    int32_t rank = 0;
    for (int32_t v = 0; v < n && rank < m; ++v) {
        const int32_t w = v / 64;
        const uint64_t bit = 1ull << (v % 64);
        int32_t p = -1;
        for (int32_t r = rank; r < m; ++r)
            if (a[static_cast<size_t>(r) * wn + w] & bit) { p = r; break; }
        if (p < 0) continue;
        for (int32_t k = 0; k < wn; ++k)
            std::swap(a[static_cast<size_t>(p) * wn + k], a[static_cast<size_t>(rank) * wn + k]);
        for (int32_t r = rank + 1; r < m; ++r)
            if (a[static_cast<size_t>(r) * wn + w] & bit)
                for (int32_t k = 0; k < wn; ++k) a[static_cast<size_t>(r) * wn + k] ^= a[static_cast<size_t>(rank) * wn + k];
        ++rank;
    }
    return rank;
}

}  // namespace

extern "C" int lbp_code_osd_form(const lbp_code *code, int32_t *dense, int32_t *rank) {
    if (!code) return LBP_EINVAL;
    if (dense) *dense = code->osd_dense;
    if (rank) *rank = code->osd_dense ? code->osd_rank : -1;
    return LBP_OK;
}

extern "C" int lbp_code_options(const lbp_code *code, int32_t *graph, int32_t *groups, int32_t *G,
                                int32_t *pool_rows, int32_t *osd_latency) {
    if (!code) return LBP_EINVAL;
    if (graph) *graph = code->env_graph;
    if (groups) *groups = code->env_S;
    if (G) *G = code->env_G;
    if (pool_rows) *pool_rows = code->env_pool_rows;
    if (osd_latency) *osd_latency = code->env_osd_lat;
    return LBP_OK;
}

extern "C" int lbp_load_code(int32_t m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                             const double *priors, lbp_code **out) {
    if (!out) return LBP_EINVAL;
    *out = nullptr;
    if (m < 0 || n < 0 || !row_ptr || (n > 0 && !priors)) return LBP_EINVAL;
    if (row_ptr[0] != 0) return LBP_EINVAL;
    int maxdeg = 0;
    for (int32_t c = 0; c < m; ++c) {
        const int32_t a = row_ptr[c], b = row_ptr[c + 1];
        if (b < a) return LBP_EINVAL;
        const int32_t deg = b - a;
        if (deg == 1 || deg > lbp::kMaxRowDeg) return LBP_EINVAL;
        for (int32_t e = a; e < b; ++e) {
            if (!col_idx || col_idx[e] < 0 || col_idx[e] >= n) return LBP_EINVAL;
            if (e > a && col_idx[e] <= col_idx[e - 1]) return LBP_EINVAL;
        }
        if (deg > maxdeg) maxdeg = deg;
    }
    const int32_t nnz = row_ptr[m];
    for (int32_t v = 0; v < n; ++v)
        if (!(priors[v] > 0.0 && priors[v] < 1.0)) return LBP_EINVAL;

    // Variable-major view: per column, its checks in ascending row order and
    // the CSR edge holding each message.
    std::vector<int32_t> col_ptr(static_cast<size_t>(n) + 1, 0), csc_row(nnz), csc_edge(nnz);
    for (int32_t e = 0; e < nnz; ++e) col_ptr[col_idx[e] + 1]++;
    int maxcol = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (col_ptr[v + 1] > maxcol) maxcol = col_ptr[v + 1];
        col_ptr[v + 1] += col_ptr[v];
    }
    {
        std::vector<int32_t> fill(n, 0);
        for (int32_t c = 0; c < m; ++c)
            for (int32_t e = row_ptr[c]; e < row_ptr[c + 1]; ++e) {
                const int32_t v = col_idx[e];
                const int32_t k = col_ptr[v] + fill[v]++;
                csc_row[k] = c;
                csc_edge[k] = e;
            }
    }
    // Alg. 1 prior LLR, binary64 then one rounding to binary32.
    std::vector<float> mu(n);
    for (int32_t v = 0; v < n; ++v) mu[v] = static_cast<float>(std::log((1.0 - priors[v]) / priors[v]));

    lbp_code *c = new (std::nothrow) lbp_code();
    if (!c) return LBP_ENOMEM;
    std::memset(c, 0, sizeof(*c));
    read_env_switches(c);
    c->m = m; c->n = n; c->nnz = nnz;
    c->max_row_deg = maxdeg; c->max_col_deg = maxcol;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return LBP_ECUDA; }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);

    auto upload = [&](void **dst, const void *src, size_t bytes) -> int {
        if (bytes == 0) bytes = 16;
        if (cudaMalloc(dst, bytes) != cudaSuccess) { cudaGetLastError(); return LBP_ENOMEM; }
        if (src && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return LBP_ECUDA;
        return LBP_OK;
    };
    int rc = upload(reinterpret_cast<void **>(&c->d_row_ptr), row_ptr, sizeof(int32_t) * (static_cast<size_t>(m) + 1));
    if (rc == LBP_OK && nnz > 0) rc = upload(reinterpret_cast<void **>(&c->d_col_idx), col_idx, sizeof(int32_t) * nnz);
    if (rc == LBP_OK) rc = upload(reinterpret_cast<void **>(&c->d_mu), n ? mu.data() : nullptr, sizeof(float) * n);

    // Compact 16-bit image for shared-memory staging.
    if (rc == LBP_OK && m < 65535 && n < 65535 && nnz < 65535) {
        lbp::GraphImage &g = c->img;
        uint32_t off = 0;
        g.off_row_ptr = off;  off = align16(off + 2u * (m + 1));
        g.off_col_idx = off;  off = align16(off + 2u * nnz);
        g.off_col_ptr = off;  off = align16(off + 2u * (n + 1));
        g.off_csc_edge = off; off = align16(off + 2u * nnz);
        g.off_csc_row = off;  off = align16(off + 2u * nnz);
        g.off_mu = off;       off = align16(off + 4u * n);
        g.bytes = off;
        std::vector<uint8_t> img(off, 0);
        auto put16 = [&](uint32_t base, const int32_t *src, size_t cnt) {
            uint16_t *d = reinterpret_cast<uint16_t *>(img.data() + base);
            for (size_t i = 0; i < cnt; ++i) d[i] = static_cast<uint16_t>(src[i]);
        };
        put16(g.off_row_ptr, row_ptr, static_cast<size_t>(m) + 1);
        put16(g.off_col_idx, col_idx, nnz);
        put16(g.off_col_ptr, col_ptr.data(), static_cast<size_t>(n) + 1);
        put16(g.off_csc_edge, csc_edge.data(), nnz);
        put16(g.off_csc_row, csc_row.data(), nnz);
        if (n) std::memcpy(img.data() + g.off_mu, mu.data(), 4u * n);
        rc = upload(reinterpret_cast<void **>(&c->d_image), img.data(), off);
    }
    // ELL image for the bounded-degree kernel.
    int ell_dc = 8, ell_dv = 4;
    if (maxdeg <= 6 && maxcol <= 2) { ell_dc = 6; ell_dv = 2; }
    else if (maxdeg <= 6 && maxcol <= 3) { ell_dc = 6; ell_dv = 3; }
    const int32_t Mp = (m + 1) & ~1, Np = (n + 1) & ~1;
    int32_t R = Mp + 2;
    // 16-bit indices when every message offset and column fits; otherwise
    // 32-bit (the kernel recovers an offset's check by a multiply-high
    // division, exact while DC * R^2 < 2^32).
    const bool fits16 = static_cast<int64_t>(ell_dc) * R < 65536 && n < 65535;
    const bool fits32 = static_cast<uint64_t>(ell_dc) * R * R < (1ull << 32);
    if (rc == LBP_OK && maxdeg <= 8 && maxcol <= 4 && (fits16 || fits32)) {
        lbp::EllImage &e = c->ell;
        // Supported (DC, DV) shapes: (6, 2), (6, 3), (8, 4).
        e.DC = ell_dc;
        e.DV = ell_dv;
        e.Mp = Mp;
        e.Np = Np;
        e.idx_bytes = fits16 ? 2 : 4;
        const uint32_t ib = static_cast<uint32_t>(e.idx_bytes);
        uint32_t off = 0;
        e.off_cidx = off; off = align16(off + ib * e.DC * Mp);
        e.off_vent = off; off = align16(off + ib * e.DV * Np);
        e.off_mu = off;   off = align16(off + 4u * (Np + 2));
        // Bank-aware layout when the image (with its pair table) and one
        // shot's FP32 state always fit in shared memory, so the index-image
        // form never reads the image from global memory: message rows padded
        // to a multiple of 32 words spread the column phase's message
        // gathers over the banks (both slots of a column then share the bank
        // pattern of its checks), and the pair table regroups the check phase.
        const int32_t Rr = (R + 31) & ~31;
        const uint32_t tab_bytes = align16(off + 2u * static_cast<uint32_t>(Mp / 2));
        if (c->env_bank_layout && fits16 && static_cast<int64_t>(ell_dc) * Rr < 65536 &&
            static_cast<size_t>(tab_bytes) + lbp::ell_state_bytes(4, ell_dc, Rr, Np, m) <=
                static_cast<size_t>(c->smem_optin)) {
            R = Rr;
            c->tab_R = Rr;
            c->tab_off_ptab = off;
            off = tab_bytes;
        }
        e.bytes = off;
        // Slot-aligned layout for a space-time matrix of Eq. 1 whose image and
        // FP32 state do not fit shared memory together (the kernel then reads
        // the image from global memory and may split the state): a check's
        // round columns fill slots 0 .. DC-3 (padded with column n), its
        // measurement column of block t-1 goes to slot DC-2 and that of block
        // t to slot DC-1.  Every message of a measurement column then sits in
        // the last two slots, which a split state keeps in the workspace, and
        // every message of a round column in the others.  The check update
        // and the lottery do not depend on slot order, so results are the same.
        lbp::RoundDesc rd;
        std::vector<uint8_t> rdimg;
        const bool aligned = !c->tab_R && ell_dc == 6 && ell_dv == 2 && fits16 &&
                             static_cast<size_t>(off) + lbp::ell_state_bytes(4, ell_dc, R, Np, m) >
                                 static_cast<size_t>(c->smem_optin) &&
                             detect_round(m, n, row_ptr, col_idx, mu, ell_dc, ell_dv, Mp, &rd, &rdimg);
        const int64_t M0 = aligned ? static_cast<int64_t>(rd.T) * rd.nr : 0;
        e.meas0 = static_cast<int32_t>(M0);
        // Slot of column v in row r.
        auto slot_of = [&](int32_t r, int32_t v, int32_t k_sorted) -> int32_t {
            if (!aligned) return k_sorted;
            if (v < M0) return k_sorted;                       // round columns come first, ascending
            const int64_t blk = (v - M0) / rd.mr, t = r / rd.mr;
            return blk == t ? ell_dc - 1 : ell_dc - 2;
        };
        std::vector<uint8_t> img(off, 0);
        auto put = [&](uint32_t base, size_t i, uint32_t v) {
            if (ib == 2) reinterpret_cast<uint16_t *>(img.data() + base)[i] = static_cast<uint16_t>(v);
            else reinterpret_cast<uint32_t *>(img.data() + base)[i] = v;
        };
        float *mu_e = reinterpret_cast<float *>(img.data() + e.off_mu);
        for (int32_t r = 0; r < Mp; ++r) {
            const int32_t a = r < m ? row_ptr[r] : 0, deg = r < m ? row_ptr[r + 1] - a : 0;
            for (int k = 0; k < e.DC; ++k) put(e.off_cidx, static_cast<size_t>(k) * Mp + r, static_cast<uint32_t>(n));
            for (int k = 0; k < deg; ++k)
                put(e.off_cidx, static_cast<size_t>(slot_of(r, col_idx[a + k], k)) * Mp + r,
                    static_cast<uint32_t>(col_idx[a + k]));
        }
        for (int32_t v = 0; v < Np; ++v) {
            const int32_t a = v < n ? col_ptr[v] : 0, deg = v < n ? col_ptr[v + 1] - a : 0;
            for (int k = 0; k < e.DV; ++k) {
                uint32_t ent = static_cast<uint32_t>(Mp);         // padding: message beta[0][Mp] = +0
                if (k < deg) {
                    const int32_t r = csc_row[a + k];
                    const int32_t slot = slot_of(r, v, csc_edge[a + k] - row_ptr[r]);
                    ent = static_cast<uint32_t>(slot * R + r);
                }
                put(e.off_vent, static_cast<size_t>(k) * Np + v, ent);
            }
        }
        for (int32_t v = 0; v < Np + 2; ++v) mu_e[v] = v < n ? mu[v] : INFINITY;
        if (c->tab_R) {
            const std::vector<uint16_t> tab = pair_table(img, e.off_cidx, e.DC, Mp);
            std::memcpy(img.data() + c->tab_off_ptab, tab.data(), 2u * tab.size());
        }
        rc = upload(reinterpret_cast<void **>(&c->d_ell), img.data(), off);
        // Implicit graph: the same shape (DC = 6, DV = 2, Mp, Np, R = Mp + 2)
        // with indices from Table III's formulas; priors that are not uniform
        // per block are read from d_mu_pad.
        if (rc == LBP_OK && ell_dc == 6 && ell_dv == 2 && detect_surface(m, n, row_ptr, col_idx, mu, &c->surf)) {
            c->surface = 1;
            if (!c->surf.mu_uniform)
                rc = upload(reinterpret_cast<void **>(&c->d_mu_pad), mu_e, 4u * (Np + 2));
        }
        // Round-periodic graph: one round's index table (Eq. 1 structure).
        std::vector<uint8_t> rimg;
        if (rc == LBP_OK && ell_dc == 6 && ell_dv == 2 &&
            detect_round(m, n, row_ptr, col_idx, mu, ell_dc, ell_dv, Mp, &c->rnd, &rimg)) {
            c->round = 1;
            rc = upload(reinterpret_cast<void **>(&c->d_round), rimg.data(), rimg.size());
            if (rc == LBP_OK && !c->rnd.mu_uniform && !c->d_mu_pad)
                rc = upload(reinterpret_cast<void **>(&c->d_mu_pad), mu_e, 4u * (Np + 2));
        }
    }
    if (rc != LBP_OK) { release(c); return rc; }
    // Dense OSD: the whole augmented matrix of a small code in one warp's
    // registers (32 rows per row slot, 64 columns per word, the syndrome bit
    // in column n).
    if (c->d_image && c->env_osd_dense && m >= 1 && m <= 160 && n + 1 <= 320) {
        c->osd_dense = 1;
        c->osd_RL = (m + 31) / 32;
        c->osd_WN = (n + 1 + 63) / 64;
        c->osd_rank = gf2_rank(m, n, row_ptr, col_idx);
    }
    *out = c;
    return LBP_OK;
}

extern "C" int lbp_free_code(lbp_code *code) {
    if (!code) return LBP_EINVAL;
    release(code);
    return LBP_OK;
}

extern "C" int lbp_code_surface(const lbp_code *code, int32_t *d, int32_t *T, int32_t *type,
                                int32_t *cyclic) {
    if (!code) return LBP_EINVAL;
    const bool on = code->surface != 0;
    if (d) *d = on ? code->surf.d : 0;
    if (T) *T = on ? code->surf.T : 0;
    if (type) *type = on ? code->surf.type : 0;
    if (cyclic) *cyclic = on ? code->surf.cyclic : 0;
    return LBP_OK;
}

extern "C" int lbp_code_rounds(const lbp_code *code, int32_t *T, int32_t *m_r, int32_t *n_r, int32_t *cyclic) {
    if (!code) return LBP_EINVAL;
    const bool on = code->round != 0;
    if (T) *T = on ? code->rnd.T : 0;
    if (m_r) *m_r = on ? static_cast<int32_t>(code->rnd.mr) : 0;
    if (n_r) *n_r = on ? static_cast<int32_t>(code->rnd.nr) : 0;
    if (cyclic) *cyclic = on ? code->rnd.cyclic : 0;
    return LBP_OK;
}

extern "C" int lbp_code_info(const lbp_code *code, int32_t *m, int32_t *n, int32_t *nnz) {
    if (!code) return LBP_EINVAL;
    if (m) *m = code->m;
    if (n) *n = code->n;
    if (nnz) *nnz = code->nnz;
    return LBP_OK;
}
