// lbp_decode_noalloc: the decode of lbp_decode for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or an allocator: a latency-bound request
// loop on a pre-sized device, where an allocation could stall or synchronise
// the device in the middle of a request, or a plugin whose host process owns
// every allocation and hands it none.  This entry point takes its scratch
// from a fixed array in device memory that the library defines, so the
// caller passes only inputs and outputs.
//
// The array is a file-scope __device__ variable of kNoAllocScratchBytes bytes:
// every GPU that loads this library holds it until the process exits.  Host
// code cannot use the array's name as a device address (it is a host-side
// stand-in), so the first call on a device does a one-time set-up: it looks
// the address up with cudaGetSymbolAddress, with that device current, and
// keeps it; the decode kernels receive that pointer.  That first call should
// come before any stream capture begins.  Every call on a device shares the array and
// it keeps the last call's contents: the decode path clears what must start at
// zero (its shot and queue counters) on the call's stream before the kernels
// run, so consecutive calls on one stream are independent, but calls that
// overlap on the GPU (two streams, or two host threads) race on the array.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = static_cast<size_t>(LBP_NOALLOC_SCRATCH_BYTES);
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `dev` (current), looked up once.
int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return LBP_ENOSYS;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LBP_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return LBP_OK;
}

}  // namespace

extern "C" int lbp_decode_noalloc(const lbp_code *code, const lbp_params *params, int64_t num_shots,
                                  const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
                                  uint8_t *osd_out, int32_t *iters_out, float *llr_out, void *stream) {
    if (!code || !params) return LBP_EINVAL;
    const size_t need = lbp_workspace_size(code, params, num_shots);
    if (need == 0) return LBP_EINVAL;               // invalid parameters or sizes
    if (need > kNoAllocScratchBytes) return LBP_E2BIG;
    if (num_shots == 0) return LBP_OK;
    if (!syndromes || !err_out || !converged || !iters_out) return LBP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != code->device) return LBP_EINVAL;
    void *scratch = nullptr;
    const int rc = scratch_address(dev, &scratch);
    if (rc) return rc;
    return lbp::decode_device(code, params, num_shots, syndromes, err_out, converged, osd_out,
                              iters_out, llr_out, scratch, kNoAllocScratchBytes,
                              static_cast<cudaStream_t>(stream));
}
