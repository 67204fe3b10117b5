// lbp_probe_smem: measured shared-memory load bandwidth of the device, the
// denominator of the on-chip roofline of K_bp (whose per-shot state lives in
// shared memory).
//
// Every SM runs two CTAs of 1024 threads; each thread reads 16-byte words
// from its CTA's 64 KB of shared memory, eight independent loads per loop
// trip at addresses that change every trip, conflict-free (a warp's 32
// consecutive 16-byte words fill four 128-byte wavefronts).  The loads are
// XOR-folded into one word per thread that is stored only when it equals a
// value it cannot take, so nothing is optimised away and nothing is written.
// Timed with a CUDA event pair on the caller's stream after one warm-up
// launch.  It changes no clock or power setting; the caller samples the
// clock it ran at.
#include <cstdint>

#include "internal.h"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeWords = 4096;          // 16-byte words: 64 KB per CTA
constexpr int kProbeLoads = 8;

__global__ void __launch_bounds__(kProbeThreads, 2) smem_probe_kernel(int trips, uint32_t *sink) {
    extern __shared__ __align__(16) uint4 buf[];
    for (int i = threadIdx.x; i < kProbeWords; i += blockDim.x)
        buf[i] = make_uint4(i, i * 3u, i * 5u, i * 7u);
    __syncthreads();
    uint32_t acc = 0;
    int base = threadIdx.x;
    for (int r = 0; r < trips; ++r) {
        #pragma unroll
        for (int j = 0; j < kProbeLoads; ++j) {
            const uint4 v = buf[(base + j * kProbeThreads / 2) & (kProbeWords - 1)];
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
        base += 32;
    }
    if (acc == 0xFFFFFFFFu) sink[blockIdx.x] = acc;    // never true: the words are small
}

}  // namespace

extern "C" int lbp_probe_smem(int32_t trips, double *bytes, float *ms, void *stream) {
    if (trips < 1 || trips > (1 << 20) || !bytes || !ms) return LBP_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LBP_ECUDA;
    }
    const size_t smem = sizeof(uint4) * kProbeWords;
    if (cudaFuncSetAttribute(smem_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess) {
        cudaGetLastError();
        return LBP_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = 2 * sms;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaEventDestroy(a);
        return LBP_ECUDA;
    }
    // The sink is never written (see the kernel); any valid address serves.
    uint32_t *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(uint32_t) * grid) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return LBP_ENOMEM;
    }
    smem_probe_kernel<<<grid, kProbeThreads, smem, s>>>(trips, sink);
    cudaEventRecord(a, s);
    smem_probe_kernel<<<grid, kProbeThreads, smem, s>>>(trips, sink);
    cudaEventRecord(b, s);
    int rc = LBP_OK;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        rc = LBP_ECUDA;
    }
    *bytes = static_cast<double>(grid) * kProbeThreads * static_cast<double>(trips) * kProbeLoads * sizeof(uint4);
    cudaFree(sink);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

// lbp_probe_phi: out[i] = phi(x[i]) with the device function the sum-product
// check-node rule uses (bp_common.cuh), so that its accuracy can be measured
// against a binary64 evaluation.
#include "bp_common.cuh"

namespace {

__global__ void phi_probe_kernel(const float *x, float *out, int64_t n) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = lbp::gallager_phi(x[i]);
}

}  // namespace

extern "C" int lbp_probe_phi(const float *x, float *out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!x || !out))) return LBP_EINVAL;
    if (n == 0) return LBP_OK;
    const int64_t blocks = (n + 255) / 256;
    phi_probe_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0,
                       static_cast<cudaStream_t>(stream)>>>(x, out, n);
    return cudaGetLastError() == cudaSuccess ? LBP_OK : LBP_ECUDA;
}
