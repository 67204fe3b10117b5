// K_osd_dense instantiations: rows per lane RL and 64-bit words per
// augmented row WN, 1..5 each (m <= 160, n + 1 <= 320).
#include <cuda_runtime.h>

#include "osd_dense_kernel.cuh"

namespace lbp {

namespace {

template <int RL, int WN>
int launch_rw(const OsdDenseArgs &a, int grid, size_t smem, cudaStream_t st) {
    auto k = osd_dense_kernel<RL, WN>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess) {
        cudaGetLastError();
        return LBP_ECUDA;
    }
    k<<<grid, kOsdDenseWarps * 32, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? LBP_OK : LBP_ECUDA;
}

template <int RL>
int launch_r(const OsdDenseArgs &a, int WN, int grid, size_t smem, cudaStream_t st) {
    switch (WN) {
        case 1: return launch_rw<RL, 1>(a, grid, smem, st);
        case 2: return launch_rw<RL, 2>(a, grid, smem, st);
        case 3: return launch_rw<RL, 3>(a, grid, smem, st);
        case 4: return launch_rw<RL, 4>(a, grid, smem, st);
        case 5: return launch_rw<RL, 5>(a, grid, smem, st);
        default: return LBP_ENOSYS;
    }
}

}  // namespace

int launch_osd_dense(const OsdDenseArgs &a, int RL, int WN, int grid, size_t smem, cudaStream_t st) {
    switch (RL) {
        case 1: return launch_r<1>(a, WN, grid, smem, st);
        case 2: return launch_r<2>(a, WN, grid, smem, st);
        case 3: return launch_r<3>(a, WN, grid, smem, st);
        case 4: return launch_r<4>(a, WN, grid, smem, st);
        case 5: return launch_r<5>(a, WN, grid, smem, st);
        default: return LBP_ENOSYS;
    }
}

}  // namespace lbp
