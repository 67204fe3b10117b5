// Launch entry points of the BP kernels (one translation unit per message
// type, so that nvcc compiles the instantiations in parallel).
#pragma once

#include <cuda_runtime.h>

#include "bp_ell_kernel.cuh"

namespace lbp {

struct LaunchShape {
    int grid, groups, G;
    size_t smem;
    bool graph_smem, state_smem, idx32;
    bool surface;            // implicit surface-code graph (no index image)
    bool round;              // round-periodic graph (one round's index image)
    bool split;              // split state: ks message slots in shared memory, the rest in the workspace
    bool multi;              // merged launch over the items of a work list
};

int launch_bp_ell_f32(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st);
int launch_bp_ell_f16(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st);
int launch_bp_ell_i8(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st);
int launch_bp_ell_sp_f32(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st);
int launch_bp_ell_sp_f16(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st);
int launch_bp_ell_sp_i8(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st);

}  // namespace lbp
