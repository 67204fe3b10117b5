// bp_ell_kernel instantiations for int8_t messages.
#include "bp_ell_launch.cuh"

namespace lbp {

int launch_bp_ell_i8(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st) {
    return launch_ell<int8_t>(s, a, DC, DV, st);
}

}  // namespace lbp
