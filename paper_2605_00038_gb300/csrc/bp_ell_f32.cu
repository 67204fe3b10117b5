// bp_ell_kernel instantiations for float messages.
#include "bp_ell_launch.cuh"

namespace lbp {

int launch_bp_ell_f32(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st) {
    return launch_ell<float, LBP_RULE_MIN_SUM>(s, a, DC, DV, st);
}

}  // namespace lbp
