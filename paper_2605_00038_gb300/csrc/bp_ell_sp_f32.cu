// bp_ell_kernel instantiations, sum-product rule, float messages.
#include "bp_ell_launch.cuh"

namespace lbp {

int launch_bp_ell_sp_f32(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st) {
    return launch_ell<float, LBP_RULE_SUM_PRODUCT>(s, a, DC, DV, st);
}

}  // namespace lbp
