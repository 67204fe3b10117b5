// bp_ell_kernel instantiations, sum-product rule, Int3.4 messages.
#include "bp_ell_launch.cuh"

namespace lbp {

int launch_bp_ell_sp_i8(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st) {
    return launch_ell<int8_t, LBP_RULE_SUM_PRODUCT>(s, a, DC, DV, st);
}

}  // namespace lbp
