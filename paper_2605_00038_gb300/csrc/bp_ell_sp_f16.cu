// bp_ell_kernel instantiations, sum-product rule, binary16 messages.
#include "bp_ell_launch.cuh"

namespace lbp {

int launch_bp_ell_sp_f16(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st) {
    return launch_ell<__half, LBP_RULE_SUM_PRODUCT>(s, a, DC, DV, st);
}

}  // namespace lbp
