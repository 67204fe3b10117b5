// bp_ell_kernel instantiations for int8_t messages.
#include "bp_ell_launch.cuh"

namespace lbp {

int launch_bp_ell_i8(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st) {
    return launch_ell<int8_t, LBP_RULE_MIN_SUM>(s, a, DC, DV, st);
}

}  // namespace lbp
