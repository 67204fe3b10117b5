// Dispatch of bp_ell_kernel over the group width G and the degree bounds
// (DC, DV) for one message type and check-node rule (kRule).
#pragma once

#include "launch.h"

namespace lbp {

template <typename MsgT, int kRule, int G, int DC, int DV, bool GS, bool SS, typename GraphT, bool SP = false,
          bool MU = false>
int launch_graph_one(const LaunchShape &s, const BpEllArgs &a, cudaStream_t st) {
    auto k = bp_ell_kernel<MsgT, G, DC, DV, GS, SS, GraphT, kRule, SP, MU>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(s.smem)) != cudaSuccess) {
        cudaGetLastError();
        return LBP_ECUDA;
    }
    k<<<s.grid, s.groups * G, s.smem, st>>>(a);
    return LBP_OK;
}

template <typename MsgT, int kRule, int G, int DC, int DV, bool GS, bool SS, typename IdxT = uint16_t,
          bool SP = false>
int launch_ell_one(const LaunchShape &s, const BpEllArgs &a, cudaStream_t st) {
    return launch_graph_one<MsgT, kRule, G, DC, DV, GS, SS, EllGraph<IdxT, DC, DV>, SP>(s, a, st);
}

// Implicit surface-code graph (Table III): no image; state in shared memory
// (any G) or in the workspace (G = 512, 1024).
template <typename MsgT, int kRule>
int launch_surface(const LaunchShape &s, const BpEllArgs &a, cudaStream_t st) {
    using GR = SurfaceGraph<6, 2>;
    if (s.state_smem) {
        switch (s.G) {
            case 64: return launch_graph_one<MsgT, kRule, 64, 6, 2, false, true, GR>(s, a, st);
            case 96: return launch_graph_one<MsgT, kRule, 96, 6, 2, false, true, GR>(s, a, st);
            case 128: return launch_graph_one<MsgT, kRule, 128, 6, 2, false, true, GR>(s, a, st);
            case 192: return launch_graph_one<MsgT, kRule, 192, 6, 2, false, true, GR>(s, a, st);
            case 256: return launch_graph_one<MsgT, kRule, 256, 6, 2, false, true, GR>(s, a, st);
            case 512: return launch_graph_one<MsgT, kRule, 512, 6, 2, false, true, GR>(s, a, st);
            case 1024: return launch_graph_one<MsgT, kRule, 1024, 6, 2, false, true, GR>(s, a, st);
            default: return LBP_ENOSYS;
        }
    }
    if (s.G == 512) return launch_graph_one<MsgT, kRule, 512, 6, 2, false, false, GR>(s, a, st);
    if (s.G == 1024) return launch_graph_one<MsgT, kRule, 1024, 6, 2, false, false, GR>(s, a, st);
    return LBP_ENOSYS;
}

template <typename MsgT, int kRule, int DC, int DV>
int launch_ell_g(const LaunchShape &s, const BpEllArgs &a, cudaStream_t st) {
    if (s.graph_smem) {
        switch (s.G) {
            case 32: return launch_ell_one<MsgT, kRule, 32, DC, DV, true, true>(s, a, st);
            case 64: return launch_ell_one<MsgT, kRule, 64, DC, DV, true, true>(s, a, st);
            case 96: return launch_ell_one<MsgT, kRule, 96, DC, DV, true, true>(s, a, st);
            case 128: return launch_ell_one<MsgT, kRule, 128, DC, DV, true, true>(s, a, st);
            case 192: return launch_ell_one<MsgT, kRule, 192, DC, DV, true, true>(s, a, st);
            case 256: return launch_ell_one<MsgT, kRule, 256, DC, DV, true, true>(s, a, st);
            case 512: return launch_ell_one<MsgT, kRule, 512, DC, DV, true, true>(s, a, st);
            case 1024: return launch_ell_one<MsgT, kRule, 1024, DC, DV, true, true>(s, a, st);
            default: return LBP_ENOSYS;
        }
    }
    // Large codes: graph in global memory; state in shared or global memory.
    if (s.idx32) {
        if (s.state_smem) {
            if (s.G == 1024) return launch_ell_one<MsgT, kRule, 1024, DC, DV, false, true, uint32_t>(s, a, st);
            return LBP_ENOSYS;
        }
        if (s.G == 512) return launch_ell_one<MsgT, kRule, 512, DC, DV, false, false, uint32_t>(s, a, st);
        return LBP_ENOSYS;
    }
    if (s.split) {
        // One shot per CTA: the shared part of a split state nearly fills it.
        switch (s.G) {
            case 512: return launch_ell_one<MsgT, kRule, 512, DC, DV, false, true, uint16_t, true>(s, a, st);
            case 768: return launch_ell_one<MsgT, kRule, 768, DC, DV, false, true, uint16_t, true>(s, a, st);
            case 1024: return launch_ell_one<MsgT, kRule, 1024, DC, DV, false, true, uint16_t, true>(s, a, st);
            default: return LBP_ENOSYS;
        }
    }
    if (s.state_smem) {
        switch (s.G) {
            case 256: return launch_ell_one<MsgT, kRule, 256, DC, DV, false, true>(s, a, st);
            case 512: return launch_ell_one<MsgT, kRule, 512, DC, DV, false, true>(s, a, st);
            case 1024: return launch_ell_one<MsgT, kRule, 1024, DC, DV, false, true>(s, a, st);
            default: return LBP_ENOSYS;
        }
    }
    switch (s.G) {
        case 256: return launch_ell_one<MsgT, kRule, 256, DC, DV, false, false>(s, a, st);
        case 512: return launch_ell_one<MsgT, kRule, 512, DC, DV, false, false>(s, a, st);
        case 1024: return launch_ell_one<MsgT, kRule, 1024, DC, DV, false, false>(s, a, st);
        default: return LBP_ENOSYS;
    }
}

// Round-periodic graph: the round image staged into shared memory; state in
// shared memory (any G) or in the workspace (G = 512, 1024).
template <typename MsgT, int kRule>
int launch_round(const LaunchShape &s, const BpEllArgs &a, cudaStream_t st) {
    using GR = RoundGraph<6, 2>;
    if (s.state_smem) {
        switch (s.G) {
            case 64: return launch_graph_one<MsgT, kRule, 64, 6, 2, true, true, GR>(s, a, st);
            case 96: return launch_graph_one<MsgT, kRule, 96, 6, 2, true, true, GR>(s, a, st);
            case 128: return launch_graph_one<MsgT, kRule, 128, 6, 2, true, true, GR>(s, a, st);
            case 192: return launch_graph_one<MsgT, kRule, 192, 6, 2, true, true, GR>(s, a, st);
            case 256: return launch_graph_one<MsgT, kRule, 256, 6, 2, true, true, GR>(s, a, st);
            case 512: return launch_graph_one<MsgT, kRule, 512, 6, 2, true, true, GR>(s, a, st);
            case 1024: return launch_graph_one<MsgT, kRule, 1024, 6, 2, true, true, GR>(s, a, st);
            default: return LBP_ENOSYS;
        }
    }
    if (s.G == 512) return launch_graph_one<MsgT, kRule, 512, 6, 2, true, false, GR>(s, a, st);
    if (s.G == 1024) return launch_graph_one<MsgT, kRule, 1024, 6, 2, true, false, GR>(s, a, st);
    return LBP_ENOSYS;
}

// Merged launch over a work list of codes with the same degree bounds (min-sum
// rule; 16-bit images read from global memory, states in shared memory).
template <typename MsgT, int kRule, int DC, int DV>
int launch_multi(const LaunchShape &s, const BpEllArgs &a, cudaStream_t st) {
    if constexpr (kRule != LBP_RULE_MIN_SUM) {
        return LBP_ENOSYS;
    } else {
        using GR = EllGraph<uint16_t, DC, DV>;
        switch (s.G) {
            case 64: return launch_graph_one<MsgT, kRule, 64, DC, DV, false, true, GR, false, true>(s, a, st);
            case 128: return launch_graph_one<MsgT, kRule, 128, DC, DV, false, true, GR, false, true>(s, a, st);
            case 192: return launch_graph_one<MsgT, kRule, 192, DC, DV, false, true, GR, false, true>(s, a, st);
            default: return LBP_ENOSYS;
        }
    }
}

template <typename MsgT, int kRule>
int launch_ell(const LaunchShape &s, const BpEllArgs &a, int DC, int DV, cudaStream_t st) {
    if (s.multi) {
        if (DC == 6 && DV == 2) return launch_multi<MsgT, kRule, 6, 2>(s, a, st);
        if (DC == 6 && DV == 3) return launch_multi<MsgT, kRule, 6, 3>(s, a, st);
        return LBP_ENOSYS;
    }
    if (s.round) return DC == 6 && DV == 2 ? launch_round<MsgT, kRule>(s, a, st) : LBP_ENOSYS;
    if (s.surface) return launch_surface<MsgT, kRule>(s, a, st);
    if (DC == 6 && DV == 2) return launch_ell_g<MsgT, kRule, 6, 2>(s, a, st);
    if (DC == 6 && DV == 3) return launch_ell_g<MsgT, kRule, 6, 3>(s, a, st);
    if (DC == 8 && DV == 4) return launch_ell_g<MsgT, kRule, 8, 4>(s, a, st);
    return LBP_ENOSYS;
}

}  // namespace lbp
