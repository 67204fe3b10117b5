// The lottery (Alg. 3) and the four baseline sign-flip policies of Sec. III-B,
// shared by the BP kernels.  Run by the 32 lanes of one warp of the group;
// lottery_pick returns the stored index of the column whose LLR is to be
// negated (v*), the same in every lane, or -1 when no check is unsatisfied.
// It is lottery_check (c*) followed by lottery_column (v*); a kernel may run
// the first half early, during iteration i's check phase, when the policy
// draws the check at random (it then depends only on s_hat(i-1) and s).
//
//   U   = s_hat(i-1) xor s (bit words sp ^ s_w); N = |U|
//   u   = SplitMix64(seed, (g << 24) + i): low 32 bits choose the check,
//         high 32 bits the column of the random-VN policies
//   CN  random: the k-th member of U in ascending row order, k = floor(u N / 2^32);
//       worst:  the member with the most columns at lambda <= 0, lowest row on ties
//   VN  proposed: most unsatisfied checks, then least |lambda|, then lowest column;
//       unreliable: least |lambda|, then lowest column;
//       random: column floor(u2 deg / 2^32) of c* in ascending column order.
//
// Acc gives the graph as the kernel stores it: col(k, c) is the stored index
// of check c's slot-k column (acc.pad when absent), ent(k, v) the message
// offset slot * R + check of stored column v's k-th check (absent checks:
// an offset whose row is not a check, or one at or past acc.ent_end), orig(v)
// the column id in H (ties are broken on it).
#pragma once

#include <cstdint>

#include "bp_common.cuh"

namespace lbp {

// True for the policies whose check depends only on U and the draw, not on
// the posteriors of this iteration (so it can be drawn early).
__device__ __forceinline__ bool lottery_random_check(int policy) {
    return policy != LBP_LOTTERY_WORST_UNRELIABLE && policy != LBP_LOTTERY_WORST_RANDOM;
}

// First half: the check c* (or -1 when U is empty) and the high 32 bits u2
// of the draw, the same in every lane.
template <int DC, typename Acc>
__device__ __forceinline__ int lottery_check(const Acc &acc, const uint32_t *sp, const uint32_t *s_w, int W32,
                                             int lane, uint64_t seed, uint64_t g, int it, int policy,
                                             const float *lam, uint32_t &u2_out) {
    uint32_t N = 0;
    for (int w0 = 0; w0 < W32; w0 += 32) {
        const int w = w0 + lane;
        const uint32_t word = (w < W32) ? (sp[w] ^ s_w[w]) : 0u;
        uint32_t pc = __popc(word);
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, o);
        N += pc;
    }
    if (N == 0) return -1;
    const uint64_t r64 = splitmix64_at(seed, (g << 24) + static_cast<uint64_t>(it));
    const uint32_t u = static_cast<uint32_t>(r64);
    u2_out = static_cast<uint32_t>(r64 >> 32);
    int cstar = -1;
    if (policy == LBP_LOTTERY_WORST_UNRELIABLE || policy == LBP_LOTTERY_WORST_RANDOM) {
        int bn = -1, bcr = 0x7fffffff;
        for (int w = lane; w < W32; w += 32) {
            uint32_t word = sp[w] ^ s_w[w];
            while (word) {
                const int c = w * 32 + __ffs(word) - 1;
                word &= word - 1u;
                int ne = 0;
                #pragma unroll
                for (int k = 0; k < DC; ++k) {
                    const uint32_t v = acc.col(k, c);
                    ne += (v != acc.pad && lam[v] <= 0.0f) ? 1 : 0;
                }
                if (ne > bn || (ne == bn && c < bcr)) { bn = ne; bcr = c; }
            }
        }
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int on = __shfl_xor_sync(0xffffffffu, bn, o);
            const int oc = __shfl_xor_sync(0xffffffffu, bcr, o);
            if (on > bn || (on == bn && oc < bcr)) { bn = on; bcr = oc; }
        }
        cstar = bcr;
    } else {
        const uint32_t k = static_cast<uint32_t>((static_cast<uint64_t>(u) * N) >> 32);
        uint32_t base = 0;
        for (int w0 = 0; w0 < W32 && cstar < 0; w0 += 32) {
            const int w = w0 + lane;
            uint32_t word = (w < W32) ? (sp[w] ^ s_w[w]) : 0u;
            const uint32_t pc = __popc(word);
            uint32_t incl = pc;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - pc;
            const bool mine = (k >= base + excl) && (k < base + incl);
            const unsigned own = __ballot_sync(0xffffffffu, mine);
            if (own) {
                int pick = 0;
                if (mine) {
                    uint32_t rr = k - base - excl;
                    while (rr--) word &= word - 1u;
                    pick = w * 32 + (__ffs(word) - 1);
                }
                cstar = __shfl_sync(0xffffffffu, pick, __ffs(own) - 1);
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    return cstar;
}

// Second half: the column v* of check c* (stored index, or -1).
template <int DC, int DV, typename Acc>
__device__ __forceinline__ int lottery_column(const Acc &acc, int cstar, uint32_t u2, const uint32_t *sp,
                                              const uint32_t *s_w, int lane, int policy, const float *lam,
                                              int m, int R, uint32_t magic) {
    if (cstar < 0) return -1;
    // Lane k < DC holds slot k of c*; ov is its column id in H (ties, order).
    const uint32_t vl = lane < DC ? acc.col(lane, cstar) : acc.pad;
    const bool present = vl != acc.pad;
    const uint32_t ov = present ? acc.orig(vl) : 0xffffffffu;
    if (policy == LBP_LOTTERY_WORST_RANDOM || policy == LBP_LOTTERY_RANDOM_RANDOM) {
        const int deg = __popc(__ballot_sync(0xffffffffu, present));
        const int kk = static_cast<int>((static_cast<uint64_t>(u2) * static_cast<uint32_t>(deg)) >> 32);
        int rank = 0;
        #pragma unroll
        for (int o = 0; o < DC; ++o) {
            const uint32_t w = __shfl_sync(0xffffffffu, ov, o);
            rank += (w < ov) ? 1 : 0;
        }
        const unsigned pick = __ballot_sync(0xffffffffu, present && rank == kk);
        return static_cast<int>(__shfl_sync(0xffffffffu, vl, __ffs(pick) - 1));
    }
    int bc = -1;
    float ba = 0.0f;
    uint32_t bo = 0xffffffffu, bv = acc.pad;
    if (present) {
        bv = vl;
        bo = ov;
        bc = 0;
        if (policy == LBP_LOTTERY_PROPOSED) {
            #pragma unroll
            for (int kk = 0; kk < DV; ++kk) {
                const uint32_t o = acc.ent(kk, vl);
                const uint32_t r = o - __umulhi(o, magic) * static_cast<uint32_t>(R);
                if (o < acc.ent_end && r < static_cast<uint32_t>(m))
                    bc += ((sp[r >> 5] ^ s_w[r >> 5]) >> (r & 31)) & 1u;
            }
        }
        ba = fabsf(lam[vl]);
    }
    #pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
        const float oa = __shfl_xor_sync(0xffffffffu, ba, o);
        const uint32_t oo = __shfl_xor_sync(0xffffffffu, bo, o);
        const uint32_t ovv = __shfl_xor_sync(0xffffffffu, bv, o);
        const bool better = oc > bc || (oc == bc && (oa < ba || (oa == ba && oo < bo)));
        if (better) { bc = oc; ba = oa; bo = oo; bv = ovv; }
    }
    bv = __shfl_sync(0xffffffffu, bv, 0);
    bc = __shfl_sync(0xffffffffu, bc, 0);
    return bc >= 0 ? static_cast<int>(bv) : -1;
}

// ---- Faster form used by the index-image kernels in shared memory ---------
// The same picks as lottery_check + lottery_column, split so that a kernel
// can do everything that does not depend on this iteration's posteriors
// early: lottery_check_fast (c*: one scan when U fits one word per lane),
// lottery_prepare (c*'s columns, their unsatisfied counts, the whole pick of
// the random-VN policies) and, after the posteriors are known,
// lottery_finish (least |lambda| among the best-counted columns, then the
// lowest column id).  Every lane takes part in each warp collective.

// Position of the r-th set bit (r counted from 0, r < popc(x)) of x.
__device__ __forceinline__ int nth_set_bit(uint32_t x, uint32_t r) {
    int pos = 0;
    #pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const uint32_t lo = __popc(x & ((1u << w) - 1u));
        if (r >= lo) { r -= lo; x >>= w; pos += w; }
    }
    return pos;
}

template <int DC, typename Acc>
__device__ __forceinline__ int lottery_check_fast(const Acc &acc, const uint32_t *sp, const uint32_t *s_w, int W32,
                                                  int lane, uint64_t seed, uint64_t g, int it, int policy,
                                                  const float *lam, uint32_t &u2_out) {
    if (W32 <= 32 && lottery_random_check(policy)) {
        // At most 1024 checks, one word of U per lane: an inclusive scan gives
        // N and the lane holding the k-th member in ascending row order.
        // (Larger codes take lottery_check: a general walk here, inline or
        // out of line, measurably slowed the kernels on small codes.)
        const uint64_t r64 = splitmix64_at(seed, (g << 24) + static_cast<uint64_t>(it));
        const uint32_t word = lane < W32 ? (sp[lane] ^ s_w[lane]) : 0u;
        const uint32_t pc = __popc(word);
        uint32_t incl = pc;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t N = __shfl_sync(0xffffffffu, incl, 31);
        if (N == 0) return -1;
        u2_out = static_cast<uint32_t>(r64 >> 32);
        const uint32_t k = static_cast<uint32_t>((static_cast<uint64_t>(static_cast<uint32_t>(r64)) * N) >> 32);
        const bool mine = k >= incl - pc && k < incl;
        const int pick = mine ? lane * 32 + nth_set_bit(word, k - (incl - pc)) : 0;
        const unsigned own = __ballot_sync(0xffffffffu, mine);
        return __shfl_sync(0xffffffffu, pick, __ffs(own) - 1);
    }
    return lottery_check<DC>(acc, sp, s_w, W32, lane, seed, g, it, policy, lam, u2_out);
}

// Per-lane state between lottery_prepare and lottery_finish: lane k < DC
// holds c*'s slot-k column.
struct LotteryPrep {
    uint32_t vl;     // stored index of the column (acc.pad when absent)
    uint32_t ov;     // its id in H
    bool top;        // present, with the most unsatisfied checks among c*'s columns
    int fixed;       // the pick when it is already known (-1: none), else -2
};

template <int DC, int DV, typename Acc>
__device__ __forceinline__ LotteryPrep lottery_prepare(const Acc &acc, int cstar, uint32_t u2, const uint32_t *sp,
                                                       const uint32_t *s_w, int lane, int policy, int m, int R,
                                                       uint32_t magic) {
    LotteryPrep lp;
    lp.fixed = -2;
    lp.top = false;
    lp.vl = acc.pad;
    lp.ov = 0xffffffffu;
    if (cstar < 0) {
        lp.fixed = -1;
        return lp;
    }
    lp.vl = lane < DC ? acc.col(lane, cstar) : acc.pad;
    const bool present = lp.vl != acc.pad;
    lp.ov = present ? acc.orig(lp.vl) : 0xffffffffu;
    if (policy == LBP_LOTTERY_WORST_RANDOM || policy == LBP_LOTTERY_RANDOM_RANDOM) {
        const int deg = __popc(__ballot_sync(0xffffffffu, present));
        const int kk = static_cast<int>((static_cast<uint64_t>(u2) * static_cast<uint32_t>(deg)) >> 32);
        int rank = 0;
        #pragma unroll
        for (int o = 0; o < DC; ++o) {
            const uint32_t w = __shfl_sync(0xffffffffu, lp.ov, o);
            rank += (w < lp.ov) ? 1 : 0;
        }
        const unsigned pick = __ballot_sync(0xffffffffu, present && rank == kk);
        const int chosen = static_cast<int>(__shfl_sync(0xffffffffu, lp.vl, __ffs(pick) - 1));
        lp.fixed = pick ? chosen : -1;
        return lp;
    }
    uint32_t bc = 0;
    if (present && policy == LBP_LOTTERY_PROPOSED) {
        #pragma unroll
        for (int kk = 0; kk < DV; ++kk) {
            const uint32_t o = acc.ent(kk, lp.vl);
            const uint32_t r = o - __umulhi(o, magic) * static_cast<uint32_t>(R);
            if (o < acc.ent_end && r < static_cast<uint32_t>(m))
                bc += ((sp[r >> 5] ^ s_w[r >> 5]) >> (r & 31)) & 1u;
        }
    }
    const uint32_t key = present ? bc + 1u : 0u;
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
    lp.top = present && key == kmax;
    return lp;
}

__device__ __forceinline__ int lottery_finish(const LotteryPrep &lp, const float *lam) {
    if (lp.fixed != -2) return lp.fixed;
    const uint32_t ab = lp.top ? __float_as_uint(fabsf(lam[lp.vl])) : 0xffffffffu;
    const uint32_t amin = __reduce_min_sync(0xffffffffu, ab);
    const bool t1 = lp.top && ab == amin;
    const uint32_t oo = t1 ? lp.ov : 0xffffffffu;
    const uint32_t omin = __reduce_min_sync(0xffffffffu, oo);
    const unsigned win = __ballot_sync(0xffffffffu, t1 && oo == omin);
    const int chosen = static_cast<int>(__shfl_sync(0xffffffffu, lp.vl, __ffs(win) - 1));
    return win ? chosen : -1;
}

template <int DC, int DV, typename Acc>
__device__ __forceinline__ int lottery_pick(const Acc &acc, const uint32_t *sp, const uint32_t *s_w, int W32,
                                            int lane, uint64_t seed, uint64_t g, int it, int policy,
                                            const float *lam, int m, int R, uint32_t magic) {
    uint32_t u2 = 0;
    const int cstar = lottery_check<DC>(acc, sp, s_w, W32, lane, seed, g, it, policy, lam, u2);
    return lottery_column<DC, DV>(acc, cstar, u2, sp, s_w, lane, policy, lam, m, R, magic);
}

}  // namespace lbp
