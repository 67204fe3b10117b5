// K_bp (bounded degree): the Alg. 1 + Alg. 3 iteration of bp_kernel,
// specialised for codes whose checks have at most DC ones and whose columns
// at most DV ones (every surface-code space-time matrix: DC = 6, DV = 2; BB
// codes: DC = 6, DV = 3).
//
// Layout (all slot-major; uint16 indices, or uint32 for codes too large for
// 16-bit message offsets, whose image is then read from global memory):
//  * Check side: cidx[k][c] is the k-th column of check c (ascending), padded
//    with column n, whose prior and posterior are +inf: a neutral element of
//    the check update (positive sign, never the minimum).  beta[k][c], row
//    stride R = Mp + 2 (Mp = m rounded up to even), is the message on slot k.
//    When the index image always sits in shared memory, R is Mp + 2 rounded
//    up to a multiple of 32 words and a pair table orders the check phase
//    (bank-aware layout, built by lbp_load_code).
//  * Column side: vent[k][v] is the message offset k' * R + c of v's k-th
//    check (ascending), padded with offset Mp, the message beta[0][Mp] = +0
//    (x + 0 == x for every partial sum, which is never -0), so the LLR update
//    sums exactly the oracle's sequence of binary32 additions.  The check of
//    an offset, needed only by the syndrome scatter and the lottery, is
//    offset mod R by an exact multiply-high division.
//  * Each thread updates a pair of adjacent checks and a pair of adjacent
//    columns, so index, message, prior and posterior accesses are paired
//    32/64-bit accesses; an odd m or n gets one padding check / column.
// Check update per check: sign bits r_k = [alpha_k < 0] << 31 and their XOR
// t (with (-1)^{s_c}); exclusive minima of |alpha| from prefix and suffix
// minima; beta_k = f * excl_k carrying sign bit t ^ r_k.  Same values as the
// min1/min2/argmin form of bp_kernel, with fewer instructions.  The
// sum-product instantiation (kRule = LBP_RULE_SUM_PRODUCT) keeps the signs
// and replaces the minima by exclusive sums of phi(|alpha|) (prefix plus
// suffix, so no term is ever subtracted back out), beta_k = min(phi(excl_k),
// 25) with the same sign; the padding column (+inf) has phi = 0, still a
// neutral element.
// Placement: the graph image and each group's state sit in shared memory when
// they fit (kGraphSmem, kStateSmem); otherwise they are read from global
// memory (the image is L2-resident; the state goes to a per-group slice of the
// workspace).  A state slightly too large for shared memory (the d=25
// space-time code with binary32 messages) is split (kSplit): the posteriors,
// syndrome words and the first ks message slots stay in shared memory, the
// other slots go to the workspace.  The check phase moves those slots as
// coalesced pairs; the column phase gathers them, which for a space-time
// matrix touches only the measurement columns, whose messages of one round
// block are contiguous.
// Lottery: the group's last warp, which has the fewest rounds in both phases,
// runs it.  For the random-check policies it draws c* right after its
// check-phase rounds (c* depends only on s_hat(i-1), s and the draw).  The
// index-image instantiations in shared memory (kTab) draw with a single scan
// when the code has at most 1024 checks and also prepare c*'s columns then,
// so after the termination test only lottery_finish's |lambda| comparison
// remains; the other instantiations run lottery_column after the test.
// Everything else (groups of G threads per shot, named barriers, s_hat
// scatter, early termination, outputs, OSD hand-off) is as in bp_kernel.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "bp_common.cuh"
#include "bp_graph.cuh"
#include "bp_lottery.cuh"
#include "internal.h"

namespace lbp {

struct BpEllArgs {
    const uint8_t *image;     // ELL graph image (global)
    EllImage img;
    int32_t m, n;
    int32_t max_iter, scale_mode;
    float scale_const;
    int32_t lottery, lottery_skip, osd, policy, rule;
    uint64_t seed, shot_offset;
    int64_t num_shots;
    const uint64_t *syn;
    uint64_t *err;
    uint8_t *conv;
    uint8_t *osd_out;
    int32_t *iters;
    float *llr;
    unsigned int *counters;
    uint32_t *osd_list;
    float *osd_llr;
    uint32_t state_bytes;
    uint32_t off_beta, off_lam, off_s, off_shat, off_misc;
    uint8_t *gstate;          // per-group state slices when not in shared memory
    // Split state (kSplit): message slots [0, ks) live in shared memory with
    // the rest of the shot's state, slots [ks, DC) in a per-group workspace
    // slice of gbeta_bytes at gstate.
    int32_t ks;
    uint32_t gbeta_bytes;
    uint32_t magic;           // floor(2^32 / R) + 1: offset / R by multiply-high
    SurfaceDesc surf;         // implicit graph (SurfaceGraph)
    RoundDesc rnd;            // round-periodic graph (RoundGraph)
    const float *mu_tab;      // its mu[Np + 2] when not uniform per block
    // Index-image form with the bank-aware layout (0, 0 otherwise): message
    // row stride in words and the image offset of the check-pair table.
    int32_t tab_R;
    uint32_t off_ptab;
};

// Exclusive minima and signed outputs of one check (DC slots).
template <typename MsgT, int DC>
__device__ __forceinline__ void check_update(const float (&al)[DC], uint32_t sbit, float f,
                                             MsgT (&out)[DC]) {
    uint32_t r[DC];
    uint32_t tot = sbit << 31;
    #pragma unroll
    for (int k = 0; k < DC; ++k) {
        r[k] = al[k] < 0.0f ? 0x80000000u : 0u;
        tot ^= r[k];
    }
    float pre[DC], suf[DC];
    pre[0] = fabsf(al[0]);
    #pragma unroll
    for (int k = 1; k < DC; ++k) pre[k] = fminf(pre[k - 1], fabsf(al[k]));
    suf[DC - 1] = fabsf(al[DC - 1]);
    #pragma unroll
    for (int k = DC - 2; k >= 0; --k) suf[k] = fminf(suf[k + 1], fabsf(al[k]));
    #pragma unroll
    for (int k = 0; k < DC; ++k) {
        const float ex = k == 0 ? suf[1] : (k == DC - 1 ? pre[DC - 2] : fminf(pre[k - 1], suf[k + 1]));
        out[k] = Msg<MsgT>::store_signed(__fmul_rn(f, ex), tot ^ r[k]);
    }
}

// Sum-product form: exclusive sums of phi(|alpha|), beta_k = phi(excl_k)
// saturated at 25, sign as in the min-sum update.
template <typename MsgT, int DC>
__device__ __forceinline__ void check_update_sp(const float (&al)[DC], uint32_t sbit,
                                                MsgT (&out)[DC]) {
    uint32_t r[DC];
    uint32_t tot = sbit << 31;
    float ph[DC];
    #pragma unroll
    for (int k = 0; k < DC; ++k) {
        r[k] = al[k] < 0.0f ? 0x80000000u : 0u;
        tot ^= r[k];
        ph[k] = gallager_phi(fabsf(al[k]));
    }
    float pre[DC], suf[DC];
    pre[0] = ph[0];
    #pragma unroll
    for (int k = 1; k < DC; ++k) pre[k] = __fadd_rn(pre[k - 1], ph[k]);
    suf[DC - 1] = ph[DC - 1];
    #pragma unroll
    for (int k = DC - 2; k >= 0; --k) suf[k] = __fadd_rn(suf[k + 1], ph[k]);
    #pragma unroll
    for (int k = 0; k < DC; ++k) {
        const float ex = k == 0 ? suf[1] : (k == DC - 1 ? pre[DC - 2] : __fadd_rn(pre[k - 1], suf[k + 1]));
        out[k] = Msg<MsgT>::store_signed(fminf(gallager_phi(ex), kSpMaxMag), tot ^ r[k]);
    }
}

// A split state runs one shot per CTA, so its block is exactly G threads and
// the register budget follows G (64 per thread at 1024, 80 at 768, 128 at 512).
template <typename MsgT, int G, int DC, int DV, bool kGraphSmem, bool kStateSmem, typename GraphT,
          int kRule = LBP_RULE_MIN_SUM, bool kSplit = false>
__global__ void __launch_bounds__(kSplit ? G : 1024, 1) bp_ell_kernel(const BpEllArgs a) {
    static_assert(DC >= 2 && DC <= 8 && DV <= 8, "bounded degrees");
    static_assert(GraphT::kImage || !kGraphSmem, "an implicit graph has no image to stage");
    static_assert(!kSplit || (kStateSmem && !kGraphSmem), "a split state keeps its shared part beside a global image");
    using PairT = typename Pair<MsgT>::type;
    extern __shared__ __align__(16) uint8_t smem[];
    if (kGraphSmem) {
        const int4 *src = reinterpret_cast<const int4 *>(a.image);
        int4 *dst = reinterpret_cast<int4 *>(smem);
        const int words = static_cast<int>(a.img.bytes >> 4);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    const int m = a.m, n = a.n, I = a.max_iter;
    // The bank-aware layout exists only for the index image staged in shared
    // memory; every other instantiation keeps R = Mp + 2 and no pair table.
    constexpr bool kTab = kGraphSmem && GraphT::kEll;
    // Index image read from global memory: prefetch its words one trip ahead.
    constexpr bool kPf = !kGraphSmem && GraphT::kEll;
    const int Mp = a.img.Mp, Np = a.img.Np, R = (kTab && a.tab_R > 0) ? a.tab_R : Mp + 2;
    const uint16_t *ptab =
        (kTab && a.off_ptab != 0u) ? reinterpret_cast<const uint16_t *>(smem + a.off_ptab) : nullptr;
    const int mpairs = Mp >> 1, npairs = Np >> 1;
    const GraphT gr(a.img, kGraphSmem ? smem : a.image, a.surf, a.rnd, a.mu_tab, m, n);
    const uint32_t image_smem = kGraphSmem ? a.img.bytes : 0u;

    const int grp = threadIdx.x / G;
    const int t = threadIdx.x % G;
    const int lane = threadIdx.x & 31;
    const int bar = grp + 1;
    const int groups = blockDim.x / G;
    uint8_t *st = kStateSmem
        ? smem + image_smem + static_cast<size_t>(grp) * a.state_bytes
        : a.gstate + (static_cast<size_t>(blockIdx.x) * groups + grp) * a.state_bytes;
    // The group's shot counter slot always lives in shared memory.
    volatile uint32_t *misc = kStateSmem
        ? reinterpret_cast<volatile uint32_t *>(st + a.off_misc)
        : reinterpret_cast<volatile uint32_t *>(smem + image_smem + 16 * grp);
    MsgT *beta = reinterpret_cast<MsgT *>(st + a.off_beta);
    PairT *beta2 = reinterpret_cast<PairT *>(beta);
    // Message slots [ks, DC) of a split state: gbeta[(k - ks) * R + c].
    const int ks = kSplit ? a.ks : DC;
    const uint32_t ksR = static_cast<uint32_t>(ks) * static_cast<uint32_t>(R);
    MsgT *gbeta = kSplit ? reinterpret_cast<MsgT *>(a.gstate + (static_cast<size_t>(blockIdx.x) * groups + grp) *
                                                                  a.gbeta_bytes)
                         : nullptr;
    PairT *gbeta2 = reinterpret_cast<PairT *>(gbeta);
    float *lam = reinterpret_cast<float *>(st + a.off_lam);
    float2 *lam2 = reinterpret_cast<float2 *>(lam);
    uint32_t *s_w = reinterpret_cast<uint32_t *>(st + a.off_s);
    uint32_t *shat = reinterpret_cast<uint32_t *>(st + a.off_shat);
    if (t == 0) {
        beta[Mp] = Msg<MsgT>::store(0.0f);                // column-side padding message
        lam[n] = __int_as_float(0x7f800000);              // check-side padding column
    }
    __syncthreads();

    const int W32 = (m + 31) >> 5;
    const int wm64 = (m + 63) >> 6;
    const int wn64 = (n + 63) >> 6;
    const uint32_t last_mask = (m & 31) ? ((1u << (m & 31)) - 1u) : 0xffffffffu;

    while (true) {
        if (t == 0) misc[0] = atomicAdd(&a.counters[0], 1u);
        group_sync<G>(bar);
        const uint32_t b = misc[0];
        if (static_cast<int64_t>(b) >= a.num_shots) break;

        const uint32_t *syn32 = reinterpret_cast<const uint32_t *>(a.syn + static_cast<size_t>(b) * wm64);
        for (int w = t; w < W32; w += G) {
            uint32_t x = __ldg(syn32 + w);
            if (w == W32 - 1) x &= last_mask;
            s_w[w] = x;
            shat[w] = 0u;
            shat[W32 + w] = 0u;
            shat[2 * W32 + w] = 0u;
        }
        group_sync<G>(bar);

        int prev = 0, cur = 1, nxt = 2;
        bool converged = false;
        int it = 0;
        for (; it < I; ++it) {
            const float f = scale_at(a.scale_mode, a.scale_const, it);
            const bool lot = a.lottery && it >= a.lottery_skip && it < I - 1;
            // The group's last warp (the least loaded in both phases) runs the
            // lottery; a random check is drawn while the other warps finish
            // their check-phase rounds.
            const bool lw = t >= G - 32;
            const bool early = lottery_random_check(a.policy);
            int cpre = -1;
            uint32_t u2pre = 0;
            LotteryPrep lp;          // index-image instantiations in shared memory only
            // ---- C2V, two adjacent checks per thread ---------------------------
            // With the index image in global memory (L2), each trip's index
            // words are loaded one trip ahead, so their latency overlaps the
            // previous pair's work.
            typename GraphT::IP pfc[DC];
            if constexpr (kPf) {
                if (t < mpairs) gr.cols2_raw(t, pfc);
            }
            for (int ip = t; ip < mpairs; ip += G) {
                const int pr = (kTab && ptab) ? static_cast<int>(ptab[ip]) : ip;
                const int c = 2 * pr;
                float al0[DC], al1[DC];
                uint32_t v0[DC], v1[DC];
                if constexpr (kPf) {
                    GraphT::template unpack<DC>(pfc, v0, v1);
                    if (ip + G < mpairs) gr.cols2_raw(ip + G, pfc);
                } else {
                    gr.cols2(pr, v0, v1);
                }
                if (it == 0) {
                    #pragma unroll
                    for (int k = 0; k < DC; ++k) {
                        al0[k] = gr.mu(v0[k]);
                        al1[k] = gr.mu(v1[k]);
                    }
                } else {
                    #pragma unroll
                    for (int k = 0; k < DC; ++k) {
                        const PairT bb = (kSplit && k >= ks) ? gbeta2[(((k - ks) * R) >> 1) + pr]
                                                             : beta2[((k * R) >> 1) + pr];
                        al0[k] = __fsub_rn(lam[v0[k]], Msg<MsgT>::load(pair_lo<MsgT>(bb)));
                        al1[k] = __fsub_rn(lam[v1[k]], Msg<MsgT>::load(pair_hi<MsgT>(bb)));
                    }
                }
                const uint32_t sw = s_w[c >> 5];               // c even: c and c + 1 share a word
                MsgT o0[DC], o1[DC];
                if (kRule == LBP_RULE_SUM_PRODUCT) {
                    check_update_sp<MsgT, DC>(al0, (sw >> (c & 31)) & 1u, o0);
                    check_update_sp<MsgT, DC>(al1, (sw >> ((c & 31) + 1)) & 1u, o1);
                } else {
                    check_update<MsgT, DC>(al0, (sw >> (c & 31)) & 1u, f, o0);
                    check_update<MsgT, DC>(al1, (sw >> ((c & 31) + 1)) & 1u, f, o1);
                }
                #pragma unroll
                for (int k = 0; k < DC; ++k) {
                    if (kSplit && k >= ks) gbeta2[(((k - ks) * R) >> 1) + pr] = make_pair(o0[k], o1[k]);
                    else beta2[((k * R) >> 1) + pr] = make_pair(o0[k], o1[k]);
                }
            }
            if (lot && early && lw) {
                if constexpr (kTab) {
                    // c* and its columns now; after the termination test only
                    // the |lambda| comparison remains.
                    uint32_t u2 = 0;
                    const uint32_t *sp = shat + prev * W32;
                    const int cs = lottery_check_fast<DC>(gr, sp, s_w, W32, lane, a.seed, a.shot_offset + b, it,
                                                          a.policy, lam, u2);
                    lp = lottery_prepare<DC, DV>(gr, cs, u2, sp, s_w, lane, a.policy, m, R, a.magic);
                } else {
                    cpre = lottery_check<DC>(gr, shat + prev * W32, s_w, W32, lane, a.seed, a.shot_offset + b, it,
                                             a.policy, lam, u2pre);
                }
            }
            group_sync<G>(bar);
            // ---- LLR update, hard decision, syndrome scatter: column pairs ------
            uint32_t *sh_cur = shat + cur * W32;
            typename GraphT::IP pfe[DV];
            float2 pfm = make_float2(0.0f, 0.0f);
            if constexpr (kPf) {
                if (t < npairs) {
                    gr.ents2_raw(t, pfe);
                    pfm = gr.mu2_ldg(t);
                }
            }
            for (int q = t; q < npairs; q += G) {
                uint32_t e0[DV], e1[DV];
                float2 mm;
                if constexpr (kPf) {
                    GraphT::template unpack<DV>(pfe, e0, e1);
                    mm = pfm;
                    if (q + G < npairs) {
                        gr.ents2_raw(q + G, pfe);
                        pfm = gr.mu2_ldg(q + G);
                    }
                } else {
                    gr.ents2(q, e0, e1);
                    mm = gr.mu2(q);
                }
                float acc0 = mm.x, acc1 = mm.y;
                #pragma unroll
                for (int k = 0; k < DV; ++k) {
                    if (kSplit) {
                        const MsgT m0 = e0[k] >= ksR ? gbeta[e0[k] - ksR] : beta[e0[k]];
                        const MsgT m1 = e1[k] >= ksR ? gbeta[e1[k] - ksR] : beta[e1[k]];
                        acc0 = __fadd_rn(acc0, Msg<MsgT>::load(m0));
                        acc1 = __fadd_rn(acc1, Msg<MsgT>::load(m1));
                    } else {
                        acc0 = __fadd_rn(acc0, Msg<MsgT>::load(beta[e0[k]]));
                        acc1 = __fadd_rn(acc1, Msg<MsgT>::load(beta[e1[k]]));
                    }
                }
                lam2[q] = make_float2(acc0, acc1);
                if (acc0 <= 0.0f || acc1 <= 0.0f) {
                    #pragma unroll
                    for (int k = 0; k < DV; ++k) {
                        #pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if ((h == 0 ? acc0 : acc1) <= 0.0f) {
                                const unsigned o = h == 0 ? e0[k] : e1[k];
                                const unsigned r = o - __umulhi(o, a.magic) * static_cast<unsigned>(R);
                                if (r < static_cast<unsigned>(m)) atomicXor(&sh_cur[r >> 5], 1u << (r & 31));
                            }
                        }
                    }
                }
            }
            group_sync<G>(bar);
            // ---- early termination ------------------------------------------
            bool mism = false;
            uint32_t *sh_nxt = shat + nxt * W32;
            for (int w = t; w < W32; w += G) {
                mism |= (sh_cur[w] != s_w[w]);
                sh_nxt[w] = 0u;
            }
            if (!group_sync_or<G>(bar, mism)) { converged = true; break; }
            // ---- lottery (Alg. 3, or a baseline policy of Sec. III-B) ---------
            if (lot) {
                if (lw) {
                    const uint32_t *sp = shat + prev * W32;
                    if constexpr (kTab) {
                        if (!early) {
                            uint32_t u2 = 0;
                            const int cs = lottery_check_fast<DC>(gr, sp, s_w, W32, lane, a.seed, a.shot_offset + b,
                                                                  it, a.policy, lam, u2);
                            lp = lottery_prepare<DC, DV>(gr, cs, u2, sp, s_w, lane, a.policy, m, R, a.magic);
                        }
                        const int vs = lottery_finish(lp, lam);
                        if (lane == 0 && vs >= 0) lam[vs] = -lam[vs];
                    } else {
                        if (!early)
                            cpre = lottery_check<DC>(gr, sp, s_w, W32, lane, a.seed, a.shot_offset + b, it, a.policy,
                                                     lam, u2pre);
                        const int vs = lottery_column<DC, DV>(gr, cpre, u2pre, sp, s_w, lane, a.policy, lam, m, R,
                                                              a.magic);
                        if (lane == 0 && vs >= 0) lam[vs] = -lam[vs];
                    }
                }
                group_sync<G>(bar);
            }
            const int tmp = prev; prev = cur; cur = nxt; nxt = tmp;
        }

        // ---- results ------------------------------------------------------------
        {
            const int nw = G / 32;
            const int gw = t >> 5;
            uint32_t *err32 = reinterpret_cast<uint32_t *>(a.err + static_cast<size_t>(b) * wn64);
            for (int w = gw; w < 2 * wn64; w += nw) {
                const int v = w * 32 + lane;
                const bool e = (v < n) && (lam[v] <= 0.0f);
                const unsigned bits = __ballot_sync(0xffffffffu, e);
                if (lane == 0) err32[w] = bits;
            }
            if (a.llr) {
                float *dst = a.llr + static_cast<size_t>(b) * n;
                for (int v = t; v < n; v += G) dst[v] = lam[v];
            }
            if (t == 0) {
                a.conv[b] = converged ? 1 : 0;
                a.iters[b] = converged ? it + 1 : I;
                if (a.osd_out) a.osd_out[b] = LBP_OSD_NOT_RUN;
            }
            if (!converged && a.osd) {
                if (t == 0) {
                    const uint32_t slot = atomicAdd(&a.counters[1], 1u);
                    a.osd_list[slot] = b;
                    misc[1] = slot;
                }
                group_sync<G>(bar);
                float *dst = a.osd_llr + static_cast<size_t>(misc[1]) * n;
                for (int v = t; v < n; v += G) dst[v] = lam[v];
            }
        }
        group_sync<G>(bar);
    }
}

}  // namespace lbp
