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
// syndrome words and the first DC - 2 message slots stay in shared memory,
// the last two slots go to the workspace.  The check phase moves those slots
// as coalesced pairs; with the slot-aligned image of a space-time matrix
// they hold exactly the measurement columns' messages, so the column phase
// reads each column's messages from one place (those of one round block are
// contiguous).
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
    // Split state (kSplit): message slots [0, DC - 2) live in shared memory
    // with the rest of the shot's state, the last two slots in a per-group
    // workspace slice of gbeta_bytes at gstate.
    uint32_t gbeta_bytes;
    uint32_t magic;           // floor(2^32 / R) + 1: offset / R by multiply-high
    SurfaceDesc surf;         // implicit graph (SurfaceGraph)
    RoundDesc rnd;            // round-periodic graph (RoundGraph)
    const float *mu_tab;      // its mu[Np + 2] when not uniform per block
    // Index-image form with the bank-aware layout (0, 0 otherwise): message
    // row stride in words and the image offset of the check-pair table.
    int32_t tab_R;
    uint32_t off_ptab;
    // Merged launch (kMulti): the launch's arguments hold the claim counter
    // (counters[0]), the total shot count (num_shots), the largest state
    // (state_bytes) and the items; each item is a whole BpEllArgs of its own
    // code, parameters and buffers, whose shots are the launch's work indices
    // [first, first + num_shots).
    const BpEllArgs *items;
    int32_t n_items;
    int64_t first;
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
// A merged launch (kMulti) decodes the shots of several codes of the same
// degree bounds: each group claims the next work index, finds its item (a
// binary search over the items' first indices) and decodes that shot with the
// item's image (read from global memory, L2-resident), parameters and
// buffers; every code-dependent value is rebound per shot, and the group's
// shared-memory state is sized for the largest code.
template <typename MsgT, int G, int DC, int DV, bool kGraphSmem, bool kStateSmem, typename GraphT,
          int kRule = LBP_RULE_MIN_SUM, bool kSplit = false, bool kMulti = false>
__global__ void __launch_bounds__(kSplit ? G : 1024, 1) bp_ell_kernel(const BpEllArgs a) {
    static_assert(DC >= 2 && DC <= 8 && DV <= 8, "bounded degrees");
    static_assert(GraphT::kImage || !kGraphSmem, "an implicit graph has no image to stage");
    static_assert(!kSplit || (kStateSmem && !kGraphSmem), "a split state keeps its shared part beside a global image");
    static_assert(!kMulti || (GraphT::kEll && !kGraphSmem && kStateSmem && !kSplit),
                  "a merged launch reads its images from global memory and keeps its states in shared memory");
    using PairT = typename Pair<MsgT>::type;
    // Message slots a split state keeps in shared memory: all but the last two
    // (which a slot-aligned space-time image reserves for the measurement
    // columns).
    constexpr int kKs = kSplit ? DC - 2 : DC;
    extern __shared__ __align__(16) uint8_t smem[];
    if (kGraphSmem) {
        const int4 *src = reinterpret_cast<const int4 *>(a.image);
        int4 *dst = reinterpret_cast<int4 *>(smem);
        const int words = static_cast<int>(a.img.bytes >> 4);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    // The shot's item in a merged launch; LBP_ARG(f) is the argument f of the
    // shot being decoded (the launch's own arguments otherwise).
    const BpEllArgs *item = nullptr;
#define LBP_ARG(f) (kMulti ? item->f : a.f)
    // The bank-aware layout exists only for the index image staged in shared
    // memory; every other instantiation keeps R = Mp + 2 and no pair table.
    constexpr bool kTab = kGraphSmem && GraphT::kEll;
    // Index image read from global memory: prefetch its words one trip ahead.
    constexpr bool kPf = !kGraphSmem && GraphT::kEll;
    const uint32_t image_smem = kGraphSmem ? a.img.bytes : 0u;

    const int grp = threadIdx.x / G;
    const int t = threadIdx.x % G;
    const int lane = threadIdx.x & 31;
    const int bar = grp + 1;
    const int groups = blockDim.x / G;
    // A merged launch keeps the groups' shot slots ahead of their states.
    const uint32_t misc_smem = kMulti ? 16u * static_cast<uint32_t>(groups) : 0u;
    uint8_t *st = kStateSmem
        ? smem + image_smem + misc_smem + static_cast<size_t>(grp) * a.state_bytes
        : a.gstate + (static_cast<size_t>(blockIdx.x) * groups + grp) * a.state_bytes;
    // The group's shot counter slot always lives in shared memory.
    volatile uint32_t *misc = (kStateSmem && !kMulti)
        ? reinterpret_cast<volatile uint32_t *>(st + a.off_misc)
        : reinterpret_cast<volatile uint32_t *>(smem + image_smem + 16 * grp);
    // Message slots [ks, DC) of a split state: gbeta[(k - ks) * R + c].
    MsgT *gbeta = kSplit ? reinterpret_cast<MsgT *>(a.gstate + (static_cast<size_t>(blockIdx.x) * groups + grp) *
                                                                  a.gbeta_bytes)
                         : nullptr;
    PairT *gbeta2 = reinterpret_cast<PairT *>(gbeta);

    // Code-dependent values: bound once, or per shot in a merged launch.
    int m, n, I, Mp, Np, R, mpairs, npairs, ks, W32, wm64, wn64;
    uint32_t ksR, last_mask;
    const uint16_t *ptab;
    MsgT *beta;
    PairT *beta2;
    float *lam;
    float2 *lam2;
    uint32_t *s_w, *shat;
    GraphT gr(a.img, kGraphSmem ? smem : a.image, a.surf, a.rnd, a.mu_tab, a.m, a.n);
    auto bind = [&]() {
        m = LBP_ARG(m);
        n = LBP_ARG(n);
        I = LBP_ARG(max_iter);
        Mp = LBP_ARG(img.Mp);
        Np = LBP_ARG(img.Np);
        // The message row stride the image's offsets were built with: the
        // bank-aware stride when the code has one (a merged launch reads such
        // an image from global memory, without its pair table), else Mp + 2.
        R = ((kTab || kMulti) && LBP_ARG(tab_R) > 0) ? LBP_ARG(tab_R) : Mp + 2;
        ptab = (kTab && a.off_ptab != 0u) ? reinterpret_cast<const uint16_t *>(smem + a.off_ptab) : nullptr;
        mpairs = Mp >> 1;
        npairs = Np >> 1;
        if constexpr (kMulti) gr = GraphT(item->img, item->image, item->surf, item->rnd, item->mu_tab, m, n);
        beta = reinterpret_cast<MsgT *>(st + LBP_ARG(off_beta));
        beta2 = reinterpret_cast<PairT *>(beta);
        ks = kKs;
        ksR = static_cast<uint32_t>(ks) * static_cast<uint32_t>(R);
        lam = reinterpret_cast<float *>(st + LBP_ARG(off_lam));
        lam2 = reinterpret_cast<float2 *>(lam);
        s_w = reinterpret_cast<uint32_t *>(st + LBP_ARG(off_s));
        shat = reinterpret_cast<uint32_t *>(st + LBP_ARG(off_shat));
        W32 = (m + 31) >> 5;
        wm64 = (m + 63) >> 6;
        wn64 = (n + 63) >> 6;
        last_mask = (m & 31) ? ((1u << (m & 31)) - 1u) : 0xffffffffu;
    };
    if constexpr (!kMulti) {
        bind();
        if (t == 0) {
            beta[Mp] = Msg<MsgT>::store(0.0f);                // column-side padding message
            lam[n] = __int_as_float(0x7f800000);              // check-side padding column
        }
    }
    __syncthreads();

    while (true) {
        if (t == 0) misc[0] = atomicAdd(&a.counters[0], 1u);
        group_sync<G>(bar);
        uint32_t b = misc[0];
        if (static_cast<int64_t>(b) >= a.num_shots) break;
        if constexpr (kMulti) {
            int lo = 0, hi = a.n_items - 1;              // last item with first <= b
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.items[mid].first <= static_cast<int64_t>(b)) lo = mid;
                else hi = mid - 1;
            }
            item = a.items + lo;
            b -= static_cast<uint32_t>(item->first);
            bind();
            if (t == 0) {
                beta[Mp] = Msg<MsgT>::store(0.0f);
                lam[n] = __int_as_float(0x7f800000);
            }
        }

        const uint32_t *syn32 = reinterpret_cast<const uint32_t *>(LBP_ARG(syn) + static_cast<size_t>(b) * wm64);
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
            const float f = scale_at(LBP_ARG(scale_mode), LBP_ARG(scale_const), it);
            const bool lot = LBP_ARG(lottery) && it >= LBP_ARG(lottery_skip) && it < I - 1;
            // The group's last warp (the least loaded in both phases) runs the
            // lottery; a random check is drawn while the other warps finish
            // their check-phase rounds.
            const bool lw = t >= G - 32;
            // (The ablation policy, U from this iteration's s_hat, exists in the
            // shared-image form only and draws after the column phase.)
            const bool early = lottery_random_check(LBP_ARG(policy)) &&
                               !(kTab && LBP_ARG(policy) == LBP_LOTTERY_PROPOSED_CURRENT);
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
                    const int cs = lottery_check_fast<DC>(gr, sp, s_w, W32, lane, LBP_ARG(seed), LBP_ARG(shot_offset) + b, it,
                                                          LBP_ARG(policy), lam, u2);
                    lp = lottery_prepare<DC, DV>(gr, cs, u2, sp, s_w, lane, LBP_ARG(policy), m, R, LBP_ARG(magic));
                } else {
                    cpre = lottery_check<DC>(gr, shat + prev * W32, s_w, W32, lane, LBP_ARG(seed), LBP_ARG(shot_offset) + b, it,
                                             LBP_ARG(policy), lam, u2pre);
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
            // A split state over a slot-aligned image: column pairs below
            // q_lo have every message in shared memory, pairs in [q_hi, q_end)
            // every message in the workspace; the one or two pairs between
            // (a round and a measurement column, or the padding column) pick
            // per message.  Without the aligned layout every pair picks.
            const int meas0 = kSplit ? LBP_ARG(img.meas0) : 0;
            const int q_lo = meas0 > 0 ? meas0 >> 1 : 0;
            const int q_hi = meas0 > 0 ? (meas0 + 1) >> 1 : npairs;
            const int q_end = meas0 > 0 ? n >> 1 : npairs;
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
                if (kSplit && q >= q_lo) {
                    if (q >= q_hi && q < q_end) {
                        #pragma unroll
                        for (int k = 0; k < DV; ++k) {
                            acc0 = __fadd_rn(acc0, Msg<MsgT>::load(gbeta[e0[k] - ksR]));
                            acc1 = __fadd_rn(acc1, Msg<MsgT>::load(gbeta[e1[k] - ksR]));
                        }
                    } else {
                        #pragma unroll
                        for (int k = 0; k < DV; ++k) {
                            const MsgT m0 = e0[k] >= ksR ? gbeta[e0[k] - ksR] : beta[e0[k]];
                            const MsgT m1 = e1[k] >= ksR ? gbeta[e1[k] - ksR] : beta[e1[k]];
                            acc0 = __fadd_rn(acc0, Msg<MsgT>::load(m0));
                            acc1 = __fadd_rn(acc1, Msg<MsgT>::load(m1));
                        }
                    }
                } else {
                    #pragma unroll
                    for (int k = 0; k < DV; ++k) {
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
                                const unsigned r = o - __umulhi(o, LBP_ARG(magic)) * static_cast<unsigned>(R);
                                if (r < static_cast<unsigned>(m)) atomicXor(&sh_cur[r >> 5], 1u << (r & 31));
                            }
                        }
                    }
                }
            }
            group_sync<G>(bar);
            // ---- lottery (Alg. 3, or a baseline policy of Sec. III-B) ---------
            // Index-image instantiations in shared memory (kTab): the lottery's
            // inputs (s_hat(i-1), s, lambda(i)) are complete here, so the
            // lottery warp picks and flips v* now, alongside the termination
            // test, whose barrier also orders the flip before the next check
            // phase; if the shot has converged the flip is undone before the
            // results read lambda.  The other instantiations run the lottery
            // after the test, behind a barrier of its own.
            int vflip = -1;
            if constexpr (kTab) {
                if (lot && lw) {
                    const uint32_t *sp = shat + prev * W32;
                    if (!early) {
                        // The ablation policy draws like Alg. 3 from this
                        // iteration's s_hat (and is not drawn early).
                        const bool cur_u = LBP_ARG(policy) == LBP_LOTTERY_PROPOSED_CURRENT;
                        if (cur_u) sp = sh_cur;
                        const int pol = cur_u ? LBP_LOTTERY_PROPOSED : LBP_ARG(policy);
                        uint32_t u2 = 0;
                        const int cs = lottery_check_fast<DC>(gr, sp, s_w, W32, lane, LBP_ARG(seed), LBP_ARG(shot_offset) + b,
                                                              it, pol, lam, u2);
                        lp = lottery_prepare<DC, DV>(gr, cs, u2, sp, s_w, lane, pol, m, R, LBP_ARG(magic));
                    }
                    vflip = lottery_finish(lp, lam);
                    if (lane == 0 && vflip >= 0) lam[vflip] = -lam[vflip];
                }
            }
            // ---- early termination ------------------------------------------
            bool mism = false;
            uint32_t *sh_nxt = shat + nxt * W32;
            for (int w = t; w < W32; w += G) {
                mism |= (sh_cur[w] != s_w[w]);
                sh_nxt[w] = 0u;
            }
            if (!group_sync_or<G>(bar, mism)) {
                if constexpr (kTab) {
                    if (lane == 0 && vflip >= 0) lam[vflip] = -lam[vflip];
                    group_sync<G>(bar);
                }
                converged = true;
                break;
            }
            if constexpr (!kTab) {
                if (lot) {
                    if (lw) {
                        const uint32_t *sp = shat + prev * W32;
                        if (!early)
                            cpre = lottery_check<DC>(gr, sp, s_w, W32, lane, LBP_ARG(seed), LBP_ARG(shot_offset) + b, it,
                                                     LBP_ARG(policy), lam, u2pre);
                        const int vs = lottery_column<DC, DV>(gr, cpre, u2pre, sp, s_w, lane, LBP_ARG(policy), lam, m, R,
                                                              LBP_ARG(magic));
                        if (lane == 0 && vs >= 0) lam[vs] = -lam[vs];
                    }
                    group_sync<G>(bar);
                }
            }
            const int tmp = prev; prev = cur; cur = nxt; nxt = tmp;
        }

        // ---- results ------------------------------------------------------------
        {
            const int nw = G / 32;
            const int gw = t >> 5;
            uint32_t *err32 = reinterpret_cast<uint32_t *>(LBP_ARG(err) + static_cast<size_t>(b) * wn64);
            for (int w = gw; w < 2 * wn64; w += nw) {
                const int v = w * 32 + lane;
                const bool e = (v < n) && (lam[v] <= 0.0f);
                const unsigned bits = __ballot_sync(0xffffffffu, e);
                if (lane == 0) err32[w] = bits;
            }
            if (LBP_ARG(llr)) {
                float *dst = LBP_ARG(llr) + static_cast<size_t>(b) * n;
                for (int v = t; v < n; v += G) dst[v] = lam[v];
            }
            if (t == 0) {
                LBP_ARG(conv)[b] = converged ? 1 : 0;
                LBP_ARG(iters)[b] = converged ? it + 1 : I;
                if (LBP_ARG(osd_out)) LBP_ARG(osd_out)[b] = LBP_OSD_NOT_RUN;
            }
            if (!converged && LBP_ARG(osd)) {
                if (t == 0) {
                    const uint32_t slot = atomicAdd(&LBP_ARG(counters)[1], 1u);
                    LBP_ARG(osd_list)[slot] = b;
                    misc[1] = slot;
                }
                group_sync<G>(bar);
                float *dst = LBP_ARG(osd_llr) + static_cast<size_t>(misc[1]) * n;
                for (int v = t; v < n; v += G) dst[v] = lam[v];
            }
        }
        group_sync<G>(bar);
    }
#undef LBP_ARG
}

}  // namespace lbp
