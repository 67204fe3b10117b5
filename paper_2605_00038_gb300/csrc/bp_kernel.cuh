// K_bp: normalised min-sum BP with the lottery sign flip, one shot per
// thread group, the whole Tanner graph and every shot's messages resident in
// shared memory.
//
// Alg. 1 (per iteration i, per shot):
//   V2C   alpha_{v->c} = mu_v (i = 0) or lambda_v - beta_{v<-c}
//   C2V   beta_{v<-c} = (-1)^{s_c} f_i prod_{v' != v} sign(alpha) min_{v' != v} |alpha|
//   LLR   lambda_v = mu_v + sum_{c in C(v)} beta_{v<-c}   (rows ascending)
//   HD    e_v = [lambda_v <= 0];  s_hat = H e (mod 2);  stop when s_hat == s
// Alg. 3 (lottery, lottery_skip <= i < I-1, shot not converged):
//   U = s_hat(i-1) xor s, c* = k-th member of U with k = floor(u |U| / 2^32),
//   v* = argmax_{v in V(c*)} |C(v) ∩ U|, then min |lambda_v|, then lowest v;
//   lambda_{v*} <- -lambda_{v*}.
//
// Layout and schedule (GB300):
//  * One CTA per SM (persistent).  It copies the compact 16-bit graph image
//    (CSR + CSC + mu) into shared memory once and keeps it for every shot.
//  * The CTA hosts S independent groups of G threads; each group decodes one
//    shot at a time, fetched from a global atomic counter, so early-exiting
//    shots free their group immediately.  Groups synchronise with named
//    barriers (bar.sync id, G), never with the whole CTA.
//  * A group's per-shot state lives in shared memory: beta[E] (message type
//    MsgT), lambda[n] f32, s and three rolling s_hat bit buffers.  Nothing of
//    the iteration touches global memory: DRAM traffic per shot is the
//    syndrome in and the results out.
//  * C2V: a thread owns whole checks; one pass over the check's edges keeps
//    min1, min2, the argmin slot and the sign parity (the exclusive minimum
//    is min2 at the argmin slot and min1 elsewhere), a second pass writes
//    beta.  LLR: a thread owns whole columns and sums in ascending row order,
//    which fixes the binary32 rounding sequence; the columns with
//    lambda <= 0 scatter their checks into s_hat with shared-memory XOR
//    atomics (few columns are in error, so this is cheap).
//  * Convergence: s_hat == s word by word, OR-reduced by the barrier itself
//    (bar.red.or.pred).  The lottery runs in the group's first warp:
//    ballot/popc prefix sums pick c*, one lane per neighbour counts
//    |C(v) ∩ U| and a shuffle reduction picks v*.
//  * The sum-product rule (a.rule) replaces the minima by exclusive sums of
//    Gallager's phi(|alpha|) and beta = phi(sum), saturated at 25.
//  * All arithmetic is explicit round-to-nearest binary32 (__fadd_rn,
//    __fsub_rn, __fmul_rn; the library builds with -fmad=false), so results
//    are bit-reproducible.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "bp_common.cuh"
#include "internal.h"

namespace lbp {

struct BpArgs {
    const uint8_t *image;     // compact graph image (global), copied to shared memory
    GraphImage img;
    int32_t m, n;
    int32_t max_iter, scale_mode;
    float scale_const;
    int32_t lottery, lottery_skip, osd, policy, rule;
    uint64_t seed, shot_offset;
    int64_t num_shots;
    const uint64_t *syn;      // [B][wm64]
    uint64_t *err;            // [B][wn64]
    uint8_t *conv;            // [B]
    uint8_t *osd_out;         // [B] or null
    int32_t *iters;           // [B]
    float *llr;               // [B][n] or null
    unsigned int *counters;   // [0] shot counter, [1] OSD queue length
    uint32_t *osd_list;       // [B] shot ids handed to OSD
    float *osd_llr;           // [B][n] their final lambda
    uint32_t state_bytes;     // per group
    uint32_t off_beta, off_lam, off_s, off_shat, off_misc;
};

// ------------------------------------------------------------------ kernel

template <typename MsgT, int G>
__global__ void __launch_bounds__(1024, 1) bp_kernel(const BpArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    // Stage the graph image once per CTA.
    {
        const int4 *src = reinterpret_cast<const int4 *>(a.image);
        int4 *dst = reinterpret_cast<int4 *>(smem);
        const int words = static_cast<int>(a.img.bytes >> 4);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();

    const uint16_t *row_ptr = reinterpret_cast<const uint16_t *>(smem + a.img.off_row_ptr);
    const uint16_t *col_idx = reinterpret_cast<const uint16_t *>(smem + a.img.off_col_idx);
    const uint16_t *col_ptr = reinterpret_cast<const uint16_t *>(smem + a.img.off_col_ptr);
    const uint16_t *csc_edge = reinterpret_cast<const uint16_t *>(smem + a.img.off_csc_edge);
    const uint16_t *csc_row = reinterpret_cast<const uint16_t *>(smem + a.img.off_csc_row);
    const float *mu = reinterpret_cast<const float *>(smem + a.img.off_mu);

    const int grp = threadIdx.x / G;
    const int t = threadIdx.x % G;
    const int lane = threadIdx.x & 31;
    const int bar = grp + 1;
    uint8_t *st = smem + a.img.bytes + static_cast<size_t>(grp) * a.state_bytes;
    MsgT *beta = reinterpret_cast<MsgT *>(st + a.off_beta);
    float *lam = reinterpret_cast<float *>(st + a.off_lam);
    uint32_t *s_w = reinterpret_cast<uint32_t *>(st + a.off_s);
    uint32_t *shat = reinterpret_cast<uint32_t *>(st + a.off_shat);
    volatile uint32_t *misc = reinterpret_cast<volatile uint32_t *>(st + a.off_misc);

    const int m = a.m, n = a.n, I = a.max_iter;
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

        int prev = 0, cur = 1, nxt = 2;   // s_hat(i-1), s_hat(i), next
        bool converged = false;
        int it = 0;
        for (; it < I; ++it) {
            const float f = scale_at(a.scale_mode, a.scale_const, it);
            // ---- C2V (check-node update) --------------------------------
            for (int c = t; c < m && a.rule == LBP_RULE_SUM_PRODUCT; c += G) {
                // Sum-product: exclusive sums of phi(|alpha|) from prefix sums
                // and a running suffix sum (deg <= 32), in the same order of
                // binary32 additions as the bounded-degree kernel.
                const int e0 = row_ptr[c];
                const int deg = row_ptr[c + 1] - e0;
                unsigned parity = (s_w[c >> 5] >> (c & 31)) & 1u;
                unsigned negmask = 0u;
                float ph[32], pre[32];
                for (int k = 0; k < deg; ++k) {
                    const int v = col_idx[e0 + k];
                    const float al = (it == 0) ? mu[v] : __fsub_rn(lam[v], Msg<MsgT>::load(beta[e0 + k]));
                    if (al < 0.0f) { negmask |= 1u << k; parity ^= 1u; }
                    ph[k] = gallager_phi(fabsf(al));
                    pre[k] = k == 0 ? ph[0] : __fadd_rn(pre[k - 1], ph[k]);
                }
                float suf = 0.0f;
                for (int k = deg - 1; k >= 0; --k) {
                    const float ex = k == deg - 1 ? pre[deg - 2] : (k == 0 ? suf : __fadd_rn(pre[k - 1], suf));
                    suf = k == deg - 1 ? ph[k] : __fadd_rn(suf, ph[k]);
                    const uint32_t sg = ((parity ^ (negmask >> k)) & 1u) << 31;
                    beta[e0 + k] = Msg<MsgT>::store_signed(fminf(gallager_phi(ex), kSpMaxMag), sg);
                }
            }
            for (int c = t; c < m && a.rule != LBP_RULE_SUM_PRODUCT; c += G) {
                const int e0 = row_ptr[c];
                const int deg = row_ptr[c + 1] - e0;
                unsigned parity = (s_w[c >> 5] >> (c & 31)) & 1u;   // (-1)^{s_c}
                unsigned negmask = 0u;
                float min1 = __int_as_float(0x7f800000), min2 = min1;
                int pos = 0;
                for (int k = 0; k < deg; ++k) {
                    const int v = col_idx[e0 + k];
                    const float al = (it == 0) ? mu[v] : __fsub_rn(lam[v], Msg<MsgT>::load(beta[e0 + k]));
                    if (al < 0.0f) { negmask |= 1u << k; parity ^= 1u; }
                    const float aa = fabsf(al);
                    if (aa < min1) { min2 = min1; min1 = aa; pos = k; }
                    else if (aa < min2) { min2 = aa; }
                }
                const float m1 = __fmul_rn(f, min1);
                const float m2 = __fmul_rn(f, min2);
                for (int k = 0; k < deg; ++k) {
                    const float mag = (k == pos) ? m2 : m1;
                    const bool neg = (parity ^ (negmask >> k)) & 1u;
                    beta[e0 + k] = Msg<MsgT>::store(neg ? -mag : mag);
                }
            }
            group_sync<G>(bar);
            // ---- LLR update, hard decision, syndrome scatter ----------------
            uint32_t *sh_cur = shat + cur * W32;
            for (int v = t; v < n; v += G) {
                const int j0 = col_ptr[v], j1 = col_ptr[v + 1];
                float acc = mu[v];
                for (int j = j0; j < j1; ++j) acc = __fadd_rn(acc, Msg<MsgT>::load(beta[csc_edge[j]]));
                lam[v] = acc;
                if (acc <= 0.0f) {
                    for (int j = j0; j < j1; ++j) {
                        const int r = csc_row[j];
                        atomicXor(&sh_cur[r >> 5], 1u << (r & 31));
                    }
                }
            }
            group_sync<G>(bar);
            // ---- early termination check ---------------------------------
            bool mism = false;
            uint32_t *sh_nxt = shat + nxt * W32;
            for (int w = t; w < W32; w += G) {
                mism |= (sh_cur[w] != s_w[w]);
                sh_nxt[w] = 0u;
            }
            if (!group_sync_or<G>(bar, mism)) { converged = true; break; }
            // ---- lottery (Alg. 3, or a baseline policy of Sec. III-B) ---------
            if (a.lottery && it >= a.lottery_skip && it < I - 1) {
                if (t < 32) {
                    // The ablation policy draws like Alg. 3 from this iteration's s_hat.
                    const bool cur_u = a.policy == LBP_LOTTERY_PROPOSED_CURRENT;
                    const int pol = cur_u ? LBP_LOTTERY_PROPOSED : a.policy;
                    const uint32_t *sp = cur_u ? sh_cur : shat + prev * W32;
                    uint32_t N = 0;
                    for (int w0 = 0; w0 < W32; w0 += 32) {
                        const int w = w0 + lane;
                        const uint32_t word = (w < W32) ? (sp[w] ^ s_w[w]) : 0u;
                        uint32_t pc = __popc(word);
                        #pragma unroll
                        for (int o = 16; o > 0; o >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, o);
                        N += pc;
                    }
                    if (N > 0) {
                        const uint64_t g = a.shot_offset + b;
                        const uint64_t r64 = splitmix64_at(a.seed, (g << 24) + static_cast<uint64_t>(it));
                        const uint32_t u = static_cast<uint32_t>(r64), u2 = static_cast<uint32_t>(r64 >> 32);
                        int cstar = -1;
                        if (pol == LBP_LOTTERY_WORST_UNRELIABLE || pol == LBP_LOTTERY_WORST_RANDOM) {
                            // Worst CN: most columns estimated in error, lowest row on ties.
                            int bn = -1, bcr = 0x7fffffff;
                            for (int w = lane; w < W32; w += 32) {
                                uint32_t word = sp[w] ^ s_w[w];
                                while (word) {
                                    const int c = w * 32 + __ffs(word) - 1;
                                    word &= word - 1u;
                                    int ne = 0;
                                    for (int e = row_ptr[c]; e < row_ptr[c + 1]; ++e)
                                        ne += lam[col_idx[e]] <= 0.0f ? 1 : 0;
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
                            // Random CN: member k = floor(u N / 2^32) of U, ascending rows.
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
                        int bc = -1, bv = 0x7fffffff;
                        float ba = 0.0f;
                        if (pol == LBP_LOTTERY_WORST_RANDOM || pol == LBP_LOTTERY_RANDOM_RANDOM) {
                            // Random VN: column floor(u2 deg / 2^32) of c*.
                            const int e0 = row_ptr[cstar];
                            const int deg = row_ptr[cstar + 1] - e0;
                            const int kk = static_cast<int>((static_cast<uint64_t>(u2) * static_cast<uint32_t>(deg)) >> 32);
                            bv = col_idx[e0 + kk];
                            bc = 0;
                        } else {
                            // Unreliable VN (the proposed rule first prefers the column
                            // with the most unsatisfied checks), then lowest column.
                            const int e0 = row_ptr[cstar];
                            const int deg = row_ptr[cstar + 1] - e0;
                            if (lane < deg) {
                                bv = col_idx[e0 + lane];
                                bc = 0;
                                if (pol == LBP_LOTTERY_PROPOSED) {
                                    for (int j = col_ptr[bv]; j < col_ptr[bv + 1]; ++j) {
                                        const int r = csc_row[j];
                                        bc += ((sp[r >> 5] ^ s_w[r >> 5]) >> (r & 31)) & 1u;
                                    }
                                }
                                ba = fabsf(lam[bv]);
                            }
                            #pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
                                const float oa = __shfl_xor_sync(0xffffffffu, ba, o);
                                const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
                                const bool better = oc > bc || (oc == bc && (oa < ba || (oa == ba && ov < bv)));
                                if (better) { bc = oc; ba = oa; bv = ov; }
                            }
                        }
                        if (lane == 0 && bc >= 0) lam[bv] = -lam[bv];
                    }
                }
                group_sync<G>(bar);
            }
            const int tmp = prev; prev = cur; cur = nxt; nxt = tmp;
        }

        // ---- results ----------------------------------------------------------
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
