// K_osd_warp: OSD-0 (Alg. 2), one warp per shot, exploiting that H stays
// sparse during the elimination.
//
// Per shot:
//  1. LLR sorting: warp bitonic sort of 64-bit keys (order-preserving bits of
//     lambda, column) gives pi: perm[j] = column at position j, inv = pi^-1.
//  2. Basis selection with the L/U factorisation folded in (forward
//     elimination in permuted column order): at position j the candidates are
//     the non-pivot rows with a one there.  The lowest such row becomes the
//     pivot of j (so j joins the basis S, the first rank(H) independent
//     columns) and every other candidate is replaced by its sum with the
//     pivot row, syndrome bit included (forward substitution).  Non-pivot
//     rows never hold a one left of j, so "row r has a one at j" is "j is
//     r's lowest position".
//  3. Backward substitution over the pivots in reverse order:
//     e_S[k] = s'[p_k] xor <row p_k, e_S at later positions>; positions
//     outside S are zero; the estimate maps back through pi.
// A row that no elimination touched is still a row of H: its ones are the
// positions inv[v] of its columns, read from the CSR image in shared memory.
// Only rows that an elimination changes get a dense 64-bit copy, from a
// per-warp pool of C rows in the workspace (measured: about 40 rows per shot
// on the d=11 space-time code, 35 on BB [[144,12,12]]).  A shot that needs
// more than C dense rows is handed to the block-wide kernel K_osd unchanged.
#pragma once

#include <cstdint>

#include "internal.h"

namespace lbp {

struct OsdWarpArgs {
    const uint8_t *image;
    GraphImage img;
    int32_t m, n, wn, n_pad, C;
    const uint64_t *syn;
    uint64_t *err;
    uint8_t *osd_out;
    unsigned int *counters;        // [1] queue length, [2] overflow count
    const uint32_t *osd_list;
    const float *osd_llr;
    uint32_t *overflow;            // queue positions handed to K_osd
    uint64_t *slots;               // [total warps][C][wn] dense rows
    uint64_t *gkeys;               // [total warps][n_pad] sort keys when not in shared memory
    uint32_t region_bytes;         // per-warp shared memory
    uint32_t off_perm, off_inv, off_rflag, off_pivb, off_saug, off_x, off_ebits, off_low,
        off_mlist, off_pcol, off_prow, off_keys;
};

__device__ __forceinline__ uint32_t osd_order_bits(float x) {
    const uint32_t u = __float_as_uint(__fadd_rn(x, 0.0f));   // -0 -> +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ unsigned warp_parity(unsigned bit) {
    return __popc(__ballot_sync(0xffffffffu, bit & 1u)) & 1u;
}

template <bool kKeysSmem>
__global__ void __launch_bounds__(256) osd_warp_kernel(const OsdWarpArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
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
    const uint16_t *csc_row = reinterpret_cast<const uint16_t *>(smem + a.img.off_csc_row);

    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wid;
    const int total = gridDim.x * (blockDim.x >> 5);
    uint8_t *reg = smem + a.img.bytes + static_cast<size_t>(wid) * a.region_bytes;
    uint16_t *perm = reinterpret_cast<uint16_t *>(reg + a.off_perm);
    uint16_t *inv = reinterpret_cast<uint16_t *>(reg + a.off_inv);
    uint16_t *rflag = reinterpret_cast<uint16_t *>(reg + a.off_rflag);   // 0xffff: still a row of H
    uint32_t *pivb = reinterpret_cast<uint32_t *>(reg + a.off_pivb);
    uint32_t *saug = reinterpret_cast<uint32_t *>(reg + a.off_saug);
    uint64_t *X = reinterpret_cast<uint64_t *>(reg + a.off_x);
    uint32_t *X32 = reinterpret_cast<uint32_t *>(X);
    uint32_t *ebits = reinterpret_cast<uint32_t *>(reg + a.off_ebits);
    uint16_t *low = reinterpret_cast<uint16_t *>(reg + a.off_low);      // per slot: lowest position
    uint16_t *mlist = reinterpret_cast<uint16_t *>(reg + a.off_mlist);  // dense non-pivot rows
    uint16_t *pcol = reinterpret_cast<uint16_t *>(reg + a.off_pcol);
    uint16_t *prow = reinterpret_cast<uint16_t *>(reg + a.off_prow);
    uint64_t *keys = kKeysSmem ? reinterpret_cast<uint64_t *>(reg + a.off_keys)
                               : a.gkeys + static_cast<size_t>(gw) * a.n_pad;
    uint64_t *slots = a.slots + static_cast<size_t>(gw) * a.C * a.wn;

    const int m = a.m, n = a.n, wn = a.wn, C = a.C;
    const int W32 = (m + 31) >> 5;
    const int wm64 = (m + 63) >> 6;
    const uint32_t queue = a.counters[1];

    for (uint32_t q = gw; q < queue; q += total) {
        const uint32_t b = a.osd_list[q];
        const float *lam = a.osd_llr + static_cast<size_t>(q) * n;

        // ---- 1. sort -------------------------------------------------------
        for (int j = lane; j < a.n_pad; j += 32)
            keys[j] = (j < n) ? ((static_cast<uint64_t>(osd_order_bits(lam[j])) << 32) | static_cast<uint32_t>(j))
                              : ~0ull;
        __syncwarp();
        for (int k = 2; k <= a.n_pad; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = lane; i < a.n_pad; i += 32) {
                    const int l = i ^ jj;
                    if (l > i) {
                        const uint64_t x = keys[i], y = keys[l];
                        if ((x > y) == ((i & k) == 0)) { keys[i] = y; keys[l] = x; }
                    }
                }
                __syncwarp();
            }
        }
        for (int j = lane; j < n; j += 32) {
            const uint16_t v = static_cast<uint16_t>(keys[j]);
            perm[j] = v;
            inv[v] = static_cast<uint16_t>(j);
        }
        __syncwarp();

        // ---- 2. state ----------------------------------------------------------
        const uint32_t *sp = reinterpret_cast<const uint32_t *>(a.syn + static_cast<size_t>(b) * wm64);
        for (int r = lane; r < m; r += 32) rflag[r] = 0xffffu;
        for (int w = lane; w < W32; w += 32) {
            uint32_t x = sp[w];
            if (w == W32 - 1 && (m & 31)) x &= (1u << (m & 31)) - 1u;
            saug[w] = x;
            pivb[w] = 0u;
        }
        for (int w = lane; w < wn; w += 32) X[w] = 0ull;
        __syncwarp();

        int rank = 0, M = 0, nslots = 0;
        bool overflow = false;

        // ---- 3. forward elimination in permuted order ------------------------
        for (int j = 0; j < n && rank < m && !overflow; ++j) {
            const int v = perm[j];
            const int c0 = col_ptr[v], cw = col_ptr[v + 1] - c0;
            // Lowest candidate row p (rows of H's column v that are untouched
            // and not pivots; dense non-pivot rows whose lowest one is at j).
            int best = 0x7fffffff;
            int ncand = 0;
            for (int k0 = 0; k0 < cw; k0 += 32) {
                const int k = k0 + lane;
                int r = 0x7fffffff;
                if (k < cw) {
                    const int rr = csc_row[c0 + k];
                    if (rflag[rr] == 0xffffu && !((pivb[rr >> 5] >> (rr & 31)) & 1u)) r = rr;
                }
                ncand += __popc(__ballot_sync(0xffffffffu, r != 0x7fffffff));
                best = min(best, r);
            }
            for (int i0 = 0; i0 < M; i0 += 32) {
                const int i = i0 + lane;
                int r = 0x7fffffff;
                if (i < M) {
                    const int rr = mlist[i];
                    if (low[rflag[rr]] == j) r = rr;
                }
                ncand += __popc(__ballot_sync(0xffffffffu, r != 0x7fffffff));
                best = min(best, r);
            }
            if (ncand == 0) continue;
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
            const int p = best;

            if (ncand > 1) {
                // Replace every other candidate r by r + row p (rare).
                const unsigned sp_bit = (saug[p >> 5] >> (p & 31)) & 1u;
                const int pslot = rflag[p];
                for (int pass = 0; pass < 2 && !overflow; ++pass) {
                    const int cnt = pass == 0 ? cw : M;
                    // Rows that pass 0 turns dense join mlist; after the sum with
                    // row p their lowest one lies right of j, so pass 1 skips them.
                    for (int i0 = 0; i0 < cnt && !overflow; i0 += 32) {
                        const int i = i0 + lane;
                        int r = -1;
                        if (i < cnt) {
                            if (pass == 0) {
                                const int rr = csc_row[c0 + i];
                                if (rr != p && rflag[rr] == 0xffffu && !((pivb[rr >> 5] >> (rr & 31)) & 1u)) r = rr;
                            } else {
                                const int rr = mlist[i];
                                if (rr != p && low[rflag[rr]] == j) r = rr;
                            }
                        }
                        unsigned todo = __ballot_sync(0xffffffffu, r >= 0);
                        while (todo) {
                            const int src = __ffs(todo) - 1;
                            todo &= todo - 1;
                            const int rr = __shfl_sync(0xffffffffu, r, src);
                            int s = rflag[rr];
                            if (s == 0xffff) {
                                // Give rr a dense copy built from its row of H.
                                if (nslots >= C) { overflow = true; break; }
                                s = nslots++;
                                uint64_t *row = slots + static_cast<size_t>(s) * wn;
                                for (int w = lane; w < wn; w += 32) row[w] = 0ull;
                                __syncwarp();
                                const int e0 = row_ptr[rr], deg = row_ptr[rr + 1] - e0;
                                if (lane < deg) {
                                    const uint32_t pos = inv[col_idx[e0 + lane]];
                                    atomicOr(reinterpret_cast<unsigned int *>(row) + (pos >> 5), 1u << (pos & 31));
                                }
                                __syncwarp();
                                if (lane == 0) {
                                    rflag[rr] = static_cast<uint16_t>(s);
                                    mlist[M] = static_cast<uint16_t>(rr);
                                }
                                ++M;
                            }
                            uint64_t *row = slots + static_cast<size_t>(s) * wn;
                            if (pslot == 0xffff) {
                                const int e0 = row_ptr[p], deg = row_ptr[p + 1] - e0;
                                if (lane < deg) {
                                    const uint32_t pos = inv[col_idx[e0 + lane]];
                                    atomicXor(reinterpret_cast<unsigned int *>(row) + (pos >> 5), 1u << (pos & 31));
                                }
                            } else {
                                const uint64_t *prw = slots + static_cast<size_t>(pslot) * wn;
                                for (int w = (j >> 6) + lane; w < wn; w += 32) row[w] ^= prw[w];
                            }
                            __syncwarp();
                            if (lane == 0 && sp_bit) saug[rr >> 5] ^= 1u << (rr & 31);
                            // New lowest position of rr (0xffff when the row vanished).
                            int lo = 0xffff;
                            for (int w0 = j >> 6; w0 < wn; w0 += 32) {
                                const int w = w0 + lane;
                                const uint64_t x = (w < wn) ? row[w] : 0ull;
                                const unsigned nz = __ballot_sync(0xffffffffu, x != 0ull);
                                if (nz) {
                                    const int src2 = __ffs(nz) - 1;
                                    const uint64_t xx = __shfl_sync(0xffffffffu, x, src2);
                                    lo = (w0 + src2) * 64 + __ffsll(static_cast<long long>(xx)) - 1;
                                    break;
                                }
                            }
                            if (lane == 0) low[s] = static_cast<uint16_t>(lo);
                            __syncwarp();
                        }
                    }
                }
                if (overflow) break;
            }
            // p becomes the pivot of position j.
            if (lane == 0) {
                pivb[p >> 5] |= 1u << (p & 31);
                pcol[rank] = static_cast<uint16_t>(j);
                prow[rank] = static_cast<uint16_t>(p);
            }
            if (rflag[p] != 0xffffu) {
                // Drop p from the dense non-pivot list.
                int at = -1;
                for (int i0 = 0; i0 < M; i0 += 32) {
                    const int i = i0 + lane;
                    const unsigned hit = __ballot_sync(0xffffffffu, i < M && mlist[i] == p);
                    if (hit) { at = i0 + __ffs(hit) - 1; break; }
                }
                __syncwarp();
                if (lane == 0 && at >= 0) mlist[at] = mlist[M - 1];
                --M;
            }
            ++rank;
            __syncwarp();
        }

        if (overflow) {
            if (lane == 0) {
                const uint32_t k = atomicAdd(&a.counters[2], 1u);
                a.overflow[k] = q;
            }
            __syncwarp();
            continue;
        }

        // ---- 4. consistency: rows without a pivot must end with s' = 0 ---------
        unsigned bad = 0u;
        for (int w = lane; w < W32; w += 32) bad |= saug[w] & ~pivb[w];
        const bool nosol = __any_sync(0xffffffffu, bad != 0u);

        if (!nosol) {
            // ---- 5. backward substitution ---------------------------------------
            for (int k = rank - 1; k >= 0; --k) {
                const int p = prow[k], j = pcol[k];
                unsigned par;
                const int s = rflag[p];
                if (s == 0xffff) {
                    const int e0 = row_ptr[p], deg = row_ptr[p + 1] - e0;
                    unsigned bit = 0u;
                    if (lane < deg) {
                        const uint32_t pos = inv[col_idx[e0 + lane]];
                        bit = (X32[pos >> 5] >> (pos & 31)) & 1u;
                    }
                    par = warp_parity(bit);
                } else {
                    const uint64_t *row = slots + static_cast<size_t>(s) * wn;
                    unsigned acc = 0u;
                    for (int w = (j >> 6) + lane; w < wn; w += 32) acc += __popcll(row[w] & X[w]);
                    par = warp_parity(acc);
                }
                par ^= (saug[p >> 5] >> (p & 31)) & 1u;
                if (lane == 0 && par) X32[j >> 5] |= 1u << (j & 31);
                __syncwarp();
            }
            // ---- 6. e' = (e_S, 0) mapped back through pi -------------------------
            for (int w = lane; w < 2 * wn; w += 32) ebits[w] = 0u;
            __syncwarp();
            for (int k = lane; k < rank; k += 32) {
                const int j = pcol[k];
                if ((X32[j >> 5] >> (j & 31)) & 1u) {
                    const int v = perm[j];
                    atomicOr(&ebits[v >> 5], 1u << (v & 31));
                }
            }
            __syncwarp();
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.err + static_cast<size_t>(b) * wn);
            for (int w = lane; w < 2 * wn; w += 32) dst[w] = ebits[w];
        }
        if (lane == 0 && a.osd_out) a.osd_out[b] = nosol ? LBP_OSD_NO_SOLUTION : LBP_OSD_APPLIED;
        __syncwarp();
    }
}

}  // namespace lbp
