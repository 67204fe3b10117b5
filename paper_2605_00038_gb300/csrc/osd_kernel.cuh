// K_osd: OSD-0 (Alg. 2), one CTA per shot, dense rows.  This is the general
// path: it serves codes whose sizes do not fit the 16-bit shared-memory
// image, and the shots K_osd_warp hands over because their elimination
// needed more dense rows than its pool holds.  Per shot:
//   1. sort lambda ascending, ties by column (bitonic sort of 64-bit keys
//      (order-preserving bits of lambda, column) in shared memory), which
//      defines the permutation pi of the LLR sorting step;
//   2. build H_OSD = H P_pi as packed 64-bit rows (bit j of row r set when
//      column pi(j) of H has a one in row r), plus the syndrome bit of each row;
//   3. Gauss-Jordan elimination column by column in permuted order: a column
//      with a one in a not-yet-pivot row becomes a basis column (these are the
//      first rank(H) independent columns of H_OSD), and its bit is cleared in
//      every other row, syndrome bits included;
//   4. each basis column takes the reduced syndrome bit of its pivot row, all
//      other columns are zero; columns map back through pi.
// Given the basis, the solution e_S is unique, so this elimination returns
// exactly what the LU decomposition with forward and backward substitution
// of Alg. 2 returns.  If a non-pivot row keeps a syndrome bit, s is outside
// the column space: the BP estimate stays and the status says so.
//
// Row elimination spreads (row, word) pairs over all threads, touching only
// the words at and right of the pivot column's word: columns to the left are
// either basis columns (already cleared) or non-basis columns whose bits no
// longer matter.  The dense matrix lives in shared memory when it fits,
// otherwise in a per-CTA slice of the workspace (served from L2).
#pragma once

#include <cstdint>

#include "internal.h"

namespace lbp {

struct OsdArgs {
    int32_t m, n;
    const int32_t *row_ptr;    // CSR of H (global)
    const int32_t *col_idx;
    const uint64_t *syn;       // [B][wm64]
    uint64_t *err;             // [B][wn64]
    uint8_t *osd_out;          // [B] or null
    const unsigned int *counters;   // queue lengths
    int count_slot;            // counters[count_slot] = entries to process
    const uint32_t *qmap;      // entry -> OSD queue position (null: identity)
    const uint32_t *osd_list;
    const float *osd_llr;
    uint64_t *gmat;            // per-CTA dense matrices when not in shared memory
    int32_t n_pad;             // power of two >= n
    int32_t wn;                // 64-bit words per matrix row = ceil(n / 64)
    uint32_t off_keys, off_inv, off_flags, off_piv, off_ebits, off_mat;
};

__device__ __forceinline__ uint32_t order_bits(float x) {
    // Ascending float order as unsigned order; -0 and +0 compare equal first.
    const uint32_t u = __float_as_uint(__fadd_rn(x, 0.0f));
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <bool kMatSmem>
__global__ void __launch_bounds__(1024, 1) osd_kernel(const OsdArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *keys = reinterpret_cast<uint64_t *>(smem + a.off_keys);
    uint32_t *inv = reinterpret_cast<uint32_t *>(smem + a.off_inv);
    uint8_t *hb = smem + a.off_flags;                 // [m] row has the current column's bit
    uint8_t *ispiv = hb + a.m;                        // [m] row is a pivot row
    uint8_t *saug = ispiv + a.m;                      // [m] reduced syndrome bits
    int32_t *piv = reinterpret_cast<int32_t *>(smem + a.off_piv);   // [2] candidates, [2..] scratch
    int32_t *pcol = piv + 4;                          // [m] basis column of k-th pivot
    int32_t *prow = pcol + a.m;                       // [m] its row
    uint32_t *ebits = reinterpret_cast<uint32_t *>(smem + a.off_ebits);
    uint64_t *mat = kMatSmem ? reinterpret_cast<uint64_t *>(smem + a.off_mat)
                             : a.gmat + static_cast<size_t>(blockIdx.x) * a.m * a.wn;

    const int m = a.m, n = a.n, wn = a.wn, T = blockDim.x, tid = threadIdx.x;
    const int wm64 = (m + 63) >> 6;
    const uint32_t queue = a.counters[a.count_slot];

    for (uint32_t qi = blockIdx.x; qi < queue; qi += gridDim.x) {
        const uint32_t q = a.qmap ? a.qmap[qi] : qi;
        const uint32_t b = a.osd_list[q];
        const float *lam = a.osd_llr + static_cast<size_t>(q) * n;

        // 1. Sort.
        for (int j = tid; j < a.n_pad; j += T)
            keys[j] = (j < n) ? ((static_cast<uint64_t>(order_bits(lam[j])) << 32) | static_cast<uint32_t>(j))
                              : ~0ull;
        __syncthreads();
        for (int k = 2; k <= a.n_pad; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < a.n_pad; i += T) {
                    const int l = i ^ j;
                    if (l > i) {
                        const uint64_t x = keys[i], y = keys[l];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) { keys[i] = y; keys[l] = x; }
                    }
                }
                __syncthreads();
            }
        }
        for (int j = tid; j < n; j += T) inv[static_cast<uint32_t>(keys[j])] = j;
        // 2. Permuted dense matrix and syndrome bits.
        const uint64_t *sp = a.syn + static_cast<size_t>(b) * wm64;
        for (size_t i = tid; i < static_cast<size_t>(m) * wn; i += T) mat[i] = 0ull;
        for (int r = tid; r < m; r += T) {
            saug[r] = static_cast<uint8_t>((sp[r >> 6] >> (r & 63)) & 1ull);
            ispiv[r] = 0;
        }
        if (tid < 2) piv[tid] = 0x7fffffff;
        __syncthreads();
        for (int r = tid; r < m; r += T) {
            uint64_t *row = mat + static_cast<size_t>(r) * wn;
            for (int e = a.row_ptr[r]; e < a.row_ptr[r + 1]; ++e) {
                const uint32_t j = inv[a.col_idx[e]];
                row[j >> 6] |= 1ull << (j & 63);
            }
        }
        __syncthreads();
        // 3. Gauss-Jordan in permuted column order.
        int rank = 0;
        for (int j = 0; j < n && rank < m; ++j) {
            const int w = j >> 6;
            const uint64_t bit = 1ull << (j & 63);
            int *cand = piv + (j & 1);
            // The other buffer is next column's; nobody still reads it here
            // (its last reader passed a barrier, or it still holds the reset value).
            if (tid == 0) piv[(j + 1) & 1] = 0x7fffffff;
            for (int r = tid; r < m; r += T) {
                const bool h = (mat[static_cast<size_t>(r) * wn + w] & bit) != 0ull;
                hb[r] = h;
                if (h && !ispiv[r]) atomicMin(cand, r);
            }
            __syncthreads();
            const int p = *cand;
            if (p == 0x7fffffff) continue;
            const int span = wn - w;
            const uint64_t *prw = mat + static_cast<size_t>(p) * wn;
            for (int i = tid; i < m * span; i += T) {
                const int r = i / span;
                if (r != p && hb[r]) {
                    const int ww = w + (i - r * span);
                    mat[static_cast<size_t>(r) * wn + ww] ^= prw[ww];
                }
            }
            for (int r = tid; r < m; r += T)
                if (r != p && hb[r]) saug[r] ^= saug[p];
            if (tid == 0) {
                ispiv[p] = 1;
                pcol[rank] = j;
                prow[rank] = p;
            }
            ++rank;
            __syncthreads();
        }
        // 4. Consistency, solution, inverse permutation.
        int bad = 0;
        for (int r = tid; r < m; r += T) bad |= (!ispiv[r] && saug[r]) ? 1 : 0;
        bad = __syncthreads_or(bad);
        if (!bad) {
            for (int i = tid; i < 2 * wn; i += T) ebits[i] = 0u;
            __syncthreads();
            for (int k = tid; k < rank; k += T) {
                if (saug[prow[k]]) {
                    const uint32_t v = static_cast<uint32_t>(keys[pcol[k]]);
                    atomicOr(&ebits[v >> 5], 1u << (v & 31));
                }
            }
            __syncthreads();
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.err + static_cast<size_t>(b) * wn);
            for (int i = tid; i < 2 * wn; i += T) dst[i] = ebits[i];
        }
        if (tid == 0 && a.osd_out) a.osd_out[b] = bad ? LBP_OSD_NO_SOLUTION : LBP_OSD_APPLIED;
        __syncthreads();
    }
}

}  // namespace lbp
