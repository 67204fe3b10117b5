// K_osd_dense: OSD-0 (Alg. 2) for small codes, one warp per shot, the whole
// augmented matrix [H | s] in registers.
//
// For m <= 32 RL rows and n + 1 <= 64 WN columns, RL and WN up to 5 (the
// BB [[144,12,12]] code: RL = 3, WN = 3; BB [[288,12,18]]: RL = 5, WN = 5) every row of H, with its syndrome bit at column n, is
// packed into WN 64-bit words, and lane l holds rows l, l + 32, ... .  Per
// shot:
//   1. LLR sorting: the rank of column v in the order of Alg. 2 (lambda
//      ascending, ties by column) is the number of columns u whose key
//      (order-preserving bits of lambda_u, u) is smaller; perm[rank] = v.
//   2. Gauss-Jordan elimination over the columns in that order: the column's
//      bit in every row comes from registers, a ballot finds the rows that are
//      not yet pivots and have the bit (the lowest-numbered one becomes the
//      pivot), the pivot row is broadcast by shuffles and added to every other
//      row with the bit, pivot rows included.  A column without a candidate is
//      dependent on the earlier ones.  The scan stops once rank(H) pivots are
//      found (rank(H) is computed when the code is loaded): the remaining
//      non-pivot rows are then zero in H.
//   3. The basis columns are those with a pivot, so e_S is the pivot rows'
//      reduced syndrome bits and every other column is zero: the unique
//      solution of H_S e_S = s that the LU decomposition with forward and
//      backward substitution of Alg. 2 returns.  A non-pivot row with a
//      syndrome bit left means s is outside the column space: the BP
//      estimate stays and the status says so.
// The event-driven K_osd_warp keeps the rows an elimination changes in a
// workspace pool; on codes whose elimination changes nearly every row (the BB
// codes) each of its events then waits on L2, which this form avoids.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "internal.h"
#include "osd_kernel.cuh"

namespace lbp {

constexpr int kOsdDenseWarps = 16;     // warps per CTA

struct OsdDenseArgs {
    const uint8_t *image;          // 16-bit CSR image (GraphImage); row_ptr and col_idx are staged
    GraphImage img;
    uint32_t image_bytes;          // bytes of the staged prefix (row_ptr + col_idx)
    int32_t m, n, wn, rank;        // wn = 64-bit words of n columns; rank = rank(H) over GF(2)
    const uint64_t *syn;           // [B][ceil(m / 64)]
    uint64_t *err;                 // [B][wn]
    uint8_t *osd_out;              // [B] or null
    const unsigned int *counters;  // [1] = OSD queue length
    const uint32_t *osd_list;      // queue position -> shot
    const float *osd_llr;          // queue position -> lambda[n]
    uint32_t region_bytes;         // per warp: order bits u32[n], perm u16[n], solution u32[2 wn]
    uint32_t off_perm, off_x;
};

// Launch over the OSD queue with RL rows per lane and WN words per row
// (osd_dense.cu); grid CTAs of kOsdDenseWarps warps, smem bytes of shared
// memory (the staged image prefix and one region per warp).
int launch_osd_dense(const OsdDenseArgs &a, int RL, int WN, int grid, size_t smem, cudaStream_t st);

// Word w (uniform across the warp) of a packed row held in registers.
template <int WN>
__device__ __forceinline__ uint64_t row_word(const uint64_t (&r)[WN], int w) {
    uint64_t x = r[0];
    #pragma unroll
    for (int k = 1; k < WN; ++k) x = (w == k) ? r[k] : x;
    return x;
}

template <int RL, int WN>
__global__ void __launch_bounds__(kOsdDenseWarps * 32) osd_dense_kernel(const OsdDenseArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    {
        const int4 *src = reinterpret_cast<const int4 *>(a.image);
        int4 *dst = reinterpret_cast<int4 *>(smem);
        const int words = static_cast<int>(a.image_bytes >> 4);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    const uint16_t *row_ptr = reinterpret_cast<const uint16_t *>(smem + a.img.off_row_ptr);
    const uint16_t *col_idx = reinterpret_cast<const uint16_t *>(smem + a.img.off_col_idx);

    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wid;
    const int total = gridDim.x * (blockDim.x >> 5);
    uint8_t *reg = smem + a.image_bytes + static_cast<size_t>(wid) * a.region_bytes;
    uint32_t *kb = reinterpret_cast<uint32_t *>(reg);                  // [n] order bits of lambda
    uint16_t *perm = reinterpret_cast<uint16_t *>(reg + a.off_perm);   // [n] columns in sorted order
    uint32_t *X32 = reinterpret_cast<uint32_t *>(reg + a.off_x);       // [2 wn] solution bits

    const int m = a.m, n = a.n, wn = a.wn;
    const int wm64 = (m + 63) >> 6;
    const uint32_t queue = a.counters[1];

    for (uint32_t q = gw; q < queue; q += total) {
        const uint32_t b = a.osd_list[q];
        const float *lam = a.osd_llr + static_cast<size_t>(q) * n;

        // ---- 1. LLR sorting by rank ---------------------------------------------
        for (int v = lane; v < n; v += 32) kb[v] = order_bits(__ldg(lam + v));
        __syncwarp();
        constexpr int kCols = (64 * WN + 31) / 32;     // columns per lane (n < 64 WN)
        uint32_t kv[kCols];
        int rk[kCols];
        #pragma unroll
        for (int i = 0; i < kCols; ++i) {
            const int v = lane + 32 * i;
            kv[i] = v < n ? kb[v] : 0u;
            rk[i] = 0;
        }
        for (int u = 0; u < n; ++u) {
            const uint32_t ku = kb[u];
            #pragma unroll
            for (int i = 0; i < kCols; ++i) {
                const int v = lane + 32 * i;
                rk[i] += (ku < kv[i] || (ku == kv[i] && u < v)) ? 1 : 0;
            }
        }
        #pragma unroll
        for (int i = 0; i < kCols; ++i) {
            const int v = lane + 32 * i;
            if (v < n) perm[rk[i]] = static_cast<uint16_t>(v);
        }

        // ---- rows of [H | s] ----------------------------------------------------
        uint64_t row[RL][WN];
        bool piv[RL];
        int pcol[RL];
        const uint64_t *sw = a.syn + static_cast<size_t>(b) * wm64;
        #pragma unroll
        for (int jj = 0; jj < RL; ++jj) {
            #pragma unroll
            for (int k = 0; k < WN; ++k) row[jj][k] = 0ull;
            piv[jj] = false;
            pcol[jj] = 0;
            const int r = lane + 32 * jj;
            if (r < m) {
                for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                    const int c = col_idx[e];
                    #pragma unroll
                    for (int k = 0; k < WN; ++k)
                        row[jj][k] |= ((c >> 6) == k) ? (1ull << (c & 63)) : 0ull;
                }
                const uint64_t sb = (__ldg(sw + (r >> 6)) >> (r & 63)) & 1ull;
                #pragma unroll
                for (int k = 0; k < WN; ++k)
                    row[jj][k] |= ((n >> 6) == k) ? (sb << (n & 63)) : 0ull;
            }
        }
        __syncwarp();

        // ---- 2. Gauss-Jordan over the sorted columns ------------------------------
        int found = 0;
        for (int i = 0; i < n && found < a.rank; ++i) {
            const int v = perm[i];
            const int w = v >> 6;
            const uint64_t msk = 1ull << (v & 63);
            bool hb[RL];
            int jsel = -1;
            unsigned bsel = 0u;
            #pragma unroll
            for (int jj = 0; jj < RL; ++jj) {
                hb[jj] = (row_word<WN>(row[jj], w) & msk) != 0ull;
                const unsigned bl = __ballot_sync(0xffffffffu, hb[jj] && !piv[jj]);
                if (jsel < 0 && bl != 0u) {
                    jsel = jj;
                    bsel = bl;
                }
            }
            if (jsel < 0) continue;                        // dependent column
            const int owner = __ffs(bsel) - 1;             // lowest-numbered candidate row
            uint64_t pw[WN];
            #pragma unroll
            for (int k = 0; k < WN; ++k) {
                uint64_t x = row[0][k];
                #pragma unroll
                for (int jj = 1; jj < RL; ++jj) x = (jsel == jj) ? row[jj][k] : x;
                pw[k] = __shfl_sync(0xffffffffu, x, owner);
            }
            #pragma unroll
            for (int jj = 0; jj < RL; ++jj) {
                const bool self = lane == owner && jj == jsel;
                if (hb[jj] && !self) {
                    #pragma unroll
                    for (int k = 0; k < WN; ++k) row[jj][k] ^= pw[k];
                }
                if (self) {
                    piv[jj] = true;
                    pcol[jj] = v;
                }
            }
            ++found;
        }

        // ---- 3. consistency and the solution --------------------------------------
        bool bad = false;
        #pragma unroll
        for (int jj = 0; jj < RL; ++jj) {
            const bool sbit = (row_word<WN>(row[jj], n >> 6) >> (n & 63)) & 1ull;
            bad |= !piv[jj] && sbit;
        }
        const bool nosol = __any_sync(0xffffffffu, bad);
        if (!nosol) {
            for (int w = lane; w < 2 * wn; w += 32) X32[w] = 0u;
            __syncwarp();
            #pragma unroll
            for (int jj = 0; jj < RL; ++jj) {
                const bool sbit = (row_word<WN>(row[jj], n >> 6) >> (n & 63)) & 1ull;
                if (piv[jj] && sbit) atomicOr(&X32[pcol[jj] >> 5], 1u << (pcol[jj] & 31));
            }
            __syncwarp();
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.err + static_cast<size_t>(b) * wn);
            for (int w = lane; w < 2 * wn; w += 32) dst[w] = X32[w];
        }
        if (lane == 0 && a.osd_out) a.osd_out[b] = nosol ? LBP_OSD_NO_SOLUTION : LBP_OSD_APPLIED;
        __syncwarp();
    }
}

}  // namespace lbp
