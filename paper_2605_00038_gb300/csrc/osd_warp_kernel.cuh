// K_osd_warp: OSD-0 (Alg. 2), one warp per shot, event-driven elimination.
//
// Alg. 2 sorts the columns by lambda (pi), takes the first rank(H) columns of
// H P_pi that are independent (basis S), solves H_S e_S = s by LU with
// forward and backward substitution and sets every other column to zero.
// This kernel computes exactly that e, without materialising P_pi:
//
//  * Column order.  Column v has the key K(v) = (order-preserving bits of
//    lambda_v, v): ascending K is the sorted order of Alg. 2 (ties by column).
//  * Forward elimination as events.  Scanning columns in K order, a row of H
//    first meets the scan at the smallest key among its columns; a row that
//    an elimination changed meets it again at the smallest key among its new
//    columns.  At the column v of an event, the rows meeting there are the
//    candidates: the lowest-numbered becomes the pivot of v (v joins S) and
//    every other candidate becomes its sum with the pivot row, syndrome bit
//    included, then waits for its next event.  Columns where no row meets are
//    dependent on earlier ones and skipped.  So the scan costs one event per
//    row plus one per elimination, not one step per column.
//  * Rows are sorted once by their first key: a stable LSD radix sort of
//    the 48 key bits of (K, row) pairs, 8 bits per pass, ranks within a warp
//    step from __match_any_sync (rows with equal K are one event, so their
//    order does not matter).  Runs of events that concern a single row, with no
//    changed row waiting at or before them, commit 32 at a time: each lane's
//    row becomes the pivot of its column.  Events with several rows are
//    handled one at a time.
//  * Only changed rows are stored densely (bits by original column), in a
//    per-warp pool of C rows in the workspace; untouched rows are read from
//    the CSR image of H.  Measured: about 40 changed rows per shot on the d=11
//    space-time code.  A shot that needs more than C rows goes to the
//    block-wide kernel K_osd, which computes the same e.
//  * Shared memory per warp is reused by lifetime, since resident warps set
//    the throughput of this latency-bound kernel: during the sort only the
//    keys, the radix buffer and the digit histogram are live, so the
//    elimination's arrays (pivot columns and rows, row flags, pivot and
//    syndrome bits, waiting rows) share the buffer's bytes; after the
//    elimination the keys are dead, so the solution bits and the column ->
//    pivot index map (rebuilt from the pivot columns) take their place.
//  * Latency layout (kLat, for batches of at most one shot per SM): one warp
//    per CTA, whose shared memory also holds the order bits of the shot's
//    lambda (read once, coalesced) and the first Cs rows of the dense-row
//    pool, so most steps of the event chain are shared-memory accesses
//    instead of L2 round trips.  Rows past Cs stay in the workspace, so the
//    pool holds as many rows as in the throughput layout.
//  * Backward substitution over the pivots in reverse order, 32 per batch:
//    each lane folds in the solution bits of later batches and records which
//    pivots of its own batch its row touches (changed rows are scanned by the
//    whole warp); the batch is then resolved level by level, all pivots whose
//    dependencies are known at once.  The solution bits sit at the original
//    column indices, so they are the output directly (no inverse
//    permutation).
#pragma once

#include <cstdint>

#include "internal.h"
#include "osd_kernel.cuh"

namespace lbp {

struct OsdWarpArgs {
    const uint8_t *image;          // CSR image (GraphImage layout); only row_ptr / col_idx are read
    GraphImage img;
    int32_t m, n, wn, C;
    const uint64_t *syn;
    uint64_t *err;
    uint8_t *osd_out;
    unsigned int *counters;        // [1] queue length, [2] handed over to K_osd
    const uint32_t *osd_list;
    const float *osd_llr;
    uint32_t *overflow;            // queue positions handed to K_osd
    uint64_t *slots;               // [total warps][C][wn] dense rows
    uint32_t image_bytes;          // bytes of the image prefix staged (row_ptr + col_idx)
    uint32_t region_bytes;         // per-warp shared memory
    uint32_t off_keys, off_tmp, off_hist, off_rflag, off_pivk, off_pivb, off_saug, off_x, off_pcol, off_prow,
        off_pend;             // off_tmp / off_hist (sort) overlap the elimination's arrays;
                              // off_x / off_pivk (after it) may overlap the keys
    uint32_t off_lb, off_pool;     // latency layout: lambda order bits [n], pool rows [Cs][wn]
    int32_t Cs;                    // latency layout: pool rows in shared memory (0 otherwise)
};

constexpr uint64_t kNoKey = ~0ull;

// 48-bit column key: order-preserving bits of lambda (ties: column index),
// from lambda in global memory or from its order bits lb in shared memory.
template <bool kLat>
__device__ __forceinline__ uint64_t col_key(const float *lam, const uint32_t *lb, int v) {
    const uint32_t o = kLat ? lb[v] : order_bits(__ldg(lam + v));
    return (static_cast<uint64_t>(o) << 16) | static_cast<uint32_t>(v);
}

// Warp minimum of a 64-bit key: the least high word, then the least low word
// among the lanes holding it (two redux.sync; every lane takes part in both).
__device__ __forceinline__ uint64_t warp_min_u64(uint64_t x) {
    const uint32_t hi = static_cast<uint32_t>(x >> 32);
    const uint32_t mhi = __reduce_min_sync(0xffffffffu, hi);
    const uint32_t lo = hi == mhi ? static_cast<uint32_t>(x) : 0xffffffffu;
    const uint32_t mlo = __reduce_min_sync(0xffffffffu, lo);
    return (static_cast<uint64_t>(mhi) << 32) | mlo;
}

template <int MaxWarps, bool kLat>
__global__ void __launch_bounds__(MaxWarps * 32) osd_warp_kernel(const OsdWarpArgs a) {
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
    uint64_t *keys = reinterpret_cast<uint64_t *>(reg + a.off_keys);     // [m] (K << 16 | row)
    uint64_t *tmp = reinterpret_cast<uint64_t *>(reg + a.off_tmp);       // [m] sort buffer
    uint32_t *hist = reinterpret_cast<uint32_t *>(reg + a.off_hist);     // [256] digit counts
    uint16_t *rflag = reinterpret_cast<uint16_t *>(reg + a.off_rflag);   // [m] dense slot or 0xffff
    uint16_t *pivk = reinterpret_cast<uint16_t *>(reg + a.off_pivk);     // [n] pivot index of column (after)
    uint32_t *pivb = reinterpret_cast<uint32_t *>(reg + a.off_pivb);     // [W32] row is a pivot
    uint32_t *saug = reinterpret_cast<uint32_t *>(reg + a.off_saug);     // [W32] reduced syndrome
    uint64_t *X = reinterpret_cast<uint64_t *>(reg + a.off_x);           // [wn] solution (may alias keys)
    uint32_t *X32 = reinterpret_cast<uint32_t *>(X);
    uint16_t *pcol = reinterpret_cast<uint16_t *>(reg + a.off_pcol);     // [m] column of pivot k
    uint16_t *prow = reinterpret_cast<uint16_t *>(reg + a.off_prow);     // [m] row of pivot k
    uint64_t *pend = reinterpret_cast<uint64_t *>(reg + a.off_pend);     // [C] waiting changed rows
    uint32_t *lb = kLat ? reinterpret_cast<uint32_t *>(reg + a.off_lb) : nullptr;  // [n] lambda order bits
    uint64_t *gslots = a.slots + static_cast<size_t>(gw) * a.C * a.wn;
    uint64_t *sslots = kLat ? reinterpret_cast<uint64_t *>(reg + a.off_pool) : nullptr;
    const int Cs = kLat ? a.Cs : 0;
    // Row s of the pool: shared memory for s < Cs, else the workspace.
    auto pool_row = [&](int s) -> uint64_t * {
        return (s < Cs ? sslots : gslots) + static_cast<size_t>(s) * a.wn;
    };

    const int m = a.m, n = a.n, wn = a.wn, C = a.C;
    const int W32 = (m + 31) >> 5;
    const int wm64 = (m + 63) >> 6;
    const uint32_t queue = a.counters[1];

    for (uint32_t q = gw; q < queue; q += total) {
        const uint32_t b = a.osd_list[q];
        const float *lam = a.osd_llr + static_cast<size_t>(q) * n;
        if (kLat) {
            #pragma unroll 4
            for (int v = lane; v < n; v += 32) lb[v] = order_bits(__ldg(lam + v));
            __syncwarp();
        }

        // ---- rows keyed by their first column, sorted -----------------------
        for (int r = lane; r < m; r += 32) {
            uint64_t k = kNoKey;
            for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                const uint64_t kc = col_key<kLat>(lam, lb, col_idx[e]);
                k = kc < k ? kc : k;
            }
            if (k != kNoKey) k = (k << 16) | static_cast<uint32_t>(r);
            keys[r] = k;
        }
        __syncwarp();
        // Stable LSD radix sort of keys[0, m) on bits 16..63, 8 bits a pass;
        // six passes leave the result in keys.
        for (int pass = 0; pass < 6; ++pass) {
            const uint64_t *src = (pass & 1) ? tmp : keys;
            uint64_t *dst = (pass & 1) ? keys : tmp;
            const int sh = 16 + 8 * pass;
            for (int d = lane; d < 256; d += 32) hist[d] = 0u;
            __syncwarp();
            for (int j0 = 0; j0 < m; j0 += 32) {
                const int i = j0 + lane;
                const unsigned act = __ballot_sync(0xffffffffu, i < m);
                if (i < m) {
                    const unsigned dg = static_cast<unsigned>(src[i] >> sh) & 255u;
                    const unsigned peers = __match_any_sync(act, dg);
                    if (lane == __ffs(peers) - 1) hist[dg] += __popc(peers);
                }
                __syncwarp();
            }
            // Exclusive prefix over the 256 counts: 8 per lane, then across lanes.
            uint32_t c8[8], tot = 0;
            #pragma unroll
            for (int j = 0; j < 8; ++j) { c8[j] = hist[lane * 8 + j]; tot += c8[j]; }
            uint32_t incl = tot;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t run = incl - tot;
            __syncwarp();
            #pragma unroll
            for (int j = 0; j < 8; ++j) { hist[lane * 8 + j] = run; run += c8[j]; }
            __syncwarp();
            for (int j0 = 0; j0 < m; j0 += 32) {
                const int i = j0 + lane;
                const unsigned act = __ballot_sync(0xffffffffu, i < m);
                if (i < m) {
                    const uint64_t x = src[i];
                    const unsigned dg = static_cast<unsigned>(x >> sh) & 255u;
                    const unsigned peers = __match_any_sync(act, dg);
                    const unsigned before = __popc(peers & ((1u << lane) - 1u));
                    dst[hist[dg] + before] = x;
                    __syncwarp(act);
                    if (lane == __ffs(peers) - 1) hist[dg] += __popc(peers);
                }
                __syncwarp();
            }
        }
        // The sort's buffer is dead from here on: its bytes become the
        // elimination's row flags, pivot and syndrome bits.
        for (int r = lane; r < m; r += 32) rflag[r] = 0xffffu;
        {
            const uint32_t *sp = reinterpret_cast<const uint32_t *>(a.syn + static_cast<size_t>(b) * wm64);
            for (int w = lane; w < W32; w += 32) {
                uint32_t x = sp[w];
                if (w == W32 - 1 && (m & 31)) x &= (1u << (m & 31)) - 1u;
                saug[w] = x;
                pivb[w] = 0u;
            }
        }
        __syncwarp();

        // ---- forward elimination, event by event ------------------------------
        int ptr = 0, rank = 0, npend = 0, nslots = 0;
        uint64_t pmin = kNoKey;          // smallest key among waiting changed rows
        bool overflow = false;
        while (!overflow) {
            const int i = ptr + lane;
            const uint64_t ki = (i < m) ? keys[i] : kNoKey;
            const uint64_t Ki = ki == kNoKey ? kNoKey : (ki >> 16);
            uint64_t Kprev = __shfl_up_sync(0xffffffffu, Ki, 1);
            if (lane == 0) Kprev = (ptr > 0) ? (keys[ptr - 1] >> 16) : kNoKey - 1;
            uint64_t Knext = __shfl_down_sync(0xffffffffu, Ki, 1);
            if (lane == 31) {
                const uint64_t kn = (i + 1 < m) ? keys[i + 1] : kNoKey;
                Knext = kn == kNoKey ? kNoKey : (kn >> 16);
            }
            const bool single = Ki != kNoKey && Ki != Kprev && Ki != Knext &&
                                (pmin == kNoKey || Ki < (pmin >> 16));
            const unsigned notsingle = __ballot_sync(0xffffffffu, !single);
            const int L = notsingle ? __ffs(notsingle) - 1 : 32;
            if (L > 0) {
                if (lane < L) {
                    const int r = static_cast<int>(ki & 0xffffu);
                    const int v = static_cast<int>(Ki & 0xffffu);
                    pcol[rank + lane] = static_cast<uint16_t>(v);
                    prow[rank + lane] = static_cast<uint16_t>(r);
                    atomicOr(&pivb[r >> 5], 1u << (r & 31));
                }
                rank += L;
                ptr += L;
                __syncwarp();
                continue;
            }
            // The event at the smallest pending key: sorted rows and waiting rows.
            const uint64_t K0 = __shfl_sync(0xffffffffu, Ki, 0);
            const uint64_t Kev = (pmin != kNoKey && (pmin >> 16) < K0) ? (pmin >> 16) : K0;
            if (Kev == kNoKey) break;
            const int v = static_cast<int>(Kev & 0xffffu);
            // Candidates among the sorted run starting at ptr ...
            int nsorted = 0;
            while (true) {
                const int j = ptr + nsorted + lane;
                const uint64_t kj = (j < m) ? keys[j] : kNoKey;
                const bool eq = kj != kNoKey && (kj >> 16) == Kev;
                const unsigned bal = __ballot_sync(0xffffffffu, eq);
                const int run = (~bal) ? __ffs(~bal) - 1 : 32;
                nsorted += run;
                if (run < 32) break;
            }
            // ... and among the waiting rows.
            int best = 0x7fffffff;
            for (int j0 = 0; j0 < nsorted; j0 += 32) {
                const int j = j0 + lane;
                if (j < nsorted) best = min(best, static_cast<int>(keys[ptr + j] & 0xffffu));
            }
            for (int j0 = 0; j0 < npend; j0 += 32) {
                const int j = j0 + lane;
                if (j < npend && (pend[j] >> 16) == Kev) best = min(best, static_cast<int>(pend[j] & 0xffffu));
            }
            const int p = __reduce_min_sync(0xffffffffu, best);
            const unsigned sp_bit = (saug[p >> 5] >> (p & 31)) & 1u;
            const int pslot = rflag[p];
            // Every other candidate r: r <- r + row p, then it waits at its next
            // key (appended to pend; those entries have keys above Kev, so the
            // scan of pass 1 skips them).  Pass 0: rows of H from the sorted run;
            // pass 1: changed rows waiting at Kev.
            const int npend0 = npend;
            for (int pass = 0; pass < 2 && !overflow; ++pass) {
                const int cnt = pass == 0 ? nsorted : npend0;
                for (int j0 = 0; j0 < cnt && !overflow; j0 += 32) {
                    const int j = j0 + lane;
                    int r = -1;
                    if (j < cnt) {
                        if (pass == 0) {
                            const int rr = static_cast<int>(keys[ptr + j] & 0xffffu);
                            if (rr != p) r = rr;
                        } else {
                            const uint64_t e = pend[j];
                            const int rr = static_cast<int>(e & 0xffffu);
                            if ((e >> 16) == Kev && rr != p) r = rr;
                        }
                    }
                    unsigned todo = __ballot_sync(0xffffffffu, r >= 0);
                    while (todo) {
                        const int src = __ffs(todo) - 1;
                        todo &= todo - 1;
                        const int rr = __shfl_sync(0xffffffffu, r, src);
                        int s = rflag[rr];
                        uint64_t *row;
                        if (s == 0xffff) {
                            if (nslots >= C) { overflow = true; break; }
                            s = nslots++;
                            row = pool_row(s);
                            for (int w = lane; w < wn; w += 32) row[w] = 0ull;
                            __syncwarp();
                            for (int e = row_ptr[rr] + lane; e < row_ptr[rr + 1]; e += 32) {
                                const uint32_t u = col_idx[e];
                                atomicOr(reinterpret_cast<unsigned int *>(row) + (u >> 5), 1u << (u & 31));
                            }
                            if (lane == 0) rflag[rr] = static_cast<uint16_t>(s);
                            __syncwarp();
                        } else {
                            row = pool_row(s);
                        }
                        if (pslot == 0xffff) {
                            for (int e = row_ptr[p] + lane; e < row_ptr[p + 1]; e += 32) {
                                const uint32_t u = col_idx[e];
                                atomicXor(reinterpret_cast<unsigned int *>(row) + (u >> 5), 1u << (u & 31));
                            }
                        } else {
                            const uint64_t *prw = pool_row(pslot);
                            for (int w = lane; w < wn; w += 32) row[w] ^= prw[w];
                        }
                        __syncwarp();
                        if (lane == 0 && sp_bit) saug[rr >> 5] ^= 1u << (rr & 31);
                        // Next key of rr: the smallest key among its remaining columns
                        // (all above Kev).  A row that vanished waits no more.
                        uint64_t kmin = kNoKey;
                        for (int w = lane; w < wn; w += 32) {
                            uint64_t x = row[w];
                            while (x) {
                                const int bit = __ffsll(static_cast<long long>(x)) - 1;
                                x &= x - 1;
                                const uint64_t kc = col_key<kLat>(lam, lb, w * 64 + bit);
                                kmin = kc < kmin ? kc : kmin;
                            }
                        }
                        kmin = warp_min_u64(kmin);
                        if (kmin != kNoKey) {
                            if (npend >= C) { overflow = true; break; }
                            if (lane == 0) pend[npend] = (kmin << 16) | static_cast<uint32_t>(rr);
                            ++npend;
                        }
                        __syncwarp();
                    }
                }
            }
            // Drop the waiting entries consumed by this event; the smallest
            // key among those kept is the next pending event.
            uint64_t mn = kNoKey;
            if (!overflow) {
                int kept = 0;
                for (int j0 = 0; j0 < npend; j0 += 32) {
                    const int j = j0 + lane;
                    const uint64_t e = (j < npend) ? pend[j] : kNoKey;
                    const bool keep = j < npend && (e >> 16) != Kev;
                    const unsigned bk = __ballot_sync(0xffffffffu, keep);
                    __syncwarp();
                    if (keep) {
                        pend[kept + __popc(bk & ((1u << lane) - 1u))] = e;
                        mn = e < mn ? e : mn;
                    }
                    kept += __popc(bk);
                    __syncwarp();
                }
                npend = kept;
            }
            if (overflow) break;
            // p becomes the pivot of v.
            if (lane == 0) {
                pcol[rank] = static_cast<uint16_t>(v);
                prow[rank] = static_cast<uint16_t>(p);
                pivb[p >> 5] |= 1u << (p & 31);
            }
            ++rank;
            ptr += nsorted;
            pmin = warp_min_u64(mn);
        }

        if (overflow) {
            if (lane == 0) {
                const uint32_t k = atomicAdd(&a.counters[2], 1u);
                a.overflow[k] = q;
            }
            __syncwarp();
            continue;
        }

        // The solution bits and the column -> pivot index map may share the
        // sorted keys' bytes, dead from here on.
        for (int w = lane; w < wn; w += 32) X[w] = 0ull;
        for (int v = lane; v < n; v += 32) pivk[v] = 0xffffu;
        __syncwarp();
        for (int k = lane; k < rank; k += 32) pivk[pcol[k]] = static_cast<uint16_t>(k);
        __syncwarp();

        // ---- consistency: rows without a pivot must end with s' = 0 ---------------
        unsigned bad = 0u;
        for (int w = lane; w < W32; w += 32) bad |= saug[w] & ~pivb[w];
        const bool nosol = __any_sync(0xffffffffu, bad != 0u);

        if (!nosol) {
            // ---- backward substitution, 32 pivots per batch -------------------
            // Lane k of a batch holds pivot k's equation x_k = s'_k + sum of
            // the later pivots' x over its row's other pivot columns: `part`
            // folds in those of later batches, `dep` marks those inside the
            // batch.  Rows of H are scanned by their own lane; changed (dense)
            // rows by the whole warp, one word per lane.  The batch is then
            // solved level by level: every pivot whose dependencies are known
            // resolves in the same step (dependencies point only to higher
            // pivots, so each step resolves at least the highest open one).
            for (int hi = rank; hi > 0;) {
                const int lo = hi > 32 ? hi - 32 : 0;
                const int k = lo + lane;
                unsigned part = 0u, dep = 0u;
                int slot = 0xffff;
                if (k < hi) {
                    const int p = prow[k];
                    part = (saug[p >> 5] >> (p & 31)) & 1u;
                    slot = rflag[p];
                    if (slot == 0xffff) {
                        for (int e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
                            const int u = col_idx[e];
                            const int kk = pivk[u];
                            if (kk == 0xffff || kk == k) continue;
                            if (kk >= hi) part ^= (X32[u >> 5] >> (u & 31)) & 1u;
                            else if (kk > k) dep |= 1u << (kk - lo);
                        }
                    }
                }
                unsigned dense = __ballot_sync(0xffffffffu, k < hi && slot != 0xffff);
                while (dense) {
                    const int src = __ffs(dense) - 1;
                    dense &= dense - 1u;
                    const int ss = __shfl_sync(0xffffffffu, slot, src);
                    const int k0 = lo + src;
                    const uint64_t *row = pool_row(ss);
                    unsigned mp = 0u, md = 0u;
                    for (int w = lane; w < wn; w += 32) {
                        uint64_t x = row[w];
                        while (x) {
                            const int bit = __ffsll(static_cast<long long>(x)) - 1;
                            x &= x - 1;
                            const int u = w * 64 + bit;
                            const int kk = pivk[u];
                            if (kk == 0xffff || kk == k0) continue;
                            if (kk >= hi) mp ^= (X32[u >> 5] >> (u & 31)) & 1u;
                            else if (kk > k0) md |= 1u << (kk - lo);
                        }
                    }
                    const unsigned pp = __popc(__ballot_sync(0xffffffffu, mp != 0u)) & 1u;
                    const unsigned dd = __reduce_or_sync(0xffffffffu, md);
                    if (lane == src) { part ^= pp; dep |= dd; }
                }
                const unsigned valid = __ballot_sync(0xffffffffu, k < hi);
                unsigned E = 0u, done = 0u;
                while (done != valid) {
                    const bool open = k < hi && !((done >> lane) & 1u);
                    const bool ready = open && (dep & ~done) == 0u;
                    const unsigned mine = part ^ (__popc(dep & E) & 1u);
                    const unsigned rb = __ballot_sync(0xffffffffu, ready);
                    E |= __ballot_sync(0xffffffffu, ready && mine);
                    done |= rb;
                }
                if (k < hi && ((E >> lane) & 1u)) {
                    const int u = pcol[k];
                    atomicOr(&X32[u >> 5], 1u << (u & 31));
                }
                __syncwarp();
                hi = lo;
            }
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.err + static_cast<size_t>(b) * wn);
            for (int w = lane; w < 2 * wn; w += 32) dst[w] = X32[w];
        }
        if (lane == 0 && a.osd_out) a.osd_out[b] = nosol ? LBP_OSD_NO_SOLUTION : LBP_OSD_APPLIED;
        __syncwarp();
    }
}

}  // namespace lbp
