// Tanner-graph access policies of bp_ell_kernel.  Both present the same
// slot layout: check c's k-th neighbour (column id, padding column n whose
// prior and posterior are +inf) and column v's k-th message offset
// (slot * R + check with R = Mp + 2, padding offset Mp whose message is +0),
// the checks of a column in ascending row order.
//
//  * EllGraph: the ELL index image (cidx[DC][Mp], vent[DV][Np], mu[Np + 2]),
//    read from shared memory or, for large codes, from global memory; a
//    thread reads the indices of its two adjacent checks / columns as one
//    paired access.
//  * RoundGraph: any space-time matrix of Eq. 1 (a round matrix H_r on the
//    diagonal, identity measurement blocks between rounds): one round's index
//    table in shared memory, the round offset and the measurement columns by
//    arithmetic; slots as for SurfaceGraph (round columns, then blocks t - 1
//    and t), so the same sums in the same order.
//  * SurfaceGraph: the unrotated surface-code space-time matrix, whose
//    indices Table III gives by closed formulas (VN0..VN3 data qubits of the
//    round, VN4 / VN5 the measurement blocks before and after it); the column
//    side inverts them.  No index image exists: the kernel's shared memory
//    holds only the per-shot state.  Slots are fixed (slot k = VN k), absent
//    neighbours padded, so the real neighbours stay in ascending column order
//    (except the wrapped block of a cyclic boundary) and every LLR sum keeps
//    the ascending row order.
#pragma once

#include <cstdint>

#include "internal.h"

namespace lbp {

// Index width of the ELL image: 16-bit (the image fits shared memory) or
// 32-bit (large codes, read from global memory); P holds two indices.
template <typename IdxT> struct Idx;
template <> struct Idx<uint16_t> {
    using P = uint32_t;
    static __device__ __forceinline__ uint32_t lo(uint32_t p) { return p & 0xffffu; }
    static __device__ __forceinline__ uint32_t hi(uint32_t p) { return p >> 16; }
};
template <> struct Idx<uint32_t> {
    using P = uint2;
    static __device__ __forceinline__ uint32_t lo(uint2 p) { return p.x; }
    static __device__ __forceinline__ uint32_t hi(uint2 p) { return p.y; }
};

template <typename IdxT, int DC, int DV>
struct EllGraph {
    using IP = typename Idx<IdxT>::P;
    static constexpr bool kImage = true;
    static constexpr bool kEll = true;     // the index image (may carry the bank-aware layout)
    const IdxT *cidx;
    const IP *cidx2;
    const IdxT *vent;
    const IP *vent2;
    const float *mu_;
    const float2 *mu2_;
    int Mp, Np, mpairs, npairs;
    uint32_t pad;            // column id of absent neighbours (n)
    static constexpr uint32_t ent_end = 0xffffffffu;   // absent checks: offset Mp (row Mp >= m)

    __device__ __forceinline__ EllGraph(const EllImage &img, const uint8_t *gbase, const SurfaceDesc &,
                                        const RoundDesc &, const float *, int, int n_) {
        pad = static_cast<uint32_t>(n_);
        cidx = reinterpret_cast<const IdxT *>(gbase + img.off_cidx);
        cidx2 = reinterpret_cast<const IP *>(cidx);
        vent = reinterpret_cast<const IdxT *>(gbase + img.off_vent);
        vent2 = reinterpret_cast<const IP *>(vent);
        mu_ = reinterpret_cast<const float *>(gbase + img.off_mu);
        mu2_ = reinterpret_cast<const float2 *>(mu_);
        Mp = img.Mp;
        Np = img.Np;
        mpairs = Mp >> 1;
        npairs = Np >> 1;
    }
    // Neighbours of checks 2 pr and 2 pr + 1.
    __device__ __forceinline__ void cols2(int pr, uint32_t (&x)[DC], uint32_t (&y)[DC]) const {
        #pragma unroll
        for (int k = 0; k < DC; ++k) {
            const IP cc = cidx2[k * mpairs + pr];
            x[k] = Idx<IdxT>::lo(cc);
            y[k] = Idx<IdxT>::hi(cc);
        }
    }
    // Message offsets of columns 2 q and 2 q + 1.
    __device__ __forceinline__ void ents2(int q, uint32_t (&x)[DV], uint32_t (&y)[DV]) const {
        #pragma unroll
        for (int k = 0; k < DV; ++k) {
            const IP e = vent2[k * npairs + q];
            x[k] = Idx<IdxT>::lo(e);
            y[k] = Idx<IdxT>::hi(e);
        }
    }
    // Prefetch form for an image in global memory: the raw paired index words
    // of checks 2 pr, 2 pr + 1 (columns 2 q, 2 q + 1), loaded through the
    // read-only path one loop trip ahead of their use, and their unpacking.
    __device__ __forceinline__ void cols2_raw(int pr, IP (&w)[DC]) const {
        #pragma unroll
        for (int k = 0; k < DC; ++k) w[k] = __ldg(cidx2 + k * mpairs + pr);
    }
    __device__ __forceinline__ void ents2_raw(int q, IP (&w)[DV]) const {
        #pragma unroll
        for (int k = 0; k < DV; ++k) w[k] = __ldg(vent2 + k * npairs + q);
    }
    __device__ __forceinline__ float2 mu2_ldg(int q) const { return __ldg(mu2_ + q); }
    template <int N>
    static __device__ __forceinline__ void unpack(const IP (&w)[N], uint32_t (&x)[N], uint32_t (&y)[N]) {
        #pragma unroll
        for (int k = 0; k < N; ++k) {
            x[k] = Idx<IdxT>::lo(w[k]);
            y[k] = Idx<IdxT>::hi(w[k]);
        }
    }
    __device__ __forceinline__ uint32_t col(int k, int c) const { return cidx[k * Mp + c]; }
    __device__ __forceinline__ uint32_t ent(int k, int v) const { return vent[k * Np + v]; }
    __device__ __forceinline__ uint32_t orig(uint32_t v) const { return v; }
    __device__ __forceinline__ float mu(uint32_t v) const { return mu_[v]; }
    __device__ __forceinline__ float2 mu2(int q) const { return mu2_[q]; }
};

template <int DC, int DV>
struct SurfaceGraph {
    static_assert(DC == 6 && DV == 2, "surface-code space-time matrices have DC = 6, DV = 2");
    using IP = uint32_t;     // no index words to prefetch
    static constexpr bool kImage = false;
    static constexpr bool kEll = false;
    SurfaceDesc s;
    const float *mu_tab;     // mu[Np + 2] (global) when mu is not uniform per block
    uint32_t m, n, Mp, R, M0;
    uint32_t pad;            // column id of absent neighbours (n)
    static constexpr uint32_t ent_end = 0xffffffffu;   // absent checks: offset Mp (row Mp >= m)

    __device__ __forceinline__ SurfaceGraph(const EllImage &img, const uint8_t *, const SurfaceDesc &sd,
                                            const RoundDesc &, const float *mt, int m_, int n_)
        : s(sd), mu_tab(mt), m(static_cast<uint32_t>(m_)), n(static_cast<uint32_t>(n_)),
          Mp(static_cast<uint32_t>(img.Mp)), R(static_cast<uint32_t>(img.Mp) + 2u),
          M0(static_cast<uint32_t>(sd.T) * sd.nr), pad(static_cast<uint32_t>(n_)) {}

    // Table III: the six neighbours of check c = t m_r + j (absent ones = n).
    __device__ __forceinline__ void cols(uint32_t c, uint32_t (&v)[DC]) const {
        #pragma unroll
        for (int k = 0; k < DC; ++k) v[k] = n;
        if (c >= m) return;
        const uint32_t t = __umulhi(c, s.mg_mr), j = c - t * s.mr, bd = t * s.nr;
        const uint32_t d = static_cast<uint32_t>(s.d);
        if (s.type == 0) {
            const uint32_t r = __umulhi(j, s.mg_d), cc = j - r * d;
            const uint32_t h = bd + s.d2 + r * (d - 1u) + cc;
            v[0] = bd + j;
            v[1] = bd + j + d;
            if (cc != 0u) v[2] = h - 1u;
            if (cc != d - 1u) v[3] = h;
        } else {
            const uint32_t r = __umulhi(j, s.mg_d1), cc = j - r * (d - 1u);
            const uint32_t h = bd + s.d2 + r * (d - 1u) + cc;
            v[0] = bd + r * d + cc;
            v[1] = v[0] + 1u;
            if (r != 0u) v[2] = h - (d - 1u);
            if (r != d - 1u) v[3] = h;
        }
        int b4 = static_cast<int>(t) - 1;
        if (b4 < 0 && s.cyclic) b4 = s.T - 1;
        if (b4 >= 0 && b4 < s.nb) v[4] = M0 + static_cast<uint32_t>(b4) * s.mr + j;
        if (static_cast<int>(t) < s.nb) v[5] = M0 + t * s.mr + j;
    }
    // Inverse map: the message offsets of column v, checks ascending.
    __device__ __forceinline__ void ents(uint32_t v, uint32_t (&o)[DV]) const {
        o[0] = Mp;
        o[1] = Mp;
        if (v >= n) return;
        const uint32_t d = static_cast<uint32_t>(s.d);
        if (v < M0) {
            const uint32_t t = __umulhi(v, s.mg_nr), q = v - t * s.nr, rb = t * s.mr;
            uint32_t ja = 0, ka = 0, jb = 0, kb = 0;
            bool ha = false, hb = false;          // first / second check present
            if (q < s.d2) {
                if (s.type == 0) {
                    // VN1 of check q - d, VN0 of check q.
                    ha = q >= d;      ja = q - d; ka = 1;
                    hb = q < s.mr;    jb = q;     kb = 0;
                } else {
                    // VN1 of check (r, cc - 1), VN0 of check (r, cc).
                    const uint32_t r = __umulhi(q, s.mg_d), cc = q - r * d, j = r * (d - 1u) + cc;
                    ha = cc >= 1u;     ja = j - 1u; ka = 1;
                    hb = cc + 1u < d;  jb = j;      kb = 0;
                }
            } else {
                const uint32_t qq = q - s.d2;
                if (s.type == 0) {
                    // VN3 of check (r, cc), VN2 of check (r, cc + 1).
                    const uint32_t r = __umulhi(qq, s.mg_d1), cc = qq - r * (d - 1u);
                    ha = true; ja = r * d + cc; ka = 3;
                    hb = true; jb = ja + 1u;    kb = 2;
                } else {
                    // VN3 of check (r, cc), VN2 of check (r + 1, cc).
                    ha = true; ja = qq;           ka = 3;
                    hb = true; jb = qq + d - 1u;  kb = 2;
                }
            }
            const uint32_t oa = ka * R + rb + ja, ob = kb * R + rb + jb;
            if (ha) { o[0] = oa; if (hb) o[1] = ob; }
            else if (hb) { o[0] = ob; }
        } else {
            // Measurement block b: VN5 of check (b, j), VN4 of check (b + 1, j).
            const uint32_t u = v - M0, b = __umulhi(u, s.mg_mr), j = u - b * s.mr;
            const uint32_t b1 = b + 1u == static_cast<uint32_t>(s.T) ? 0u : b + 1u;
            const uint32_t ca = b * s.mr + j, cb = b1 * s.mr + j;
            if (cb > ca) { o[0] = 5u * R + ca; o[1] = 4u * R + cb; }
            else { o[0] = 4u * R + cb; o[1] = 5u * R + ca; }
        }
    }
    __device__ __forceinline__ void cols2(int pr, uint32_t (&x)[DC], uint32_t (&y)[DC]) const {
        cols(2u * static_cast<uint32_t>(pr), x);
        cols(2u * static_cast<uint32_t>(pr) + 1u, y);
    }
    __device__ __forceinline__ void ents2(int q, uint32_t (&x)[DV], uint32_t (&y)[DV]) const {
        ents(2u * static_cast<uint32_t>(q), x);
        ents(2u * static_cast<uint32_t>(q) + 1u, y);
    }
    __device__ __forceinline__ uint32_t col(int k, int c) const {
        uint32_t v[DC];
        cols(static_cast<uint32_t>(c), v);
        uint32_t r = v[0];
        #pragma unroll
        for (int i = 1; i < DC; ++i) if (i == k) r = v[i];
        return r;
    }
    __device__ __forceinline__ uint32_t ent(int k, int v) const {
        uint32_t o[DV];
        ents(static_cast<uint32_t>(v), o);
        return k == 0 ? o[0] : o[1];
    }
    __device__ __forceinline__ uint32_t orig(uint32_t v) const { return v; }
    __device__ __forceinline__ float mu(uint32_t v) const {
        if (v >= n) return __int_as_float(0x7f800000);
        if (s.mu_uniform) return v < M0 ? s.mu_data : s.mu_meas;
        return __ldg(mu_tab + v);
    }
    __device__ __forceinline__ float2 mu2(int q) const {
        return make_float2(mu(2u * static_cast<uint32_t>(q)), mu(2u * static_cast<uint32_t>(q) + 1u));
    }
};

template <int DC, int DV>
struct RoundGraph {
    static_assert(DV >= 2, "a measurement column has two checks");
    using IP = uint32_t;     // no index words to prefetch
    static constexpr bool kImage = true;     // the round image is staged like an index image
    static constexpr bool kEll = false;
    RoundDesc r;
    const uint16_t *rcidx;
    const uint32_t *rvent;
    const float *mu_tab;     // mu[Np + 2] (global) when mu is not uniform per block
    uint32_t m, n, Mp, R, M0;
    uint32_t pad;            // column id of absent neighbours (n)
    static constexpr uint32_t ent_end = 0xffffffffu;   // absent checks: offset Mp (row Mp >= m)

    __device__ __forceinline__ RoundGraph(const EllImage &img, const uint8_t *gbase, const SurfaceDesc &,
                                          const RoundDesc &rd, const float *mt, int m_, int n_)
        : r(rd), rcidx(reinterpret_cast<const uint16_t *>(gbase + rd.off_rcidx)),
          rvent(reinterpret_cast<const uint32_t *>(gbase + rd.off_rvent)), mu_tab(mt),
          m(static_cast<uint32_t>(m_)), n(static_cast<uint32_t>(n_)), Mp(static_cast<uint32_t>(img.Mp)),
          R(static_cast<uint32_t>(img.Mp) + 2u), M0(static_cast<uint32_t>(rd.T) * rd.nr),
          pad(static_cast<uint32_t>(n_)) {}

    // Check c = t m_r + j: the round columns of H_r's row j shifted to round
    // t, then the measurement blocks t - 1 and t (absent ones = n).
    __device__ __forceinline__ void cols(uint32_t c, uint32_t (&v)[DC]) const {
        #pragma unroll
        for (int k = 0; k < DC; ++k) v[k] = n;
        if (c >= m) return;
        const uint32_t t = __umulhi(c, r.mg_mr), j = c - t * r.mr, bd = t * r.nr;
        #pragma unroll
        for (int k = 0; k < DC - 2; ++k) {
            const uint32_t q = rcidx[k * r.mr + j];
            if (q < r.nr) v[k] = bd + q;
        }
        int b4 = static_cast<int>(t) - 1;
        if (b4 < 0 && r.cyclic) b4 = r.T - 1;
        if (b4 >= 0 && b4 < r.nb) v[DC - 2] = M0 + static_cast<uint32_t>(b4) * r.mr + j;
        if (static_cast<int>(t) < r.nb) v[DC - 1] = M0 + t * r.mr + j;
    }
    // Column v: a round column's checks in its round (from the round image),
    // or a measurement column's two checks, ascending.
    __device__ __forceinline__ void ents(uint32_t v, uint32_t (&o)[DV]) const {
        #pragma unroll
        for (int k = 0; k < DV; ++k) o[k] = Mp;
        if (v >= n) return;
        if (v < M0) {
            const uint32_t t = __umulhi(v, r.mg_nr), q = v - t * r.nr, add = t * r.mr;
            #pragma unroll
            for (int k = 0; k < DV; ++k) {
                const uint32_t e = rvent[k * r.nr + q];
                if (e != 0xffffffffu) o[k] = e + add;
            }
        } else {
            // Block b: slot DC - 1 of check (b, j), slot DC - 2 of check (b + 1, j).
            const uint32_t u = v - M0, b = __umulhi(u, r.mg_mr), j = u - b * r.mr;
            const uint32_t b1 = b + 1u == static_cast<uint32_t>(r.T) ? 0u : b + 1u;
            const uint32_t ca = b * r.mr + j, cb = b1 * r.mr + j;
            const uint32_t oa = (DC - 1) * R + ca, ob = (DC - 2) * R + cb;
            if (cb > ca) { o[0] = oa; o[1] = ob; }
            else { o[0] = ob; o[1] = oa; }
        }
    }
    __device__ __forceinline__ void cols2(int pr, uint32_t (&x)[DC], uint32_t (&y)[DC]) const {
        cols(2u * static_cast<uint32_t>(pr), x);
        cols(2u * static_cast<uint32_t>(pr) + 1u, y);
    }
    __device__ __forceinline__ void ents2(int q, uint32_t (&x)[DV], uint32_t (&y)[DV]) const {
        ents(2u * static_cast<uint32_t>(q), x);
        ents(2u * static_cast<uint32_t>(q) + 1u, y);
    }
    __device__ __forceinline__ uint32_t col(int k, int c) const {
        uint32_t v[DC];
        cols(static_cast<uint32_t>(c), v);
        uint32_t x = v[0];
        #pragma unroll
        for (int i = 1; i < DC; ++i) if (i == k) x = v[i];
        return x;
    }
    __device__ __forceinline__ uint32_t ent(int k, int v) const {
        uint32_t o[DV];
        ents(static_cast<uint32_t>(v), o);
        uint32_t x = o[0];
        #pragma unroll
        for (int i = 1; i < DV; ++i) if (i == k) x = o[i];
        return x;
    }
    __device__ __forceinline__ uint32_t orig(uint32_t v) const { return v; }
    __device__ __forceinline__ float mu(uint32_t v) const {
        if (v >= n) return __int_as_float(0x7f800000);
        if (r.mu_uniform) return v < M0 ? r.mu_data : r.mu_meas;
        return __ldg(mu_tab + v);
    }
    __device__ __forceinline__ float2 mu2(int q) const {
        return make_float2(mu(2u * static_cast<uint32_t>(q)), mu(2u * static_cast<uint32_t>(q) + 1u));
    }
};

}  // namespace lbp
