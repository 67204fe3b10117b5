// Device helpers shared by the BP kernels: message storage types, group
// barriers, the lottery's counter-based generator and the normalisation
// factor.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "internal.h"

namespace lbp {

// ------------------------------------------------------------ message types

template <typename T> struct Msg;
// store_signed(mag, sgn): the stored message of value (sgn ? -mag : mag) for
// mag >= 0 and sgn in {0, 0x80000000}; every storage rounding is symmetric
// (round to nearest even, symmetric saturation), so rounding the magnitude
// and then applying the sign equals rounding the signed value.
template <> struct Msg<float> {
    static __device__ __forceinline__ float load(float x) { return x; }
    static __device__ __forceinline__ float store(float x) { return x; }
    static __device__ __forceinline__ float store_signed(float mag, uint32_t sgn) {
        return __uint_as_float(__float_as_uint(mag) ^ sgn);
    }
};
template <> struct Msg<__half> {
    static __device__ __forceinline__ float load(__half x) { return __half2float(x); }
    static __device__ __forceinline__ __half store(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ __half store_signed(float mag, uint32_t sgn) {
        return __ushort_as_half(static_cast<unsigned short>(__half_as_ushort(__float2half_rn(mag)) ^ (sgn >> 16)));
    }
};
// Int3.4: q = clamp(rne(16 x), -127, 127), value q / 16.
template <> struct Msg<int8_t> {
    static __device__ __forceinline__ float load(int8_t q) { return __fmul_rn(static_cast<float>(q), 0.0625f); }
    static __device__ __forceinline__ int8_t store(float x) {
        int q = __float2int_rn(__fmul_rn(16.0f, x));
        q = q > 127 ? 127 : (q < -127 ? -127 : q);
        return static_cast<int8_t>(q);
    }
    static __device__ __forceinline__ int8_t store_signed(float mag, uint32_t sgn) {
        int q = __float2int_rn(__fmul_rn(16.0f, mag));
        q = q > 127 ? 127 : q;
        return static_cast<int8_t>(sgn ? -q : q);
    }
};

// Two adjacent messages of one slot row, loaded / stored as one access.
template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<__half> { using type = __half2; };
template <> struct Pair<int8_t> { using type = char2; };

template <typename T> __device__ __forceinline__ T pair_lo(typename Pair<T>::type p);
template <typename T> __device__ __forceinline__ T pair_hi(typename Pair<T>::type p);
template <> __device__ __forceinline__ float pair_lo<float>(float2 p) { return p.x; }
template <> __device__ __forceinline__ float pair_hi<float>(float2 p) { return p.y; }
template <> __device__ __forceinline__ __half pair_lo<__half>(__half2 p) { return __low2half(p); }
template <> __device__ __forceinline__ __half pair_hi<__half>(__half2 p) { return __high2half(p); }
template <> __device__ __forceinline__ int8_t pair_lo<int8_t>(char2 p) { return p.x; }
template <> __device__ __forceinline__ int8_t pair_hi<int8_t>(char2 p) { return p.y; }
__device__ __forceinline__ float2 make_pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ __half2 make_pair(__half a, __half b) { return __halves2half2(a, b); }
__device__ __forceinline__ char2 make_pair(int8_t a, int8_t b) { return make_char2(a, b); }

// -------------------------------------------------------------- group sync
//
// Named barriers over the G threads of one group.  They use the non-.aligned
// PTX forms (barrier.sync, barrier.red): the .aligned forms (bar.sync,
// bar.red) require every thread of a warp to execute the barrier together,
// and the kernels reach these barriers right after code whose trip counts or
// branches differ between the lanes of a warp (strided loops over checks and
// columns, lane-0 stores, the lottery warp's scans).  The non-aligned forms
// count arriving threads one by one, so a warp that has not reconverged
// still synchronises correctly.

template <int G>
__device__ __forceinline__ void group_sync(int bar) {
    if (G == 32) {
        __syncwarp();
    } else {
        asm volatile("barrier.sync %0, %1;" ::"r"(bar), "r"(G) : "memory");
    }
}

// Barrier that also ORs a predicate over the group.
template <int G>
__device__ __forceinline__ bool group_sync_or(int bar, bool p) {
    if (G == 32) {
        return __any_sync(0xffffffffu, p);
    } else {
        unsigned r;
        asm volatile(
            "{\n\t.reg .pred pi, po;\n\t"
            "setp.ne.u32 pi, %1, 0;\n\t"
            "barrier.red.or.pred po, %2, %3, pi;\n\t"
            "selp.u32 %0, 1, 0, po;\n\t}"
            : "=r"(r)
            : "r"(static_cast<unsigned>(p)), "r"(bar), "r"(G)
            : "memory");
        return r != 0;
    }
}

// SplitMix64 (Steele, Lea, Flood 2014), output number counter+1 of the stream
// whose state starts at seed.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Gallager's function phi(x) = ln((e^x + 1) / (e^x - 1)) = -ln tanh(x / 2)
// for x >= 0, written as log1p(2 / expm1(x)) so that it keeps full relative
// accuracy at both ends: phi(0) = +inf, phi(+inf) = 0, and phi(phi(x)) = x.
// The sum-product magnitude 2 atanh(prod tanh(|alpha_k| / 2)) equals
// phi(sum_k phi(|alpha_k|)); the product form loses everything above
// |beta| ~ 17 in binary32 (tanh rounds to 1), this form does not.
__device__ __forceinline__ float gallager_phi(float x) {
    return log1pf(__fdiv_rn(2.0f, expm1f(x)));
}

// Saturation of sum-product message magnitudes (phi of an empty or
// vanishing sum is infinite).
constexpr float kSpMaxMag = 25.0f;

// Normalisation factor at iteration i, binary32: the constant, or
// 1 - 2^-(i+1) rounded to nearest (exact for i + 1 <= 24, 1.0 beyond).
__device__ __forceinline__ float scale_at(int mode, float c, int i) {
    if (mode == LBP_SCALE_CONST) return c;
    const int k = i + 1;
    if (k >= 25) return 1.0f;
    return __fsub_rn(1.0f, __int_as_float((127 - k) << 23));
}

}  // namespace lbp
