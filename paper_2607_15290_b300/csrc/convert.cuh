// convert.cuh -- FP32 <-> FP64 conversions on the integer pipes.
//
// On this part the hardware conversion instructions between float and double issue to
// the FP64 unit and run at its multiply-add rate (measured: about 560 G conversions/s,
// the same as the FP64 FMA rate), which makes a loop such as x += Z y with FP32 Z as
// slow as twice its FP64 multiply-adds.  These routines build the IEEE bit pattern of
// the result with 32-bit integer operations instead.  Both return exactly what the
// hardware conversion returns: f2d_exact was compared on all 2^32 float patterns,
// d2f_rn (round to nearest, ties to even) on 8.4 million random, tie, overflow and
// subnormal-range doubles; NaNs stay NaNs (payloads are kept where the format allows).
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace llg {

// float -> double (exact: every float is a double)
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned s = u & 0x80000000u;
    unsigned e = (u >> 23) & 0xffu;
    unsigned mant = u & 0x7fffffu;
    unsigned ebias = 896u;   // 1023 - 127
    if (e == 0u) {
        // zero or subnormal: scaling by 2^64 in FP32 is exact and makes a subnormal normal;
        // the exponent bias then takes the 64 back off
        const unsigned u2 = __float_as_uint(f * 18446744073709551616.0f);
        e = (u2 >> 23) & 0xffu;
        mant = u2 & 0x7fffffu;
        ebias = 832u;
    }
    unsigned hi;
    if (e == 0u) hi = s;
    else if (e == 255u) hi = s | 0x7ff00000u | (mant >> 3);
    else hi = s | ((e + ebias) << 20) | (mant >> 3);
    const unsigned lo = e == 0u ? 0u : (mant << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// double -> float, rounded to nearest (ties to even), overflow to infinity, results
// below the normal range rounded into the subnormals
__device__ __forceinline__ float d2f_rn(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const unsigned s = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const int fe = e - 896;
    if (fe >= 1 && fe < 255) {
        // normal range: keep 23 mantissa bits, round on the 29 dropped ones; a carry out of
        // the mantissa moves into the exponent (and from the largest binade to infinity)
        const unsigned rest = lo & 0x1fffffffu;
        const unsigned rnd = (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
        return __uint_as_float(s | (((unsigned)fe << 23) + m23 + rnd));
    }
    if (e == 0x7ff) {
        const bool nan = ((hi & 0xfffffu) | lo) != 0u;
        return __uint_as_float(s | 0x7f800000u | (nan ? (m23 | 0x400000u) : 0u));
    }
    if (fe >= 255) return __uint_as_float(s | 0x7f800000u);
    // below the normal range: the value is M 2^(e - 1075) with M = 2^52 + mantissa, i.e.
    // M 2^-(926 - e) units of the smallest subnormal 2^-149
    const int sh = 926 - e;
    if (e == 0 || sh > 54) return __uint_as_float(s);
    const unsigned long long M = (1ull << 52) | (u & 0xfffffffffffffull);
    const unsigned long long q = M >> sh, rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    const unsigned rnd = (rem > half || (rem == half && (q & 1ull))) ? 1u : 0u;
    return __uint_as_float(s | ((unsigned)q + rnd));
}

// widening and narrowing by the routines above; same-type overloads are the identity
__device__ __forceinline__ double to_f64(float v) { return f2d_exact(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return d2f_rn(v); }
__device__ __forceinline__ float to_f32(float v) { return v; }

// (To) v with the FP32 <-> FP64 cases routed through the routines above
template <typename To, typename From>
__device__ __forceinline__ To cvt(From v) {
    if constexpr (std::is_same<To, double>::value && std::is_same<From, float>::value) return f2d_exact(v);
    else if constexpr (std::is_same<To, float>::value && std::is_same<From, double>::value) return d2f_rn(v);
    else return (To)v;
}

}  // namespace llg
