// fpair.cuh -- an FP32-pair scalar (value = hi + lo, |lo| <= half an ulp of hi) with the
// arithmetic operators, for the FP64-accurate Fourier chains run on the FP32 pipes.
//
// On this part FP64 multiply-adds issue about 64 times slower than FP32 ones, and a Fourier
// round trip in FP64 is bound by them.  The same round trip in FP32-pair arithmetic costs
// about ten FP32 operations per FP64 one, moves the same bytes (a pair is 8 bytes, a complex
// pair 16), and carries about 47 significant bits:
//   * sum: Knuth's two-sum of the leading parts (TAOCP vol. 2, 4.2.2), the trailing parts
//     added to its error term, renormalised by a fast two-sum (the "sloppy" double-word
//     addition: its error is a few 2^-48 of |a| + |b|, which is what a normwise FFT error
//     bound needs);
//   * product: Dekker's exact product of the leading parts through a fused multiply-add,
//     plus the cross terms, renormalised (error a few 2^-48 of |a b|);
//   * quotient: an FP32 quotient, one correction from the pair remainder.
// Every operation inside uses the _rn intrinsics, so the compiler cannot contract a product
// into a following sum (which would break the error-free transformations).
//
// FP64 data enter through split_f64 (integer pipes; 47 bits kept) and leave as the FP64 sum
// hi + lo.  The constructor from a double uses FP64 conversions: it serves compile-time
// constants and host-side set-up, not per-element device data.
#pragma once
#include <cuda_runtime.h>
#include "convert.cuh"
#include "f32pair.cuh"

namespace llg {

struct __align__(8) fpair {
    float hi, lo;
    fpair() = default;
    __host__ __device__ constexpr fpair(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit fpair(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr explicit fpair(int i) : hi((float)i), lo(0.0f) {}
};

struct __align__(16) cfpair {
    fpair x, y;
};

template <typename T> struct cplx_t;
template <> struct cplx_t<fpair> { using type = cfpair; };

template <typename T> struct is_fpair { static constexpr bool value = false; };
template <> struct is_fpair<fpair> { static constexpr bool value = true; };

// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ fpair fp_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
    return fpair(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ fpair fp_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return fpair(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ fpair operator-(fpair a) { return fpair(-a.hi, -a.lo); }

__device__ __forceinline__ fpair operator+(fpair a, fpair b) {
    const fpair s = fp_two_sum(a.hi, b.hi);
    return fp_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ fpair operator-(fpair a, fpair b) {
    const fpair s = fp_two_sum(a.hi, -b.hi);
    return fp_fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}
__device__ __forceinline__ fpair operator*(fpair a, fpair b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fp_fast_two_sum(p, e);
}
__device__ __forceinline__ fpair operator/(fpair a, fpair b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const fpair r = a - b * fpair(q1, 0.0f);
    return fp_fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ fpair &operator+=(fpair &a, fpair b) { return a = a + b; }
__device__ __forceinline__ fpair &operator-=(fpair &a, fpair b) { return a = a - b; }
__device__ __forceinline__ fpair &operator*=(fpair &a, fpair b) { return a = a * b; }

// a b + c d with one renormalisation: both leading products exact (fused multiply-add),
// their sum by two-sum, every smaller term gathered in one FP32 correction
__device__ __forceinline__ fpair fp_dot2(fpair a, fpair b, fpair c, fpair d) {
    const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(c.hi, d.hi);
    const fpair s = fp_two_sum(p, q);
    float t = __fmaf_rn(a.hi, b.hi, -p);
    t = __fmaf_rn(a.hi, b.lo, t);
    t = __fmaf_rn(a.lo, b.hi, t);
    t = __fadd_rn(t, __fmaf_rn(c.hi, d.hi, -q));
    t = __fmaf_rn(c.hi, d.lo, t);
    t = __fmaf_rn(c.lo, d.hi, t);
    return fp_fast_two_sum(s.hi, __fadd_rn(t, s.lo));
}

// complex product (the twiddle multiplications of the FFT stages): each part one fp_dot2
__device__ __forceinline__ cfpair cmul(cfpair a, cfpair b) {
    cfpair r;
    r.x = fp_dot2(a.x, b.x, -a.y, b.y);
    r.y = fp_dot2(a.x, b.y, a.y, b.x);
    return r;
}

// conversions of per-element data (see convert.cuh for the FP32 <-> FP64 cases)
template <> __device__ __forceinline__ fpair cvt<fpair, double>(double v) {
    const f32x2 s = split_f64(v);
    return fpair(s.hi, s.lo);
}
template <> __device__ __forceinline__ fpair cvt<fpair, float>(float v) { return fpair(v, 0.0f); }
template <> __device__ __forceinline__ double cvt<double, fpair>(fpair v) { return f2d_exact(v.hi) + f2d_exact(v.lo); }
template <> __device__ __forceinline__ float cvt<float, fpair>(fpair v) { return __fadd_rn(v.hi, v.lo); }

// read-only loads through the non-coherent cache, for the scalar and complex pair types too
template <typename T> __device__ __forceinline__ T ldg_ro(const T *p) { return __ldg(p); }
template <> __device__ __forceinline__ fpair ldg_ro<fpair>(const fpair *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return fpair(v.x, v.y);
}
template <> __device__ __forceinline__ cfpair ldg_ro<cfpair>(const cfpair *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    cfpair r;
    r.x = fpair(v.x, v.y);
    r.y = fpair(v.z, v.w);
    return r;
}

}  // namespace llg
