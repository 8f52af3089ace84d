// f32pair.cuh -- FP64 data carried through the Gram--Schmidt passes as pairs of FP32
// values (hi + lo), so that the multiply-adds run on the FP32 pipes instead of the FP64
// unit (on this part FP64 multiply-adds issue about 70 times slower than FP32 ones).
//
// Arithmetic (all error-free transformations in round-to-nearest FP32):
//   * split: a double d becomes hi = d truncated to 24 significant bits and lo = the next
//     23 bits, built from the bit fields with integer operations (the hardware
//     double->float conversion issues to the FP64 unit).  |d - (hi + lo)| < 2^-46 |d|.
//     Doubles with |d| < 2^-80 become (0, 0); |d| >= 2^128 becomes (+-inf, 0).
//   * product: Dekker's exact product of the leading parts through a fused multiply-add
//     (ph + e = ah bh exactly), plus the cross terms ah bl + al bh; al bl (< 2^-46 of the
//     product) is dropped.
//   * sum: Knuth's two-sum (Knuth, TAOCP vol. 2, 4.2.2), valid for any ordering of the
//     operands' magnitudes; rounding errors of the running sum go to a separate FP32
//     accumulator.
// Every addition and product inside a transformation uses the _rn intrinsics, so the
// compiler cannot contract a product into a following addition (which would destroy the
// exactness the transformations rely on).  A sum of n such products is accurate to about
// n 2^-46 relative to the sum of the magnitudes, between the FP32 and FP64 levels
// (FP64 multiply-adds: about n 2^-53).
#pragma once
#include <cuda_runtime.h>
#include "convert.cuh"

namespace llg {

struct f32x2 {
    float hi, lo;
};

__device__ __forceinline__ f32x2 split_f64(double d) {
    const unsigned H = (unsigned)__double2hiint(d), Lw = (unsigned)__double2loint(d);
    const unsigned s = H & 0x80000000u;
    const unsigned E = (H >> 20) & 0x7ffu;
    // hi: sign | (E - 896) << 23 | top 23 stored mantissa bits (valid for E in [897, 1150];
    // bit 31 of the shifted field is then zero and takes the sign)
    const float hi = __uint_as_float(__funnelshift_l(Lw, H - (896u << 20), 3) | s);
    // lo: stored mantissa bits 28..6 as an exact FP32 integer (2^23 + r - 2^23), scaled by
    // +-2^(E - 1069) (a normal FP32 power of two for E in [943, 1196])
    const float r = __fsub_rn(__uint_as_float(((Lw >> 6) & 0x7fffffu) | 0x4b000000u), 8388608.0f);
    const float sc = __uint_as_float(s | (((H & 0x7ff00000u) - (942u << 20)) << 3));
    const bool ok = E - 943u <= 1150u - 943u;
    f32x2 o;
    o.hi = ok ? hi : (E > 1150u ? __uint_as_float(s | 0x7f800000u) : 0.0f);
    o.lo = ok ? __fmul_rn(r, sc) : 0.0f;
    return o;
}

// s += a * b
__device__ __forceinline__ void fma_acc(const f32x2 &a, const f32x2 &b, f32x2 &s) {
    const float ph = __fmul_rn(a.hi, b.hi);
    float pl = __fmaf_rn(a.hi, b.hi, -ph);
    pl = __fmaf_rn(a.hi, b.lo, pl);
    pl = __fmaf_rn(a.lo, b.hi, pl);
    const float t = __fadd_rn(s.hi, ph);
    const float bv = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bv)), __fsub_rn(ph, bv));
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, pl));
    s.hi = t;
}

// a - b, renormalised (|lo| <= half an ulp of hi)
__device__ __forceinline__ f32x2 sub_pair(const f32x2 &a, const f32x2 &b) {
    const float t = __fsub_rn(a.hi, b.hi);
    const float bv = __fsub_rn(t, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, bv)), __fsub_rn(-b.hi, bv));
    const float lo = __fadd_rn(err, __fsub_rn(a.lo, b.lo));
    f32x2 o;
    o.hi = __fadd_rn(t, lo);
    o.lo = __fsub_rn(lo, __fsub_rn(o.hi, t));
    return o;
}

// hi + lo as a double (both widened exactly on the integer pipes, one FP64 addition)
__device__ __forceinline__ double pair_to_f64(const f32x2 &a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }

}  // namespace llg
