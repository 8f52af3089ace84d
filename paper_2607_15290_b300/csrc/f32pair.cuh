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

// ---- two FP32 pairs in packed registers: the same transformations on two independent values
// at once with the packed FP32 instructions (add/sub/mul/fma .f32x2, round to nearest): half
// the instructions, and two independent dependency chains per instruction.  Lane 0 of each
// 64-bit register belongs to the first value, lane 1 to the second.
typedef unsigned long long f32v2;
struct f32x2v2 {
    f32v2 hi, lo;
};

__device__ __forceinline__ f32v2 v2_pack(float a, float b) {
    f32v2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void v2_unpack(f32v2 v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f32v2 v2_add(f32v2 a, f32v2 b) {
    f32v2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32v2 v2_sub(f32v2 a, f32v2 b) {
    f32v2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32v2 v2_mul(f32v2 a, f32v2 b) {
    f32v2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32v2 v2_fma(f32v2 a, f32v2 b, f32v2 c) {
    f32v2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32v2 v2_neg(f32v2 a) { return a ^ 0x8000000080000000ull; }

// s += a * b in both lanes (fma_acc)
__device__ __forceinline__ void fma_acc_v2(const f32x2v2 &a, const f32x2v2 &b, f32x2v2 &s) {
    const f32v2 ph = v2_mul(a.hi, b.hi);
    f32v2 pl = v2_fma(a.hi, b.hi, v2_neg(ph));
    pl = v2_fma(a.hi, b.lo, pl);
    pl = v2_fma(a.lo, b.hi, pl);
    const f32v2 t = v2_add(s.hi, ph);
    const f32v2 bv = v2_sub(t, s.hi);
    const f32v2 err = v2_add(v2_sub(s.hi, v2_sub(t, bv)), v2_sub(ph, bv));
    s.lo = v2_add(s.lo, v2_add(err, pl));
    s.hi = t;
}

// a - b renormalised, in both lanes (sub_pair)
__device__ __forceinline__ f32x2v2 sub_pair_v2(const f32x2v2 &a, const f32x2v2 &b) {
    const f32v2 t = v2_sub(a.hi, b.hi);
    const f32v2 bv = v2_sub(t, a.hi);
    const f32v2 err = v2_add(v2_sub(a.hi, v2_sub(t, bv)), v2_sub(v2_neg(b.hi), bv));
    const f32v2 lo = v2_add(err, v2_sub(a.lo, b.lo));
    f32x2v2 o;
    o.hi = v2_add(t, lo);
    o.lo = v2_sub(lo, v2_sub(o.hi, t));
    return o;
}

// the two lanes' values hi + lo summed as doubles
__device__ __forceinline__ double pair_v2_to_f64(const f32x2v2 &a) {
    float h0, h1, l0, l1;
    v2_unpack(a.hi, h0, h1);
    v2_unpack(a.lo, l0, l1);
    return (f2d_exact(h0) + f2d_exact(l0)) + (f2d_exact(h1) + f2d_exact(l1));
}

}  // namespace llg
