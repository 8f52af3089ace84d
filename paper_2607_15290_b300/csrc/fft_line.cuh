// fft_line.cuh -- register-resident Stockham FFT of one line held by a group
// of P threads, with shared memory used only between radix stages.
//
// Thread t of a line holds the E elements {t + P*s : s < E} in registers
// (P = n / E).  Every Stockham stage reads its radix-R butterfly inputs
// j + r*n/R (j = t + P*q) from exactly that set, and the final stage writes
// its outputs back onto the same set, so a forward transform, a pointwise
// symbol and an inverse transform chain in registers without a shared-memory
// round trip at the junction.  Twiddles come from a per-length table
// tw[i] = exp(-2 pi i * i / n) (computed on the host in long double), so no
// sin/cos is evaluated on the device.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "fpair.cuh"

namespace llg {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
// SIGN * v for SIGN = +-1 (a negation, for every scalar type)
template <int SIGN, typename T> __device__ __forceinline__ T sgn(T v) { return SIGN > 0 ? v : -v; }
// multiply by SIGN * i
template <int SIGN, typename C> __device__ __forceinline__ C cmul_i(C a) {
    return SIGN > 0 ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

// in-register DFTs of radix 2, 4, 8 (sign SIGN in the exponent, unnormalised)
template <int SIGN, typename C> __device__ __forceinline__ void dft2(C &a0, C &a1) {
    C t = csub(a0, a1);
    a0 = cadd(a0, a1);
    a1 = t;
}
template <int SIGN, typename C> __device__ __forceinline__ void dft4(C &a0, C &a1, C &a2, C &a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = cmul_i<SIGN>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}
template <int SIGN, typename C> __device__ __forceinline__ void dft8(C (&a)[8]) {
    using T = decltype(C::x);
    const T h = (T)0.70710678118654752440084436210485;
    C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<SIGN>(e0, e1, e2, e3);
    dft4<SIGN>(o0, o1, o2, o3);
    // o_k *= W8^k, W8 = exp(SIGN 2 pi i / 8)
    C w1 = cmk<C>((o1.x - sgn<SIGN>(o1.y)) * h, (o1.y + sgn<SIGN>(o1.x)) * h);
    C w2 = cmul_i<SIGN>(o2);
    C w3 = cmk<C>((-o3.x - sgn<SIGN>(o3.y)) * h, (-o3.y + sgn<SIGN>(o3.x)) * h);
    a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
    a[1] = cadd(e1, w1); a[5] = csub(e1, w1);
    a[2] = cadd(e2, w2); a[6] = csub(e2, w2);
    a[3] = cadd(e3, w3); a[7] = csub(e3, w3);
}

// 16-point DFT as 4 x 4: DFTs of the four decimated sets {n2, n2 + 4, n2 + 8, n2 + 12}, the
// twiddles W16^(n2 k1), then DFTs across n2; output k1 + 4 k2 in natural order
template <int SIGN, typename C> __device__ __forceinline__ void dft16(C (&a)[16]) {
    using T = decltype(C::x);
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;   // cos, sin of pi/8
    const T h = (T)0.70710678118654752440;
    C y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C p0 = a[n2], p1 = a[n2 + 4], p2 = a[n2 + 8], p3 = a[n2 + 12];
        dft4<SIGN>(p0, p1, p2, p3);
        y[n2][0] = p0; y[n2][1] = p1; y[n2][2] = p2; y[n2][3] = p3;
    }
    // W16^m = cos(2 pi m / 16) + SIGN i sin(2 pi m / 16)
    y[1][1] = cmul(y[1][1], cmk<C>(c1, sgn<SIGN>(s1)));
    y[1][2] = cmul(y[1][2], cmk<C>(h, sgn<SIGN>(h)));
    y[1][3] = cmul(y[1][3], cmk<C>(s1, sgn<SIGN>(c1)));
    y[2][1] = cmul(y[2][1], cmk<C>(h, sgn<SIGN>(h)));
    y[2][2] = cmul_i<SIGN>(y[2][2]);
    y[2][3] = cmul(y[2][3], cmk<C>(-h, sgn<SIGN>(h)));
    y[3][1] = cmul(y[3][1], cmk<C>(s1, sgn<SIGN>(c1)));
    y[3][2] = cmul(y[3][2], cmk<C>(-h, sgn<SIGN>(h)));
    y[3][3] = cmul(y[3][3], cmk<C>(-c1, -sgn<SIGN>(s1)));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C q0 = y[0][k1], q1 = y[1][k1], q2 = y[2][k1], q3 = y[3][k1];
        dft4<SIGN>(q0, q1, q2, q3);
        a[k1] = q0; a[k1 + 4] = q1; a[k1 + 8] = q2; a[k1 + 12] = q3;
    }
}

// Shared-memory index of element e of a line: rows use a padded contiguous
// layout (one pad slot every 8 elements kills the stride-R bank conflicts of
// the first stages); column tiles interleave TW lines element by element.
struct RowLayout {
    __device__ __forceinline__ static int idx(int e, int /*SS*/) { return e + (e >> 3); }
    __host__ __device__ static int size(int n) { return n + (n >> 3); }
};
struct ColLayout {
    __device__ __forceinline__ static int idx(int e, int SS) { return e * SS; }
};

template <int R, int E, int SIGN, typename Layout, typename C>
__device__ __forceinline__ void stockham_stage(C (&a)[E], C *sm, int SS, int n, int logn, int t, int P,
                                               int Ns, int logNs, bool last, const C *__restrict__ tw) {
    constexpr int Q = E / R;
    const int tws = logn - logNs - (R == 8 ? 3 : (R == 4 ? 2 : 1)); // log2(n / (Ns R))
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int j = t + P * q;
        const int k = j & (Ns - 1);
        C b[R];
#pragma unroll
        for (int r = 0; r < R; ++r) b[r] = a[q + r * Q];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = __ldg(&tw[(r * k) << tws]);
                if (SIGN > 0) w.y = -w.y;
                b[r] = cmul(b[r], w);
            }
        }
        if constexpr (R == 2) {
            dft2<SIGN>(b[0], b[1]);
        } else if constexpr (R == 4) {
            dft4<SIGN>(b[0], b[1], b[2], b[3]);
        } else {
            dft8<SIGN>(b);
        }
        if (last) {
#pragma unroll
            for (int r = 0; r < R; ++r) a[q + r * Q] = b[r];
        } else {
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[Layout::idx(base + r * Ns, SS)] = b[r];
        }
    }
}

// Full length-n DFT of one line.  On entry and exit a[s] = element (t + P s).
// Every thread of the block must call this (it contains __syncthreads); lines
// of one block all have the same length.
template <int E, int SIGN, typename Layout, typename C>
__device__ __forceinline__ void line_fft(C (&a)[E], C *sm, int SS, int n, int logn, int t, int P,
                                         const C *__restrict__ tw) {
    int Ns = 1, logNs = 0, rem = logn;
    bool first = true;
    while (rem > 0) {
        const int lr = (rem >= 3 && E >= 8) ? 3 : ((rem >= 2 && E >= 4) ? 2 : 1);
        const bool last = (rem == lr);
        if (!first) {
#pragma unroll
            for (int s = 0; s < E; ++s) a[s] = sm[Layout::idx(t + P * s, SS)];
        }
        __syncthreads();   // all reads of this stage (and the caller's) precede any write
        if (lr == 3) {
            if constexpr (E >= 8) stockham_stage<8, E, SIGN, Layout>(a, sm, SS, n, logn, t, P, Ns, logNs, last, tw);
        } else if (lr == 2) {
            if constexpr (E >= 4) stockham_stage<4, E, SIGN, Layout>(a, sm, SS, n, logn, t, P, Ns, logNs, last, tw);
        } else {
            stockham_stage<2, E, SIGN, Layout>(a, sm, SS, n, logn, t, P, Ns, logNs, last, tw);
        }
        if (!last) __syncthreads();
        Ns <<= lr;
        logNs += lr;
        rem -= lr;
        first = false;
    }
}

// ---------------------------------------------------------------- nodal algebra

// (S~_i + lambda I)^{-1} x = (lambda I - S~_i) x / (lambda^2 + |m|^2)   (Sec. 3.2, eq. inverse S)
// transpose: (S~_i + lambda I)^{-T} x = (lambda I + S~_i) x / (lambda^2 + |m|^2)
template <typename T, bool TRANSPOSE>
__device__ __forceinline__ void nodal_inverse(T m1, T m2, T m3, T lam, T x1, T x2, T x3, T x4,
                                              T &z1, T &z2, T &z3, T &z4) {
    const T d = (T)1 / (lam * lam + m1 * m1 + m2 * m2 + m3 * m3);
    const T s = TRANSPOSE ? (T)1 : (T)-1;
    const T c1 = m2 * x3 - m3 * x2, c2 = m3 * x1 - m1 * x3, c3 = m1 * x2 - m2 * x1;
    z1 = (lam * x1 + s * (c1 + m1 * x4)) * d;
    z2 = (lam * x2 + s * (c2 + m2 * x4)) * d;
    z3 = (lam * x3 + s * (c3 + m3 * x4)) * d;
    z4 = (lam * x4 - s * (m1 * x1 + m2 * x2 + m3 * x3)) * d;
}

}  // namespace llg
