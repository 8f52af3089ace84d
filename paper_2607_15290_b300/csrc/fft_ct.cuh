// fft_ct.cuh -- the register-resident Stockham FFT of fft_line.cuh with the line
// length fixed at compile time (n = 2^LOGN, 64 <= n <= 1024).
//
// Same data placement: thread t of a line holds elements {t + P s : s < E}
// (P = n / E) on entry and on exit.  With the length known, the stage sequence
// (radix-8 stages, then one radix-4 or radix-2 stage for the remaining bits),
// every stride and every twiddle index scale are constants, and each shared-
// memory access is a per-thread base plus a compile-time offset, so a stage costs
// its butterflies, its twiddle products and one load/store per element.
//
// Exchanges between stages alternate between two buffers, so one barrier per
// stage suffices (stage S writes buffer (S + PAR) & 1, stage S + 1 reads it).
// Row layouts pad each exchange differently so that both the strided butterfly
// stores of the stage before and the unit-stride loads of the stage after are
// free of bank conflicts for 8-byte elements:
//   after stage 0 (stride 1):   one pad slot every 16 elements (every 8 when n = 64)
//   after stage 1 (stride 8):   two pad slots every 16 elements
//   after stage 2 (stride 64):  no padding
// For every element e an access touches, (base mod 2^LB) + (offset mod 2^LB) stays
// below 2^LB, so e + PAD (e >> LB) splits into the padded base plus the padded
// offset.  Column tiles interleave TW lines element by element and need no padding.
#pragma once
#include "fft_line.cuh"

namespace llg {
namespace ct {

// stages of radix 2^LR (8, or 16 for lines held 16 points a thread), then one stage for the
// remaining bits
template <int LOGN, int E, int LR = 3>
struct Plan {
    static constexpr int N = 1 << LOGN;
    static constexpr int P = N / E;
    static constexpr int NST = (LOGN + LR - 1) / LR;
    static constexpr int lr(int s) { return s < LOGN / LR ? LR : LOGN % LR; }
    static constexpr int Ns(int s) { return 1 << (LR * s); }
    static_assert(E == 8 || E == 16, "radix-8 stages need E >= 8");
    static_assert((1 << LR) <= E && (LR == 3 || LR == 4), "a stage's radix is 8 or 16, at most E");
    static_assert(LOGN >= 6 && LOGN <= 10, "compile-time plans cover 64..1024");
};

// padded row layout; exchange X is written by stage X (X = 0 also serves the
// unit-stride staging of inputs and outputs)
template <int LOGN>
struct RowL {
    static constexpr int N = 1 << LOGN;
    static constexpr int size = N + N / 8;
    static constexpr int LB(int X) { return (X == 0 && LOGN == 6) ? 3 : 4; }
    static constexpr int PAD(int X) { return X == 0 ? 1 : (X == 1 ? 2 : 0); }
    template <int X> __device__ __forceinline__ static int at(int e) { return e + PAD(X) * (e >> LB(X)); }
    template <int X> static constexpr int off(int c) { return c + PAD(X) * (c >> LB(X)); }
};

// column tile: element e of the line of column c sits at e * SS + c (the caller
// offsets the buffer by c)
template <int SS>
struct ColL {
    template <int X> __device__ __forceinline__ static int at(int e) { return e * SS; }
    template <int X> static constexpr int off(int c) { return c * SS; }
};

template <int SIGN, typename C>
__device__ __forceinline__ C tw_load(const C *__restrict__ tw, int i) {
    C w = ldg_ro(&tw[i]);
    if (SIGN > 0) w.y = -w.y;
    return w;
}

// one Stockham stage S.  DB: two exchange buffers (one barrier per stage); without
// it buf0 == buf1 and a barrier also separates this stage's loads from its stores.
template <int LOGN, int E, int SIGN, class L, int S, int PAR, bool DB, int LR, typename C>
__device__ __forceinline__ void stage(C (&a)[E], C *buf0, C *buf1, int t, const C *__restrict__ tw) {
    using PL = Plan<LOGN, E, LR>;
    constexpr int R = 1 << PL::lr(S), Ns = PL::Ns(S), Q = E / R, P = PL::P, N = PL::N;
    constexpr bool last = S == PL::NST - 1;
    constexpr int TWS = N / (R * Ns);   // twiddle index scale
    if constexpr (S > 0) {
        __syncthreads();   // stage S-1's stores are visible
        const C *src = ((S - 1 + PAR) & 1) ? buf1 : buf0;
        const int b = L::template at<S - 1>(t);
#pragma unroll
        for (int s = 0; s < E; ++s) a[s] = src[b + L::template off<S - 1>(P * s)];
    }
    if constexpr (!DB && !last) __syncthreads();   // single buffer: every load precedes any store
    C *dst = ((S + PAR) & 1) ? buf1 : buf0;
    int kt = 0, b0 = 0;
    if constexpr (Ns <= P) {
        kt = t & (Ns - 1);
        b0 = R * (t - kt) + kt;
    } else {
        b0 = t;
    }
    const int pb = L::template at<S>(b0);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        C b[R];
#pragma unroll
        for (int r = 0; r < R; ++r) b[r] = a[q + r * Q];
        if constexpr (Ns > 1) {
            int k;
            if constexpr (Ns <= P) k = kt;
            else k = t + P * (q % (Ns / P));
#pragma unroll
            for (int r = 1; r < R; ++r) b[r] = cmul(b[r], tw_load<SIGN>(tw, r * k * TWS));
        }
        if constexpr (R == 2) dft2<SIGN>(b[0], b[1]);
        else if constexpr (R == 4) dft4<SIGN>(b[0], b[1], b[2], b[3]);
        else if constexpr (R == 8) dft8<SIGN>(b);
        else dft16<SIGN>(b);
        if constexpr (last) {
#pragma unroll
            for (int r = 0; r < R; ++r) a[q + r * Q] = b[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int c0 = Ns <= P ? R * P * q + r * Ns : R * Ns * (q / (Ns / P)) + P * (q % (Ns / P)) + r * Ns;
                dst[pb + L::template off<S>(c0)] = b[r];
            }
        }
    }
    if constexpr (!last) stage<LOGN, E, SIGN, L, S + 1, PAR, DB, LR>(a, buf0, buf1, t, tw);
}

// Length-2^LOGN DFT (sign SIGN, unnormalised) of the line whose elements t + P s
// thread t holds in a[s], in place.  Stage S stores into buffer (S + PAR) & 1; the
// caller makes sure no thread still reads the buffer stage 0 writes (PAR picks it).
// Every thread of the block calls this (it contains barriers).
template <int LOGN, int E, int SIGN, class L, int PAR = 0, bool DB = true, int LR = 3, typename C>
__device__ __forceinline__ void fft(C (&a)[E], C *buf0, C *buf1, int t, const C *__restrict__ tw) {
    stage<LOGN, E, SIGN, L, 0, PAR, DB, LR>(a, buf0, buf1, t, tw);
}

// ---------------------------------------------------------------- two adjacent FP32 lines

// The same stages for two FP32 lines held by one thread (columns cc and cc + 1 of a
// column tile, ColL layout with even stride SS): every shared-memory access moves both
// lines' elements as one 16-byte word and each twiddle serves both lines.
__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

template <int LOGN, int E, int SIGN, int SS, int S, int PAR, bool DB>
__device__ __forceinline__ void stage2(float2 (&a)[E], float2 (&b)[E], float2 *buf0, float2 *buf1, int t,
                                       const float2 *__restrict__ tw) {
    using PL = Plan<LOGN, E>;
    constexpr int R = 1 << PL::lr(S), Ns = PL::Ns(S), Q = E / R, P = PL::P, N = PL::N;
    constexpr bool last = S == PL::NST - 1;
    constexpr int TWS = N / (R * Ns);
    if constexpr (S > 0) {
        __syncthreads();
        const float2 *src = ((S - 1 + PAR) & 1) ? buf1 : buf0;
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const float4 x = *reinterpret_cast<const float4 *>(&src[(t + P * s) * SS]);
            a[s] = make_float2(x.x, x.y);
            b[s] = make_float2(x.z, x.w);
        }
    }
    if constexpr (!DB && !last) __syncthreads();
    float2 *dst = ((S + PAR) & 1) ? buf1 : buf0;
    int kt = 0, b0 = 0;
    if constexpr (Ns <= P) {
        kt = t & (Ns - 1);
        b0 = R * (t - kt) + kt;
    } else {
        b0 = t;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float2 u[R], w[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { u[r] = a[q + r * Q]; w[r] = b[q + r * Q]; }
        if constexpr (Ns > 1) {
            int k;
            if constexpr (Ns <= P) k = kt;
            else k = t + P * (q % (Ns / P));
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 f = tw_load<SIGN>(tw, r * k * TWS);
                u[r] = cmul(u[r], f);
                w[r] = cmul(w[r], f);
            }
        }
        if constexpr (R == 2) { dft2<SIGN>(u[0], u[1]); dft2<SIGN>(w[0], w[1]); }
        else if constexpr (R == 4) { dft4<SIGN>(u[0], u[1], u[2], u[3]); dft4<SIGN>(w[0], w[1], w[2], w[3]); }
        else { dft8<SIGN>(u); dft8<SIGN>(w); }
        if constexpr (last) {
#pragma unroll
            for (int r = 0; r < R; ++r) { a[q + r * Q] = u[r]; b[q + r * Q] = w[r]; }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int c0 = Ns <= P ? R * P * q + r * Ns : R * Ns * (q / (Ns / P)) + P * (q % (Ns / P)) + r * Ns;
                *reinterpret_cast<float4 *>(&dst[(b0 + c0) * SS]) = pack2(u[r], w[r]);
            }
        }
    }
    if constexpr (!last) stage2<LOGN, E, SIGN, SS, S + 1, PAR, DB>(a, b, buf0, buf1, t, tw);
}

template <int LOGN, int E, int SIGN, int SS, int PAR = 0, bool DB = true>
__device__ __forceinline__ void fft2(float2 (&a)[E], float2 (&b)[E], float2 *buf0, float2 *buf1, int t,
                                     const float2 *__restrict__ tw) {
    stage2<LOGN, E, SIGN, SS, 0, PAR, DB>(a, b, buf0, buf1, t, tw);
}

// the buffer that no stage of a transform with parity PAR reads last, free for the
// caller right after the transform returns
template <int LOGN, int E, int PAR, int LR = 3>
struct FreeBuf { static constexpr int value = (Plan<LOGN, E, LR>::NST - 1 + PAR) & 1; };

}  // namespace ct
}  // namespace llg
