// spectral_kernels.cuh -- the three pass kernels of a Fourier round trip (x-pass
// forward with the nodal prologue, axis passes with the Fourier multiplier,
// x-pass inverse with the nodal epilogue) and their argument structures.
// Included by every translation unit that launches them.
#pragma once
#include "llg_internal.h"
#include "fft_line.cuh"

namespace llg {

template <typename T> using cplx = typename cplx_t<T>::type;

template <typename T, typename TIn, typename TOut>
struct RowArgs {
    cplx<T> *spec;
    const cplx<T> *tw0;
    int n0, logn0, S, G;
    long long rows, N;
    NodalIO<TIn, TOut, T> io;
};

template <typename T>
struct ColArgs {
    cplx<T> *spec;
    const cplx<T> *tw;
    long long ls, bs;
    int nl, logn, n0, S;
    const T *tx, *tl, *tb;
    T sa, sb, sscale;
    int sinv;
};

template <typename TIn, typename TOut, typename T>
__device__ __forceinline__ T in_scale(const NodalIO<TIn, TOut, T> &io) {
    return io.scale ? (T)(*io.scale) : (T)1;
}

// ------------------------------------------------------------------ x-pass forward

template <typename T, typename TIn, typename TOut, int E, int IN>
__global__ void __launch_bounds__(512) row_fwd_kernel(RowArgs<T, TIn, TOut> a) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int n0 = a.n0, P = n0 / E, LS = RowLayout::size(n0);
    const long long N = a.N, npairs = a.rows / 2, pair0 = (long long)blockIdx.x * a.G;
    const NodalIO<TIn, TOut, T> &io = a.io;
    const T s = in_scale(io);

    // prologue: node-parallel, coalesced plane loads, staged into shared memory
    for (int idx = threadIdx.x; idx < 2 * a.G * n0; idx += blockDim.x) {
        const int gp = idx / (2 * n0), rr = (idx / n0) & 1, xx = idx % n0;
        const long long pair = pair0 + gp;
        if (pair >= npairs) continue;
        const long long j = (2 * pair + rr) * n0 + xx;
        T u1, u2, u3;
        if constexpr (IN == IN_V) {
            u1 = s * (T)io.x[j];
            u2 = s * (T)io.x[N + j];
            u3 = s * (T)io.x[2 * N + j];
        } else if constexpr (IN == IN_M) {
            u1 = (T)io.x[j];
            u2 = (T)io.x[N + j];
            u3 = (T)io.x[2 * N + j];
        } else if constexpr (IN == IN_FUSED) {
            const T m1 = io.m[j], m2 = io.m[N + j], m3 = io.m[2 * N + j];
            const T v1 = s * (T)io.x[j], v2 = s * (T)io.x[N + j], v3 = s * (T)io.x[2 * N + j];
            const T r = s * (T)io.x[3 * N + j];
            u1 = m2 * v3 - m3 * v2 + m1 * r - io.lam * v1;
            u2 = m3 * v1 - m1 * v3 + m2 * r - io.lam * v2;
            u3 = m1 * v2 - m2 * v1 + m3 * r - io.lam * v3;
        } else {  // IN_NODAL_T
            const T m1 = io.m[j], m2 = io.m[N + j], m3 = io.m[2 * N + j];
            T z4;
            nodal_inverse<T, true>(m1, m2, m3, io.lam, s * (T)io.x[j], s * (T)io.x[N + j],
                                   s * (T)io.x[2 * N + j], s * (T)io.x[3 * N + j], u1, u2, u3, z4);
            io.y[3 * N + j] = (TOut)(z4 / io.lam);
        }
        sm[(3 * gp + rr) * LS + RowLayout::idx(xx, 1)] = cmk<C>(u1, u2);
        reinterpret_cast<T *>(&sm[(3 * gp + 2) * LS + RowLayout::idx(xx, 1)])[rr] = u3;
    }
    __syncthreads();

    const int line = threadIdx.x / P, t = threadIdx.x % P;
    const int gp = line / 3, kind = line % 3;
    const long long pair = pair0 + gp;
    const bool valid = pair < npairs;
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = sm[line * LS + RowLayout::idx(t + P * q, 1)];
    line_fft<E, -1, RowLayout>(v, sm + line * LS, 1, n0, a.logn0, t, P, a.tw0);
    if (kind < 2) {
        if (valid) {
            C *dst = a.spec + (2 * pair + kind) * (long long)a.S;
#pragma unroll
            for (int q = 0; q < E; ++q) dst[t + P * q] = v[q];
        }
    } else {
#pragma unroll
        for (int q = 0; q < E; ++q) sm[line * LS + RowLayout::idx(t + P * q, 1)] = v[q];
    }
    __syncthreads();
    if (kind == 2 && valid) {
        // U = FFT(c3[ya] + i c3[yb]);  C_a = (U_k + conj U_{-k}) / 2,  C_b = (U_k - conj U_{-k}) / (2i)
        C *da = a.spec + (2 * pair) * (long long)a.S + n0;
        C *db = da + a.S;
        for (int k = t; k <= n0 / 2; k += P) {
            const C uk = sm[line * LS + RowLayout::idx(k, 1)];
            const C um = sm[line * LS + RowLayout::idx((n0 - k) & (n0 - 1), 1)];
            da[k] = cmk<C>((T)0.5 * (uk.x + um.x), (T)0.5 * (uk.y - um.y));
            db[k] = cmk<C>((T)0.5 * (uk.y + um.y), (T)-0.5 * (uk.x - um.x));
        }
    }
}

// ------------------------------------------------------------------ axis passes

template <typename T, int E, int TW, int MODE>   // MODE bit 1: forward, bit 2: inverse, 4: multiplier
__global__ void __launch_bounds__(512) col_kernel(ColArgs<T> a) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int c = threadIdx.x % TW, t = threadIdx.x / TW;
    const int P = a.nl / E;
    const int col = blockIdx.x * TW + c;
    C *base = a.spec + (long long)blockIdx.y * a.bs + col;
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = base[(long long)(t + P * q) * a.ls];
    if (MODE & 1) line_fft<E, -1, ColLayout>(v, sm + c, TW, a.nl, a.logn, t, P, a.tw);
    if (MODE & 4) {
        const int hn = a.n0 / 2;
        const bool live = col <= a.n0 + hn;
        const T sx = live ? a.tx[col < a.n0 ? col : col - a.n0] : (T)0;
        const T sb = a.tb ? a.tb[blockIdx.y] : (T)0;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const T sig = sx + a.tl[t + P * q] + sb;
            const T d = a.sa + a.sb * sig;
            const T mult = live ? (a.sinv ? a.sscale / d : a.sscale * d) : (T)0;
            v[q] = cscale(v[q], mult);
        }
    }
    if (MODE & 2) line_fft<E, +1, ColLayout>(v, sm + c, TW, a.nl, a.logn, t, P, a.tw);
#pragma unroll
    for (int q = 0; q < E; ++q) base[(long long)(t + P * q) * a.ls] = v[q];
}

// ------------------------------------------------------------------ x-pass inverse

template <typename T, typename TIn, typename TOut, int E, int OUT>
__global__ void __launch_bounds__(512) row_inv_kernel(RowArgs<T, TIn, TOut> a) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int n0 = a.n0, P = n0 / E, LS = RowLayout::size(n0), hn = n0 / 2;
    const long long N = a.N, npairs = a.rows / 2, pair0 = (long long)blockIdx.x * a.G;
    const int line = threadIdx.x / P, t = threadIdx.x % P;
    const int gp = line / 3, kind = line % 3;
    const long long pair = pair0 + gp;
    const bool valid = pair < npairs;
    C v[E];
    if (valid) {
        if (kind < 2) {
            const C *src = a.spec + (2 * pair + kind) * (long long)a.S;
#pragma unroll
            for (int q = 0; q < E; ++q) v[q] = src[t + P * q];
        } else {
            const C *sa = a.spec + (2 * pair) * (long long)a.S + n0;
            const C *sb = sa + a.S;
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const int k = t + P * q;
                const int kk = k <= hn ? k : n0 - k;
                C ca = sa[kk], cb = sb[kk];
                if (k > hn) { ca.y = -ca.y; cb.y = -cb.y; }
                v[q] = cmk<C>(ca.x - cb.y, ca.y + cb.x);   // C_a + i C_b
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = cmk<C>((T)0, (T)0);
    }
    line_fft<E, +1, RowLayout>(v, sm + line * LS, 1, n0, a.logn0, t, P, a.tw0);
#pragma unroll
    for (int q = 0; q < E; ++q) sm[line * LS + RowLayout::idx(t + P * q, 1)] = v[q];
    __syncthreads();

    const NodalIO<TIn, TOut, T> &io = a.io;
    const T s = in_scale(io);
    for (int idx = threadIdx.x; idx < 2 * a.G * n0; idx += blockDim.x) {
        const int gq = idx / (2 * n0), rr = (idx / n0) & 1, xx = idx % n0;
        const long long pr = pair0 + gq;
        if (pr >= npairs) continue;
        const long long j = (2 * pr + rr) * n0 + xx;
        const C w12 = sm[(3 * gq + rr) * LS + RowLayout::idx(xx, 1)];
        const T w1 = w12.x, w2 = w12.y;
        const T w3 = reinterpret_cast<const T *>(&sm[(3 * gq + 2) * LS + RowLayout::idx(xx, 1)])[rr];
        TOut *y = io.y;
        if constexpr (OUT == OUT_APPLY) {
            const T m1 = io.m[j], m2 = io.m[N + j], m3 = io.m[2 * N + j];
            T z1, z2, z3, z4;
            nodal_inverse<T, false>(m1, m2, m3, io.lam, w1, w2, w3, s * (T)io.x[3 * N + j] / io.lam,
                                    z1, z2, z3, z4);
            y[j] = (TOut)z1; y[N + j] = (TOut)z2; y[2 * N + j] = (TOut)z3; y[3 * N + j] = (TOut)z4;
        } else if constexpr (OUT == OUT_FUSED) {
            const T m1 = io.m[j], m2 = io.m[N + j], m3 = io.m[2 * N + j];
            const T v1 = s * (T)io.x[j], v2 = s * (T)io.x[N + j], v3 = s * (T)io.x[2 * N + j];
            T z1, z2, z3, z4;
            nodal_inverse<T, false>(m1, m2, m3, io.lam, v1 + w1, v2 + w2, v3 + w3,
                                    -(m1 * v1 + m2 * v2 + m3 * v3) / io.lam, z1, z2, z3, z4);
            y[j] = (TOut)z1; y[N + j] = (TOut)z2; y[2 * N + j] = (TOut)z3; y[3 * N + j] = (TOut)z4;
        } else if constexpr (OUT == OUT_MATVEC) {
            const T m1 = io.m[j], m2 = io.m[N + j], m3 = io.m[2 * N + j];
            const T v1 = s * (T)io.x[j], v2 = s * (T)io.x[N + j], v3 = s * (T)io.x[2 * N + j];
            const T r = s * (T)io.x[3 * N + j];
            const T sg = io.transpose ? (T)-1 : (T)1;
            y[j] = (TOut)(w1 + sg * (m2 * v3 - m3 * v2 + m1 * r));
            y[N + j] = (TOut)(w2 + sg * (m3 * v1 - m1 * v3 + m2 * r));
            y[2 * N + j] = (TOut)(w3 + sg * (m1 * v2 - m2 * v1 + m3 * r));
            y[3 * N + j] = (TOut)(-sg * (m1 * v1 + m2 * v2 + m3 * v3));
        } else if constexpr (OUT == OUT_FIELD) {
            y[j] = (TOut)(w1 + io.fld[0]);
            y[N + j] = (TOut)(w2 + io.fld[1]);
            y[2 * N + j] = (TOut)(w3 + io.fld[2]);
            y[3 * N + j] = (TOut)0;
        } else if constexpr (OUT == OUT_PLAIN) {
            y[j] = (TOut)w1; y[N + j] = (TOut)w2; y[2 * N + j] = (TOut)w3;
        } else {  // OUT_JT: (J^T y)_v = w - m^n x y_v + (k/2) r y_v - m^{n+1} y_r ; (J^T y)_r = mhat . y_v
            const T a1 = s * (T)io.x[j], a2 = s * (T)io.x[N + j], a3 = s * (T)io.x[2 * N + j];
            const T ar = s * (T)io.x[3 * N + j];
            const T n1 = io.mn[j], n2 = io.mn[N + j], n3 = io.mn[2 * N + j];
            const T f1 = io.vf[j], f2 = io.vf[N + j], f3 = io.vf[2 * N + j], fr = io.vf[3 * N + j];
            const T hk = io.half_k;
            const T p1 = n1 + 2 * hk * f1, p2 = n2 + 2 * hk * f2, p3 = n3 + 2 * hk * f3;  // m^{n+1}
            const T h1 = n1 + hk * f1, h2 = n2 + hk * f2, h3 = n3 + hk * f3;              // mhat
            y[j] = (TOut)(w1 - (n2 * a3 - n3 * a2) + hk * fr * a1 - p1 * ar);
            y[N + j] = (TOut)(w2 - (n3 * a1 - n1 * a3) + hk * fr * a2 - p2 * ar);
            y[2 * N + j] = (TOut)(w3 - (n1 * a2 - n2 * a1) + hk * fr * a3 - p3 * ar);
            y[3 * N + j] = (TOut)(h1 * a1 + h2 * a2 + h3 * a3);
        }
    }
}

static inline int row_E(int n0) { return n0 >= 1024 ? 16 : (n0 >= 8 ? 8 : n0); }

struct ColPlan { int E, TW; };
template <typename T> static inline ColPlan col_plan(int nl) {
    int E = nl >= 1024 ? 16 : (nl >= 8 ? 8 : nl);
    int twmax = sizeof(T) == 8 ? 8 : 16;
    int TW = twmax;
    while (TW > 8 && TW * (nl / E) > 512) TW >>= 1;
    return {E, TW};
}

template <typename K> static inline cudaError_t set_smem(K kern, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

}  // namespace llg
