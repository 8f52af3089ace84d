// spectral.cu -- the Fourier round trip at the heart of every operator of the
// library, as three (2D) or five (3D) bandwidth-bound passes over HBM:
//
//   x-pass forward : nodal prologue (what to transform: v, m x v + m r - lambda v,
//                    m, or the transposed nodal solve) -> FFT along x of the packed
//                    pair (c1 + i c2) per row and of c3 for two rows at a time,
//                    split into two half spectra (real-input symmetry)
//   y-pass [3D]    : FFT along y
//   last axis      : FFT, pointwise real even multiplier (the shifted exchange symbol
//                    of Algorithm 1, or its non-inverted form for the matvec), inverse FFT
//   y-pass [3D]    : inverse FFT along y
//   x-pass inverse : inverse FFT along x -> nodal epilogue (closed-form 4x4 inverse of
//                    eq. (inverse S), saddle matvec, ...), written as SoA planes.
//
// Because the multiplier is real and even, the operator maps real fields to real
// fields and is complex-linear, so c1 and c2 share one complex transform; c3 is
// transformed two rows at a time and stored as a half spectrum.
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

// ------------------------------------------------------------------ launch plumbing

static int row_E(int n0) { return n0 >= 1024 ? 16 : (n0 >= 8 ? 8 : n0); }

struct ColPlan { int E, TW; };
template <typename T> static ColPlan col_plan(int nl) {
    int E = nl >= 1024 ? 16 : (nl >= 8 ? 8 : nl);
    int twmax = sizeof(T) == 8 ? 8 : 16;
    int TW = twmax;
    while (TW > 8 && TW * (nl / E) > 512) TW >>= 1;
    return {E, TW};
}

template <typename K> static cudaError_t set_smem(K kern, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

template <typename T> static const cplx<T> *tw_of(llg_ctx *c, int axis);
template <> const double2 *tw_of<double>(llg_ctx *c, int axis) { return c->tw64[axis]; }
template <> const float2 *tw_of<float>(llg_ctx *c, int axis) { return c->tw32[axis]; }
template <typename T> static const T *sig_of(llg_ctx *c, int ex, int axis);
template <> const double *sig_of<double>(llg_ctx *c, int ex, int axis) { return c->sig64[ex][axis]; }
template <> const float *sig_of<float>(llg_ctx *c, int ex, int axis) { return c->sig32[ex][axis]; }
template <typename T> static cplx<T> *spec_of(llg_ctx *c);
template <> double2 *spec_of<double>(llg_ctx *c) { return c->spec64; }
template <> float2 *spec_of<float>(llg_ctx *c) { return c->spec32; }

template <typename T, typename TIn, typename TOut, int E>
static cudaError_t launch_row_fwd_E(llg_ctx *c, int in_mode, RowArgs<T, TIn, TOut> a, int blocks, int threads, size_t sm) {
#define LLG_RF(MODE)                                                                          \
    case MODE: {                                                                              \
        auto k = row_fwd_kernel<T, TIn, TOut, E, MODE>;                                       \
        cudaError_t e = set_smem(k, sm);                                                      \
        if (e != cudaSuccess) return e;                                                       \
        k<<<blocks, threads, sm, c->stream>>>(a);                                             \
        return cudaGetLastError();                                                            \
    }
    switch (in_mode) {
        LLG_RF(IN_V) LLG_RF(IN_FUSED) LLG_RF(IN_M) LLG_RF(IN_NODAL_T)
    }
#undef LLG_RF
    return cudaErrorInvalidValue;
}

template <typename T, typename TIn, typename TOut, int E>
static cudaError_t launch_row_inv_E(llg_ctx *c, int out_mode, RowArgs<T, TIn, TOut> a, int blocks, int threads, size_t sm) {
#define LLG_RI(MODE)                                                                          \
    case MODE: {                                                                              \
        auto k = row_inv_kernel<T, TIn, TOut, E, MODE>;                                       \
        cudaError_t e = set_smem(k, sm);                                                      \
        if (e != cudaSuccess) return e;                                                       \
        k<<<blocks, threads, sm, c->stream>>>(a);                                             \
        return cudaGetLastError();                                                            \
    }
    switch (out_mode) {
        LLG_RI(OUT_APPLY) LLG_RI(OUT_FUSED) LLG_RI(OUT_MATVEC) LLG_RI(OUT_FIELD) LLG_RI(OUT_PLAIN) LLG_RI(OUT_JT)
    }
#undef LLG_RI
    return cudaErrorInvalidValue;
}

template <typename T, int E, int TW>
static cudaError_t launch_col_ETW(llg_ctx *c, int mode, const ColArgs<T> &a, dim3 grid) {
    size_t sm = (size_t)a.nl * TW * sizeof(cplx<T>);
    int threads = TW * (a.nl / E);
#define LLG_CK(MODE)                                                                          \
    case MODE: {                                                                              \
        auto k = col_kernel<T, E, TW, MODE>;                                                  \
        cudaError_t e = set_smem(k, sm);                                                      \
        if (e != cudaSuccess) return e;                                                       \
        k<<<grid, threads, sm, c->stream>>>(a);                                               \
        return cudaGetLastError();                                                            \
    }
    switch (mode) {
        LLG_CK(1) LLG_CK(2) LLG_CK(7)
    }
#undef LLG_CK
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_col(llg_ctx *c, int mode, const ColArgs<T> &a, dim3 grid) {
    ColPlan p = col_plan<T>(a.nl);
#define LLG_CE(EE, TT) if (p.E == EE && p.TW == TT) return launch_col_ETW<T, EE, TT>(c, mode, a, grid);
    LLG_CE(2, 8) LLG_CE(4, 8) LLG_CE(8, 8) LLG_CE(16, 8)
    LLG_CE(2, 16) LLG_CE(4, 16) LLG_CE(8, 16) LLG_CE(16, 16)
#undef LLG_CE
    return cudaErrorInvalidValue;
}

template <typename T, typename TIn, typename TOut>
llg_status spectral_chain(llg_ctx *c, int in_mode, int out_mode, const NodalIO<TIn, TOut, T> &io,
                          const Symbol &sym) {
    const SpecGeom &g = c->geo;
    const int n0 = g.n[0];
    const int E = row_E(n0), P = n0 / E;
    const long long pairs = g.rows / 2;
    int G = 256 / (3 * P);
    if (G < 1) G = 1;
    long long want = pairs / (2LL * c->sm_count);
    if (want < G) G = (int)(want < 1 ? 1 : want);
    const int blocks = (int)((pairs + G - 1) / G);
    const int threads = 3 * G * P;
    const size_t smr = (size_t)3 * G * RowLayout::size(n0) * sizeof(cplx<T>);

    RowArgs<T, TIn, TOut> ra;
    ra.spec = spec_of<T>(c);
    ra.tw0 = tw_of<T>(c, 0);
    ra.n0 = n0; ra.logn0 = g.logn[0]; ra.S = g.S; ra.G = G;
    ra.rows = g.rows; ra.N = g.N; ra.io = io;

    // algorithmic bytes / flops of each pass (live spectrum only; inputs read and outputs written once)
    const double W = sizeof(T), CB = 2.0 * sizeof(T), Ti = sizeof(TIn), To = sizeof(TOut);
    const double Nd = (double)g.N, live = (double)g.rows * (n0 + n0 / 2 + 1);
    auto fftf = [](double lines, int n, int logn) { return lines * 5.0 * n * logn; };
    double in_b = 3 * Nd * Ti;
    if (in_mode == IN_FUSED) in_b = 3 * Nd * W + 4 * Nd * Ti;
    if (in_mode == IN_NODAL_T) in_b = 3 * Nd * W + 4 * Nd * Ti + Nd * To;
    double out_b = 0;
    switch (out_mode) {
        case OUT_APPLY: out_b = Nd * (3 * W + Ti + 4 * To); break;
        case OUT_FUSED: out_b = Nd * (3 * W + 3 * Ti + 4 * To); break;
        case OUT_MATVEC: out_b = Nd * (3 * W + 4 * Ti + 4 * To); break;
        case OUT_FIELD: out_b = Nd * 4 * To; break;
        case OUT_PLAIN: out_b = Nd * 3 * To; break;
        default: out_b = Nd * (4 * Ti + 7 * W + 4 * To); break;
    }
    const double xf = fftf(1.5 * g.rows, n0, g.logn[0]);

    cudaError_t e;
#define LLG_DISPATCH_E(FN, MODE)                                                              \
    switch (E) {                                                                              \
        case 2: e = FN<T, TIn, TOut, 2>(c, MODE, ra, blocks, threads, smr); break;            \
        case 4: e = FN<T, TIn, TOut, 4>(c, MODE, ra, blocks, threads, smr); break;            \
        case 8: e = FN<T, TIn, TOut, 8>(c, MODE, ra, blocks, threads, smr); break;            \
        default: e = FN<T, TIn, TOut, 16>(c, MODE, ra, blocks, threads, smr); break;          \
    }
    prof_begin(c, K_XFWD, in_b + live * CB, xf);
    LLG_DISPATCH_E(launch_row_fwd_E, in_mode)
    prof_end(c);
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass forward");
    c->launches++;

    ColArgs<T> ca;
    ca.spec = spec_of<T>(c);
    ca.n0 = n0; ca.S = g.S;
    ca.tx = sig_of<T>(c, sym.exchange, 0);
    ca.sa = (T)sym.a; ca.sb = (T)sym.b; ca.sscale = (T)sym.scale; ca.sinv = sym.invert;
    auto tiles = [&](int nl) { return g.S / col_plan<T>(nl).TW; };
    if (g.dim == 2) {
        ca.tw = tw_of<T>(c, 1); ca.nl = g.n[1]; ca.logn = g.logn[1];
        ca.ls = g.S; ca.bs = 0; ca.tl = sig_of<T>(c, sym.exchange, 1); ca.tb = nullptr;
        prof_begin(c, K_AXIS, 2 * live * CB, 2 * fftf((double)(n0 + n0 / 2 + 1), g.n[1], g.logn[1]));
        e = launch_col<T>(c, 7, ca, dim3(tiles(g.n[1]), 1));
        prof_end(c);
        if (e != cudaSuccess) return cuda_check(c, e, "y-pass");
        c->launches++;
    } else {
        ColArgs<T> cy = ca;
        cy.tw = tw_of<T>(c, 1); cy.nl = g.n[1]; cy.logn = g.logn[1];
        cy.ls = g.S; cy.bs = (long long)g.n[1] * g.S; cy.tl = nullptr; cy.tb = nullptr;
        const double ylines = (double)(n0 + n0 / 2 + 1) * g.n[2], zlines = (double)(n0 + n0 / 2 + 1) * g.n[1];
        prof_begin(c, K_AXIS, 2 * live * CB, fftf(ylines, g.n[1], g.logn[1]));
        e = launch_col<T>(c, 1, cy, dim3(tiles(g.n[1]), g.n[2]));
        prof_end(c);
        if (e != cudaSuccess) return cuda_check(c, e, "y-pass forward");
        ColArgs<T> cz = ca;
        cz.tw = tw_of<T>(c, 2); cz.nl = g.n[2]; cz.logn = g.logn[2];
        cz.ls = (long long)g.n[1] * g.S; cz.bs = g.S;
        cz.tl = sig_of<T>(c, sym.exchange, 2); cz.tb = sig_of<T>(c, sym.exchange, 1);
        prof_begin(c, K_AXIS, 2 * live * CB, 2 * fftf(zlines, g.n[2], g.logn[2]));
        e = launch_col<T>(c, 7, cz, dim3(tiles(g.n[2]), g.n[1]));
        prof_end(c);
        if (e != cudaSuccess) return cuda_check(c, e, "z-pass");
        prof_begin(c, K_AXIS, 2 * live * CB, fftf(ylines, g.n[1], g.logn[1]));
        e = launch_col<T>(c, 2, cy, dim3(tiles(g.n[1]), g.n[2]));
        prof_end(c);
        if (e != cudaSuccess) return cuda_check(c, e, "y-pass inverse");
        c->launches += 3;
    }
    prof_begin(c, K_XINV, live * CB + out_b, xf);
    LLG_DISPATCH_E(launch_row_inv_E, out_mode)
    prof_end(c);
#undef LLG_DISPATCH_E
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass inverse");
    c->launches++;
    return LLG_OK;
}

template llg_status spectral_chain<double, double, double>(llg_ctx *, int, int, const NodalIO<double, double, double> &, const Symbol &);
template llg_status spectral_chain<float, double, float>(llg_ctx *, int, int, const NodalIO<double, float, float> &, const Symbol &);
template llg_status spectral_chain<float, float, double>(llg_ctx *, int, int, const NodalIO<float, double, float> &, const Symbol &);
template llg_status spectral_chain<float, float, float>(llg_ctx *, int, int, const NodalIO<float, float, float> &, const Symbol &);

}  // namespace llg
