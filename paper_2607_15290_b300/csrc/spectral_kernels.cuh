// spectral_kernels.cuh -- the three pass kernels of a Fourier round trip (x-pass
// forward with the nodal prologue, axis passes with the Fourier multiplier,
// x-pass inverse with the nodal epilogue) and their argument structures.
// Included by every translation unit that launches them.
#pragma once
#include "llg_internal.h"
#include "fft_line.cuh"
#include "convert.cuh"

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
    const int *skip;   // optional device flag: when set, the launch returns at once
};

template <typename TIn, typename TOut, typename T>
__device__ __forceinline__ T in_scale(const NodalIO<TIn, TOut, T> &io) {
    return io.scale ? cvt<T>(*io.scale) : (T)1;
}

// ------------------------------------------------------------------ x-pass forward

// Body of the forward x-pass for row-pair group `bidx`, run by the first `nthr`
// threads of the block (the remaining threads, if any, only take part in the
// barriers and work on spare shared-memory lines).
template <typename T, typename TIn, typename TOut, int E, int IN>
__device__ __forceinline__ void row_fwd_body(const RowArgs<T, TIn, TOut> &a, long long bidx, int nthr, unsigned char *smraw) {
    using C = cplx<T>;
    C *sm = reinterpret_cast<C *>(smraw);
    const int tid = threadIdx.x;
    constexpr int LE = E >= 16 ? 4 : (E >= 8 ? 3 : (E >= 4 ? 2 : 1));
    const int n0 = a.n0, ln0 = a.logn0, P = n0 >> LE, lP = ln0 - LE, LS = RowLayout::size(n0);
    const long long N = a.N, npairs = a.rows / 2, pair0 = bidx * a.G;
    const NodalIO<TIn, TOut, T> &io = a.io;
    const T s = in_scale(io);

    // prologue: node-parallel, coalesced plane loads, staged into shared memory.
    // Loads of KC nodes per thread are issued before any arithmetic so that enough
    // bytes are in flight to cover the memory latency.
    constexpr int KC = sizeof(T) == 4 ? 6 : 3;
    constexpr bool NEED_M = (IN == IN_FUSED || IN == IN_NODAL_T);
    constexpr int NX = (IN == IN_FUSED || IN == IN_NODAL_T) ? 4 : 3;
    const int total = 2 * a.G * n0;
    for (int base = tid; tid < nthr && base < total; base += KC * nthr) {
        TIn xv[KC][NX];
        T mv[KC][3];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int idx = base + k * nthr;
            const int gp = idx >> (ln0 + 1), rr = (idx >> ln0) & 1, xx = idx & (n0 - 1);
            if (idx < total && pair0 + gp < npairs) {
                const long long j = (2 * (pair0 + gp) + rr) * n0 + xx;
#pragma unroll
                for (int q = 0; q < NX; ++q) xv[k][q] = io.x[q * N + j];
                if constexpr (NEED_M) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) mv[k][q] = io.m[q * N + j];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int idx = base + k * nthr;
            const int gp = idx >> (ln0 + 1), rr = (idx >> ln0) & 1, xx = idx & (n0 - 1);
            if (!(idx < total && pair0 + gp < npairs)) continue;
            const long long j = (2 * (pair0 + gp) + rr) * n0 + xx;
            T u1, u2, u3;
            if constexpr (IN == IN_V) {
                u1 = s * cvt<T>(xv[k][0]);
                u2 = s * cvt<T>(xv[k][1]);
                u3 = s * cvt<T>(xv[k][2]);
            } else if constexpr (IN == IN_M) {
                u1 = cvt<T>(xv[k][0]);
                u2 = cvt<T>(xv[k][1]);
                u3 = cvt<T>(xv[k][2]);
            } else if constexpr (IN == IN_FUSED) {
                const T m1 = mv[k][0], m2 = mv[k][1], m3 = mv[k][2];
                const T v1 = s * cvt<T>(xv[k][0]), v2 = s * cvt<T>(xv[k][1]), v3 = s * cvt<T>(xv[k][2]);
                const T r = s * cvt<T>(xv[k][3]);
                u1 = m2 * v3 - m3 * v2 + m1 * r - io.lam * v1;
                u2 = m3 * v1 - m1 * v3 + m2 * r - io.lam * v2;
                u3 = m1 * v2 - m2 * v1 + m3 * r - io.lam * v3;
            } else {  // IN_NODAL_T
                T z4;
                nodal_inverse<T, true>(mv[k][0], mv[k][1], mv[k][2], io.lam, s * cvt<T>(xv[k][0]), s * cvt<T>(xv[k][1]),
                                       s * cvt<T>(xv[k][2]), s * cvt<T>(xv[k][3]), u1, u2, u3, z4);
                io.y[3 * N + j] = cvt<TOut>(z4 / io.lam);
            }
            sm[(3 * gp + rr) * LS + RowLayout::idx(xx, 1)] = cmk<C>(u1, u2);
            reinterpret_cast<T *>(&sm[(3 * gp + 2) * LS + RowLayout::idx(xx, 1)])[rr] = u3;
        }
    }
    __syncthreads();

    const int line = tid >> lP, t = tid & (P - 1);
    const int gp = line / 3, kind = line % 3;
    const long long pair = pair0 + gp;
    const bool valid = gp < a.G && pair < npairs;
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

template <typename T, typename TIn, typename TOut, int E, int IN>
__global__ void __launch_bounds__(512) row_fwd_kernel(RowArgs<T, TIn, TOut> a) {
    pdl_wait();
    if (a.io.skip && *a.io.skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    row_fwd_body<T, TIn, TOut, E, IN>(a, blockIdx.x, blockDim.x, smraw);
}

// ------------------------------------------------------------------ axis passes

// Body of an axis pass for column tile bx of batch by (TW * nl / E threads).
template <typename T, int E, int TW, int MODE>   // MODE bit 1: forward, bit 2: inverse, 4: multiplier
__device__ __forceinline__ void col_body(const ColArgs<T> &a, int bx, int by, unsigned char *smraw) {
    using C = cplx<T>;
    C *sm = reinterpret_cast<C *>(smraw);
    const int c = threadIdx.x % TW, t = threadIdx.x / TW;
    const int P = a.nl / E;
    const int col = bx * TW + c;
    C *base = a.spec + (long long)by * a.bs + col;
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = base[(long long)(t + P * q) * a.ls];
    if (MODE & 1) line_fft<E, -1, ColLayout>(v, sm + c, TW, a.nl, a.logn, t, P, a.tw);
    if (MODE & 4) {
        const int hn = a.n0 / 2;
        const bool live = col <= a.n0 + hn;
        const T sx = live ? a.tx[col < a.n0 ? col : col - a.n0] : (T)0;
        const T sb = a.tb ? a.tb[by] : (T)0;
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

template <typename T, int E, int TW, int MODE>
__global__ void __launch_bounds__(512, (sizeof(T) == 4 && E <= 8) ? 2 : 1) col_kernel(ColArgs<T> a) {
    pdl_wait();
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    col_body<T, E, TW, MODE>(a, blockIdx.x, blockIdx.y, smraw);
}

// ------------------------------------------------------------------ staged FP32 axis pass

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// shared-memory row stride of a staged tile: TWL complex plus padding so that
// consecutive rows start half a bank cycle apart (conflict-free column reads)
template <int TWL> struct StagedRow { static constexpr int value = TWL + ((8 - (TWL & 15)) & 15); };

// FP32 axis pass over a tile of TWL adjacent spectral columns: the whole tile
// (nl rows x TWL complex) is copied into shared memory with asynchronous 16-byte
// copies (all in flight at once, no registers held), transformed CB columns at a
// time, and written back with 16-byte stores.  Only columns < live are touched.
template <int E, int TWL, int CB, int MODE>
__global__ void __launch_bounds__(512) col_staged_kernel(ColArgs<float> a, int live) {
    pdl_wait();
    if (a.skip && *a.skip) return;
    using C = float2;
    constexpr int SROW = StagedRow<TWL>::value;
    constexpr int CPR = TWL / 2;   // 16-byte chunks per tile row
    constexpr int LE = E >= 8 ? 3 : (E >= 4 ? 2 : 1);
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int nl = a.nl, P = nl >> LE;
    const int col0 = blockIdx.x * TWL;
    C *g = a.spec + (long long)blockIdx.y * a.bs + col0;
    const int total = nl * CPR;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int e = q / CPR, cc = q % CPR;
        if (col0 + 2 * cc < live) cp_async16(&sm[e * SROW + 2 * cc], g + (long long)e * a.ls + 2 * cc);
    }
    cp_async_wait_all();
    __syncthreads();
    const int c = threadIdx.x % CB, t = threadIdx.x / CB;
    for (int b = 0; b < TWL / CB; ++b) {
        const int cl = b * CB + c, col = col0 + cl;
        C v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = sm[(t + P * q) * SROW + cl];
        if (MODE & 1) line_fft<E, -1, ColLayout>(v, sm + cl, SROW, nl, a.logn, t, P, a.tw);
        if (MODE & 4) {
            const int hn = a.n0 / 2;
            const bool lv = col <= a.n0 + hn;
            const float sx = lv ? a.tx[col < a.n0 ? col : col - a.n0] : 0.f;
            const float sb = a.tb ? a.tb[blockIdx.y] : 0.f;
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const float sig = sx + a.tl[t + P * q] + sb;
                const float d = a.sa + a.sb * sig;
                const float mult = lv ? (a.sinv ? a.sscale / d : a.sscale * d) : 0.f;
                v[q] = cscale(v[q], mult);
            }
        }
        if (MODE & 2) line_fft<E, +1, ColLayout>(v, sm + cl, SROW, nl, a.logn, t, P, a.tw);
#pragma unroll
        for (int q = 0; q < E; ++q) sm[(t + P * q) * SROW + cl] = v[q];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int e = q / CPR, cc = q % CPR;
        if (col0 + 2 * cc < live)
            *reinterpret_cast<float4 *>(g + (long long)e * a.ls + 2 * cc) =
                *reinterpret_cast<const float4 *>(&sm[e * SROW + 2 * cc]);
    }
}

// staged plan for an FP32 line length: (TWL, CB); E = 8; 512 threads; nl >= 64
struct StagedPlan { int TWL, CB; };
static inline StagedPlan staged_plan(int nl) {
    switch (nl) {
        case 64: return {64, 64};
        case 128: return {64, 32};
        case 256: return {32, 16};
        case 512: return {16, 8};
        default: return {8, 4};
    }
}

// ------------------------------------------------------------------ x-pass inverse

// Body of the inverse x-pass for row-pair group `bidx` (first `nthr` threads active).
template <typename T, typename TIn, typename TOut, int E, int OUT>
__device__ __forceinline__ void row_inv_body(const RowArgs<T, TIn, TOut> &a, long long bidx, int nthr, unsigned char *smraw) {
    using C = cplx<T>;
    C *sm = reinterpret_cast<C *>(smraw);
    const int tid = threadIdx.x;
    constexpr int LE = E >= 16 ? 4 : (E >= 8 ? 3 : (E >= 4 ? 2 : 1));
    const int n0 = a.n0, ln0 = a.logn0, P = n0 >> LE, lP = ln0 - LE, LS = RowLayout::size(n0), hn = n0 / 2;
    const long long N = a.N, npairs = a.rows / 2, pair0 = bidx * a.G;
    const int line = tid >> lP, t = tid & (P - 1);
    const int gp = line / 3, kind = line % 3;
    const long long pair = pair0 + gp;
    const bool valid = gp < a.G && pair < npairs;
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
    // epilogue: node-parallel; the plane loads of KC nodes are issued first
    constexpr int KC = sizeof(T) == 4 ? 6 : 3;
    constexpr bool NEED_M = (OUT == OUT_APPLY || OUT == OUT_FUSED || OUT == OUT_MATVEC || OUT == OUT_JT);
    constexpr int XLO = OUT == OUT_APPLY ? 3 : 0;
    constexpr int XHI = (OUT == OUT_APPLY || OUT == OUT_MATVEC || OUT == OUT_JT) ? 4 : (OUT == OUT_FUSED ? 3 : 0);
    constexpr bool NEED_F = OUT == OUT_JT;
    const int total = 2 * a.G * n0;
    for (int base = tid; tid < nthr && base < total; base += KC * nthr) {
        T mv[KC][3];
        TIn xv[KC][4];
        T fv[KC][4];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int idx = base + k * nthr;
            const int gq = idx >> (ln0 + 1), rr = (idx >> ln0) & 1, xx = idx & (n0 - 1);
            if (idx < total && pair0 + gq < npairs) {
                const long long j = (2 * (pair0 + gq) + rr) * n0 + xx;
                if constexpr (NEED_M) {
                    const T *mp = OUT == OUT_JT ? io.mn : io.m;
#pragma unroll
                    for (int q = 0; q < 3; ++q) mv[k][q] = mp[q * N + j];
                }
#pragma unroll
                for (int q = XLO; q < XHI; ++q) xv[k][q] = io.x[q * N + j];
                if constexpr (NEED_F) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) fv[k][q] = io.vf[q * N + j];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int idx = base + k * nthr;
            const int gq = idx >> (ln0 + 1), rr = (idx >> ln0) & 1, xx = idx & (n0 - 1);
            if (!(idx < total && pair0 + gq < npairs)) continue;
            const long long j = (2 * (pair0 + gq) + rr) * n0 + xx;
            const C w12 = sm[(3 * gq + rr) * LS + RowLayout::idx(xx, 1)];
            const T w1 = w12.x, w2 = w12.y;
            const T w3 = reinterpret_cast<const T *>(&sm[(3 * gq + 2) * LS + RowLayout::idx(xx, 1)])[rr];
            TOut *y = io.y;
            if constexpr (OUT == OUT_APPLY) {
                T z1 = w1, z2 = w2, z3 = w3, z4 = s * cvt<T>(xv[k][3]) / io.lam;
                if (!io.plain_nodal)
                    nodal_inverse<T, false>(mv[k][0], mv[k][1], mv[k][2], io.lam, w1, w2, w3, z4, z1, z2, z3, z4);
                y[j] = cvt<TOut>(z1); y[N + j] = cvt<TOut>(z2); y[2 * N + j] = cvt<TOut>(z3); y[3 * N + j] = cvt<TOut>(z4);
            } else if constexpr (OUT == OUT_FUSED) {
                const T m1 = mv[k][0], m2 = mv[k][1], m3 = mv[k][2];
                const T v1 = s * cvt<T>(xv[k][0]), v2 = s * cvt<T>(xv[k][1]), v3 = s * cvt<T>(xv[k][2]);
                T z1 = v1 + w1, z2 = v2 + w2, z3 = v3 + w3, z4 = -(m1 * v1 + m2 * v2 + m3 * v3) / io.lam;
                if (!io.plain_nodal) nodal_inverse<T, false>(m1, m2, m3, io.lam, z1, z2, z3, z4, z1, z2, z3, z4);
                y[j] = cvt<TOut>(z1); y[N + j] = cvt<TOut>(z2); y[2 * N + j] = cvt<TOut>(z3); y[3 * N + j] = cvt<TOut>(z4);
            } else if constexpr (OUT == OUT_MATVEC) {
                const T m1 = mv[k][0], m2 = mv[k][1], m3 = mv[k][2];
                const T v1 = s * cvt<T>(xv[k][0]), v2 = s * cvt<T>(xv[k][1]), v3 = s * cvt<T>(xv[k][2]);
                const T r = s * cvt<T>(xv[k][3]);
                const T sg = io.transpose ? (T)-1 : (T)1;
                y[j] = cvt<TOut>(w1 + sg * (m2 * v3 - m3 * v2 + m1 * r));
                y[N + j] = cvt<TOut>(w2 + sg * (m3 * v1 - m1 * v3 + m2 * r));
                y[2 * N + j] = cvt<TOut>(w3 + sg * (m1 * v2 - m2 * v1 + m3 * r));
                y[3 * N + j] = cvt<TOut>(-sg * (m1 * v1 + m2 * v2 + m3 * v3));
            } else if constexpr (OUT == OUT_FIELD) {
                T f1 = w1 + io.fld[0], f2 = w2 + io.fld[1], f3 = w3 + io.fld[2];
                if (io.hf) {
                    f1 += (T)(io.hs * io.hf[j]);
                    f2 += (T)(io.hs * io.hf[N + j]);
                    f3 += (T)(io.hs * io.hf[2 * N + j]);
                }
                y[j] = cvt<TOut>(f1);
                y[N + j] = cvt<TOut>(f2);
                y[2 * N + j] = cvt<TOut>(f3);
                y[3 * N + j] = cvt<TOut>(0);
            } else if constexpr (OUT == OUT_PLAIN) {
                y[j] = cvt<TOut>(w1); y[N + j] = cvt<TOut>(w2); y[2 * N + j] = cvt<TOut>(w3);
            } else {  // OUT_JT: (J^T y)_v = w - m^n x y_v + (k/2) r y_v - m^{n+1} y_r ; (J^T y)_r = mhat . y_v
                const T a1 = s * cvt<T>(xv[k][0]), a2 = s * cvt<T>(xv[k][1]), a3 = s * cvt<T>(xv[k][2]);
                const T ar = s * cvt<T>(xv[k][3]);
                const T n1 = mv[k][0], n2 = mv[k][1], n3 = mv[k][2];
                const T f1 = fv[k][0], f2 = fv[k][1], f3 = fv[k][2], fr = fv[k][3];
                const T hk = io.half_k;
                const T p1 = n1 + 2 * hk * f1, p2 = n2 + 2 * hk * f2, p3 = n3 + 2 * hk * f3;  // m^{n+1}
                const T h1 = n1 + hk * f1, h2 = n2 + hk * f2, h3 = n3 + hk * f3;              // mhat
                y[j] = cvt<TOut>(w1 - (n2 * a3 - n3 * a2) + hk * fr * a1 - p1 * ar);
                y[N + j] = cvt<TOut>(w2 - (n3 * a1 - n1 * a3) + hk * fr * a2 - p2 * ar);
                y[2 * N + j] = cvt<TOut>(w3 - (n1 * a2 - n2 * a1) + hk * fr * a3 - p3 * ar);
                y[3 * N + j] = cvt<TOut>(h1 * a1 + h2 * a2 + h3 * a3);
            }
        }
    }
}

template <typename T, typename TIn, typename TOut, int E, int OUT>
__global__ void __launch_bounds__(512) row_inv_kernel(RowArgs<T, TIn, TOut> a) {
    pdl_wait();
    if (a.io.skip && *a.io.skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    row_inv_body<T, TIn, TOut, E, OUT>(a, blockIdx.x, blockDim.x, smraw);
}

// elements per thread of a line: 8 (16 for 1024-point FP32 lines); FP64 stays at 8 so
// that its registers do not spill
template <typename T> static inline int row_E(int n0) {
    return (sizeof(T) == 4 && n0 >= 1024) ? 16 : (n0 >= 8 ? 8 : n0);
}

// column tiles: TW adjacent columns (16 FP32 / 8 FP64 complex = 128 B rows), narrowed
// until the block has at most 512 threads
struct ColPlan { int E, TW; };
template <typename T> static inline ColPlan col_plan(int nl) {
    const int E = (sizeof(T) == 4 && nl >= 1024) ? 16 : (nl >= 8 ? 8 : nl);
    int TW = sizeof(T) == 8 ? 8 : 16;
    while (TW > 4 && TW * (nl / E) > 512) TW >>= 1;
    return {E, TW};
}

// Dynamic shared-memory limit and the maximum shared-memory carveout, set once per
// kernel and device (the attributes apply to the current device only; the carveout keeps
// shared memory from limiting the resident blocks).
template <typename K> static inline cudaError_t set_smem(K kern, size_t bytes) {
    static thread_local const void *done[256];
    static thread_local int done_dev[256];
    static thread_local int ndone = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < ndone; ++i)
        if (done[i] == (const void *)kern && done_dev[i] == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess && ndone < 256) { done[ndone] = (const void *)kern; done_dev[ndone] = dev; ++ndone; }
    (void)bytes;
    return e;
}

}  // namespace llg
