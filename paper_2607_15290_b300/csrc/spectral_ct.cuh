// spectral_ct.cuh -- the pass kernels of spectral_kernels.cuh specialised for a
// compile-time line length 2^LOGN (64..1024): same data flow, prologues and
// epilogues, with the FFT of fft_ct.cuh (constant strides and offsets, two
// exchange buffers, one barrier per stage) and node-parallel loops whose index
// arithmetic is a constant shift/mask.  Lengths outside that range use the
// generic kernels.
#pragma once
#include "spectral_kernels.cuh"
#include "fft_ct.cuh"

namespace llg {
namespace ct {

// elements per thread of a line: 8, or 16 for 1024-point FP32 lines
template <typename T, int LOGN> struct LineE { static constexpr int value = (sizeof(T) == 4 && LOGN >= 10) ? 16 : 8; };

template <int IN> struct InShape {
    static constexpr bool NEED_M = (IN == IN_FUSED || IN == IN_NODAL_T);
    static constexpr int NX = NEED_M ? 4 : 3;
};

// ------------------------------------------------------------------ x-pass forward

// Block: G row pairs = 3G lines of P threads (line 3g: c1 + i c2 of row 2g, 3g+1:
// of row 2g+1, 3g+2: c3 of rows 2g + i 2g+1).  Shared memory: two exchange
// buffers of 3G padded lines.
// where the forward x-pass puts spectral value (row, col), row = 2 pair (+1) a global
// spectral row: by default the spectrum in HBM
template <typename C> struct SpecSink {
    C *base;
    long long S;
    __device__ __forceinline__ void operator()(long long row, int col, C v) const { base[row * S + col] = v; }
};

// prologue of the forward x pass: node-parallel, unit-stride plane loads (KC nodes per
// thread in flight), transformed nodal values staged into buf1 with layout 0
template <typename T, typename TIn, typename TOut, int LOGN, int IN>
__device__ __forceinline__ void row_fwd_stage(const RowArgs<T, TIn, TOut> &a, long long bidx, unsigned char *smraw) {
    using C = cplx<T>;
    using L = RowL<LOGN>;
    constexpr int N = 1 << LOGN, E = LineE<T, LOGN>::value, P = N / E, LS = L::size;
    const int G = a.G;
    // one line of LS per P threads: 3 G lines carry data; a block larger than 3 G P (the
    // ensemble's) transforms its spare lines without storing them
    C *buf0 = reinterpret_cast<C *>(smraw);
    C *buf1 = buf0 + (blockDim.x / P) * LS;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long Nn = a.N, pair0 = bidx * G;
    const NodalIO<TIn, TOut, T> &io = a.io;
    const T s = in_scale(io);
    constexpr int KC = sizeof(T) == 4 ? 6 : 3;
    constexpr bool NEED_M = InShape<IN>::NEED_M;
    constexpr int NX = InShape<IN>::NX;
    const int total = 2 * G * N;
    const long long j0 = pair0 * 2 * N;
    for (int base = tid; base < total; base += KC * nthr) {
        TIn xv[KC][NX];
        T mv[KC][3];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int idx = base + k * nthr;
            const long long j = j0 + idx;
            if (idx < total && j < Nn) {
#pragma unroll
                for (int q = 0; q < NX; ++q) xv[k][q] = io.x[q * Nn + j];
                if constexpr (NEED_M) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) mv[k][q] = cvt<T>(io.m[q * Nn + j]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int idx = base + k * nthr;
            const long long j = j0 + idx;
            if (!(idx < total && j < Nn)) continue;
            const int gp = idx >> (LOGN + 1), rr = (idx >> LOGN) & 1, xx = idx & (N - 1);
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
                io.y[3 * Nn + j] = cvt<TOut>(z4 / io.lam);
            }
            const int e = L::template at<0>(xx);
            buf1[(3 * gp + rr) * LS + e] = cmk<C>(u1, u2);
            reinterpret_cast<T *>(&buf1[(3 * gp + 2) * LS + e])[rr] = u3;
        }
    }
}

// the rest of the forward x pass, from the rows staged in buf1: packed transforms, half
// spectra, every spectral value handed to the sink
template <typename T, typename TIn, typename TOut, int LOGN, class Sink>
__device__ __forceinline__ void row_fwd_transform(const RowArgs<T, TIn, TOut> &a, long long bidx, unsigned char *smraw,
                                                  const Sink &sink) {
    using C = cplx<T>;
    using L = RowL<LOGN>;
    constexpr int N = 1 << LOGN, E = LineE<T, LOGN>::value, P = N / E, LS = L::size;
    constexpr int LOGP = LOGN - (E == 16 ? 4 : 3);
    const int G = a.G;
    C *buf0 = reinterpret_cast<C *>(smraw);
    C *buf1 = buf0 + (blockDim.x / P) * LS;
    const int tid = threadIdx.x;
    const long long npairs = a.rows / 2, pair0 = bidx * G;
    const int line = tid >> LOGP, t = tid & (P - 1);
    const int gp = line / 3, kind = line - 3 * gp;
    const long long pair = pair0 + gp;
    const bool valid = gp < G && pair < npairs;
    C v[E];
    {
        const C *src = buf1 + line * LS;
        const int b = L::template at<0>(t);
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = src[b + L::template off<0>(P * q)];
    }
    fft<LOGN, E, -1, L, 0>(v, buf0 + line * LS, buf1 + line * LS, t, a.tw0);
    C *fb = (FreeBuf<LOGN, E, 0>::value ? buf1 : buf0) + line * LS;
    if (kind < 2) {
        if (valid) {
#pragma unroll
            for (int q = 0; q < E; ++q) sink(2 * pair + kind, t + P * q, v[q]);
        }
    } else {
        const int b = L::template at<0>(t);
#pragma unroll
        for (int q = 0; q < E; ++q) fb[b + L::template off<0>(P * q)] = v[q];
    }
    __syncthreads();
    if (kind == 2 && valid) {
        // U = FFT(c3[ya] + i c3[yb]);  C_a = (U_k + conj U_{-k}) / 2,  C_b = (U_k - conj U_{-k}) / (2i)
#pragma unroll
        for (int q = 0; q <= E / 2; ++q) {
            const int k = t + P * q;
            if (q == E / 2 && t > 0) break;
            const C uk = fb[L::template at<0>(k)];
            const C um = fb[L::template at<0>((N - k) & (N - 1))];
            sink(2 * pair, N + k, cmk<C>((T)0.5 * (uk.x + um.x), (T)0.5 * (uk.y - um.y)));
            sink(2 * pair + 1, N + k, cmk<C>((T)0.5 * (uk.y + um.y), (T)-0.5 * (uk.x - um.x)));
        }
    }
}

template <typename T, typename TIn, typename TOut, int LOGN, int IN, class Sink>
__device__ __forceinline__ void row_fwd_ct_body_to(const RowArgs<T, TIn, TOut> &a, long long bidx, unsigned char *smraw,
                                                   const Sink &sink) {
    row_fwd_stage<T, TIn, TOut, LOGN, IN>(a, bidx, smraw);
    __syncthreads();
    row_fwd_transform<T, TIn, TOut, LOGN>(a, bidx, smraw, sink);
}

template <typename T, typename TIn, typename TOut, int LOGN, int IN>
__device__ __forceinline__ void row_fwd_ct_body(const RowArgs<T, TIn, TOut> &a, long long bidx, unsigned char *smraw) {
    row_fwd_ct_body_to<T, TIn, TOut, LOGN, IN>(a, bidx, smraw, SpecSink<cplx<T>>{a.spec, (long long)a.S});
}

template <typename T, typename TIn, typename TOut, int LOGN, int IN>
__global__ void __launch_bounds__(512) row_fwd_ct(RowArgs<T, TIn, TOut> a) {
    pdl_wait();
    if (a.io.skip && *a.io.skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    row_fwd_ct_body<T, TIn, TOut, LOGN, IN>(a, blockIdx.x, smraw);
}

// ------------------------------------------------------------------ x-pass inverse

// With `in` set, the spectrum of pair p is read from rows 2 (p - in_pair0) (+1) of `in`
// (row stride in_S) instead of the global spectrum.
// STAGE_FWD (OUT_APPLY only): the velocity part of every result is also staged into buf1 the
// way row_fwd_stage stages an unscaled IN_V input, so that row_fwd_transform can transform it
// next without reading it back
template <typename T, typename TIn, typename TOut, int LOGN, int OUT, bool STAGE_FWD = false>
__device__ __forceinline__ void row_inv_ct_body(const RowArgs<T, TIn, TOut> &a, long long bidx, unsigned char *smraw,
                                                const cplx<T> *in = nullptr, long long in_pair0 = 0, int in_S = 0) {
    static_assert(!STAGE_FWD || OUT == OUT_APPLY, "staging follows the preconditioner's epilogue");
    using C = cplx<T>;
    using L = RowL<LOGN>;
    constexpr int N = 1 << LOGN, E = LineE<T, LOGN>::value, P = N / E, LS = L::size, HN = N / 2;
    constexpr int LOGP = LOGN - (E == 16 ? 4 : 3);
    const int G = a.G;
    // as in the forward body: spare lines of a block larger than 3 G P carry no data
    C *buf0 = reinterpret_cast<C *>(smraw);
    C *buf1 = buf0 + (blockDim.x / P) * LS;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long Nn = a.N, npairs = a.rows / 2, pair0 = bidx * G;
    const int line = tid >> LOGP, t = tid & (P - 1);
    const int gp = line / 3, kind = line - 3 * gp;
    const long long pair = pair0 + gp;
    const bool valid = gp < G && pair < npairs;
    const C *const ibase = in ? in : a.spec;
    const long long irow0 = in ? 2 * (pair - in_pair0) : 2 * pair;
    const long long iS = in ? in_S : a.S;
    constexpr bool NEED_M = (OUT == OUT_APPLY || OUT == OUT_FUSED || OUT == OUT_MATVEC || OUT == OUT_JT);
    constexpr int XLO = OUT == OUT_APPLY ? 3 : 0;
    constexpr int XHI = (OUT == OUT_APPLY || OUT == OUT_MATVEC || OUT == OUT_JT) ? 4 : (OUT == OUT_FUSED ? 3 : 0);
    constexpr bool NEED_F = OUT == OUT_JT;
    const NodalIO<TIn, TOut, T> &io = a.io;
    {
        // the epilogue's nodal planes (this block's nodes are contiguous in each plane) move
        // towards L2 while the inverse transform runs: one bulk prefetch per plane
        constexpr int NM = NEED_M ? 3 : 0, NXP = XHI - XLO, NF = NEED_F ? 4 : 0;
        const long long j0 = pair0 * 2 * N;
        if (tid < NM + NXP + NF && j0 < Nn) {
            const long long cnt = (long long)2 * G * N < Nn - j0 ? (long long)2 * G * N : Nn - j0;
            if (tid < NM) {
                const nodal_t<T> *mp = OUT == OUT_JT ? io.mn : io.m;
                l2_prefetch_bulk(mp + tid * Nn + j0, cnt * sizeof(nodal_t<T>));
            } else if (tid < NM + NXP) {
                l2_prefetch_bulk(io.x + (XLO + tid - NM) * Nn + j0, cnt * sizeof(TIn));
            } else {
                l2_prefetch_bulk(io.vf + (tid - NM - NXP) * Nn + j0, cnt * sizeof(nodal_t<T>));
            }
        }
    }
    C v[E];
    if (valid) {
        if (kind < 2) {
            const C *src = ibase + (irow0 + kind) * iS;
#pragma unroll
            for (int q = 0; q < E; ++q) v[q] = src[t + P * q];
        } else {
            // full spectrum of c3[ya] + i c3[yb] from the two half spectra (Hermitian symmetry)
            const C *sa = ibase + irow0 * iS + N;
            const C *sb = sa + iS;
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const int k = t + P * q;
                const bool lower = q < E / 2 || (q == E / 2 && t == 0);   // k <= N/2
                const int kk = lower ? k : N - k;
                C ca = sa[kk], cb = sb[kk];
                if (!lower) { ca.y = -ca.y; cb.y = -cb.y; }
                v[q] = cmk<C>(ca.x - cb.y, ca.y + cb.x);   // C_a + i C_b
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = cmk<C>((T)0, (T)0);
    }
    fft<LOGN, E, +1, L, 0>(v, buf0 + line * LS, buf1 + line * LS, t, a.tw0);
    C *fbase = FreeBuf<LOGN, E, 0>::value ? buf1 : buf0;
    {
        C *fb = fbase + line * LS;
        const int b = L::template at<0>(t);
#pragma unroll
        for (int q = 0; q < E; ++q) fb[b + L::template off<0>(P * q)] = v[q];
    }
    __syncthreads();

    const T s = in_scale(io);
    constexpr int KC = sizeof(T) == 4 ? 6 : 3;
    const int total = 2 * G * N;
    const long long j0 = pair0 * 2 * N;
    for (int base = tid; base < total; base += KC * nthr) {
        T mv[KC][3];
        TIn xv[KC][4];
        T fv[KC][4];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int idx = base + k * nthr;
            const long long j = j0 + idx;
            if (idx < total && j < Nn) {
                if constexpr (NEED_M) {
                    const nodal_t<T> *mp = OUT == OUT_JT ? io.mn : io.m;
#pragma unroll
                    for (int q = 0; q < 3; ++q) mv[k][q] = cvt<T>(mp[q * Nn + j]);
                }
#pragma unroll
                for (int q = XLO; q < XHI; ++q) xv[k][q] = io.x[q * Nn + j];
                if constexpr (NEED_F) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) fv[k][q] = cvt<T>(io.vf[q * Nn + j]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int idx = base + k * nthr;
            const long long j = j0 + idx;
            if (!(idx < total && j < Nn)) continue;
            const int gq = idx >> (LOGN + 1), rr = (idx >> LOGN) & 1, xx = idx & (N - 1);
            const int e = L::template at<0>(xx);
            const C w12 = fbase[(3 * gq + rr) * LS + e];
            const T w1 = w12.x, w2 = w12.y;
            const T w3 = reinterpret_cast<const T *>(&fbase[(3 * gq + 2) * LS + e])[rr];
            TOut *y = io.y;
            if constexpr (OUT == OUT_APPLY) {
                T z1 = w1, z2 = w2, z3 = w3, z4 = s * cvt<T>(xv[k][3]) / io.lam;
                if (!io.plain_nodal)
                    nodal_inverse<T, false>(mv[k][0], mv[k][1], mv[k][2], io.lam, w1, w2, w3, z4, z1, z2, z3, z4);
                y[j] = cvt<TOut>(z1); y[Nn + j] = cvt<TOut>(z2); y[2 * Nn + j] = cvt<TOut>(z3); y[3 * Nn + j] = cvt<TOut>(z4);
                if constexpr (STAGE_FWD) {
                    // this node's slots of the staging layout (read above as fbase when fbase
                    // is buf1: the same thread, read before written)
                    buf1[(3 * gq + rr) * LS + e] = cmk<C>(cvt<T>(cvt<TOut>(z1)), cvt<T>(cvt<TOut>(z2)));
                    reinterpret_cast<T *>(&buf1[(3 * gq + 2) * LS + e])[rr] = cvt<T>(cvt<TOut>(z3));
                }
            } else if constexpr (OUT == OUT_FUSED) {
                const T m1 = mv[k][0], m2 = mv[k][1], m3 = mv[k][2];
                const T v1 = s * cvt<T>(xv[k][0]), v2 = s * cvt<T>(xv[k][1]), v3 = s * cvt<T>(xv[k][2]);
                T z1 = v1 + w1, z2 = v2 + w2, z3 = v3 + w3, z4 = -(m1 * v1 + m2 * v2 + m3 * v3) / io.lam;
                if (!io.plain_nodal) nodal_inverse<T, false>(m1, m2, m3, io.lam, z1, z2, z3, z4, z1, z2, z3, z4);
                y[j] = cvt<TOut>(z1); y[Nn + j] = cvt<TOut>(z2); y[2 * Nn + j] = cvt<TOut>(z3); y[3 * Nn + j] = cvt<TOut>(z4);
            } else if constexpr (OUT == OUT_MATVEC) {
                const T m1 = mv[k][0], m2 = mv[k][1], m3 = mv[k][2];
                const T v1 = s * cvt<T>(xv[k][0]), v2 = s * cvt<T>(xv[k][1]), v3 = s * cvt<T>(xv[k][2]);
                const T r = s * cvt<T>(xv[k][3]);
                // the transpose flips the signs of the skew part (exact negations)
                const bool tr = io.transpose != 0;
                const T k1 = m2 * v3 - m3 * v2 + m1 * r, k2 = m3 * v1 - m1 * v3 + m2 * r;
                const T k3 = m1 * v2 - m2 * v1 + m3 * r, k4 = m1 * v1 + m2 * v2 + m3 * v3;
                y[j] = cvt<TOut>(w1 + (tr ? -k1 : k1));
                y[Nn + j] = cvt<TOut>(w2 + (tr ? -k2 : k2));
                y[2 * Nn + j] = cvt<TOut>(w3 + (tr ? -k3 : k3));
                y[3 * Nn + j] = cvt<TOut>(tr ? k4 : -k4);
            } else if constexpr (OUT == OUT_FIELD) {
                T f1 = w1 + io.fld[0], f2 = w2 + io.fld[1], f3 = w3 + io.fld[2];
                if (io.hf) {
                    f1 += cvt<T>(io.hs * io.hf[j]);
                    f2 += cvt<T>(io.hs * io.hf[Nn + j]);
                    f3 += cvt<T>(io.hs * io.hf[2 * Nn + j]);
                }
                y[j] = cvt<TOut>(f1);
                y[Nn + j] = cvt<TOut>(f2);
                y[2 * Nn + j] = cvt<TOut>(f3);
                y[3 * Nn + j] = cvt<TOut>(0);
            } else if constexpr (OUT == OUT_PLAIN) {
                y[j] = cvt<TOut>(w1); y[Nn + j] = cvt<TOut>(w2); y[2 * Nn + j] = cvt<TOut>(w3);
            } else {  // OUT_JT: (J^T y)_v = w - m^n x y_v + (k/2) r y_v - m^{n+1} y_r ; (J^T y)_r = mhat . y_v
                const T a1 = s * cvt<T>(xv[k][0]), a2 = s * cvt<T>(xv[k][1]), a3 = s * cvt<T>(xv[k][2]);
                const T ar = s * cvt<T>(xv[k][3]);
                const T n1 = mv[k][0], n2 = mv[k][1], n3 = mv[k][2];
                const T f1 = fv[k][0], f2 = fv[k][1], f3 = fv[k][2], fr = fv[k][3];
                const T hk = io.half_k;
                const T p1 = n1 + 2 * hk * f1, p2 = n2 + 2 * hk * f2, p3 = n3 + 2 * hk * f3;  // m^{n+1}
                const T h1 = n1 + hk * f1, h2 = n2 + hk * f2, h3 = n3 + hk * f3;              // mhat
                y[j] = cvt<TOut>(w1 - (n2 * a3 - n3 * a2) + hk * fr * a1 - p1 * ar);
                y[Nn + j] = cvt<TOut>(w2 - (n3 * a1 - n1 * a3) + hk * fr * a2 - p2 * ar);
                y[2 * Nn + j] = cvt<TOut>(w3 - (n1 * a2 - n2 * a1) + hk * fr * a3 - p3 * ar);
                y[3 * Nn + j] = cvt<TOut>(h1 * a1 + h2 * a2 + h3 * a3);
            }
        }
    }
}

// FP32-pair blocks (at most 3 x 128 threads) are held to 85 registers so that three blocks of
// a 128-point row group fit an SM: the pair epilogue is latency-bound at two
template <typename T> struct RowInvBounds {
    static constexpr int threads = is_fpair<T>::value ? 384 : (sizeof(T) == 4 ? 256 : 512);
    static constexpr int blocks = is_fpair<T>::value ? 2 : (sizeof(T) == 4 ? 3 : 1);
};
template <typename T, typename TIn, typename TOut, int LOGN, int OUT>
__global__ void __launch_bounds__(RowInvBounds<T>::threads, RowInvBounds<T>::blocks) row_inv_ct(RowArgs<T, TIn, TOut> a) {
    pdl_wait();
    if (a.io.skip && *a.io.skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    row_inv_ct_body<T, TIn, TOut, LOGN, OUT>(a, blockIdx.x, smraw);
}

// x-pass inverse of the preconditioner (OUT_APPLY, z written) fused with the x-pass forward of
// the matvec that follows it on z (IN_V, unscaled): the forward reads z from shared memory.
// Each block reads its own rows of the spectrum before it writes them, so one buffer serves.
template <typename TIn1, int LOGN>
__global__ void __launch_bounds__(512) row_inv_fwd_ct(RowArgs<float, TIn1, float> a1, RowArgs<float, float, float> a2) {
    pdl_wait();
    if (a1.io.skip && *a1.io.skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    row_inv_ct_body<float, TIn1, float, LOGN, OUT_APPLY, true>(a1, blockIdx.x, smraw);
    __syncthreads();
    row_fwd_transform<float, float, float, LOGN>(a2, blockIdx.x, smraw, SpecSink<float2>{a2.spec, (long long)a2.S});
}

// ------------------------------------------------------------------ axis passes

// the pointwise multiplier of the last axis (Algorithm 1 step 2 when sinv, else the
// symbol itself): scale / (a + b sigma) or scale * (a + b sigma), zero on padding columns
template <typename T> __device__ __forceinline__ T symbol_div(T num, T den);
template <> __device__ __forceinline__ float symbol_div<float>(float num, float den) { return __fdividef(num, den); }
template <> __device__ __forceinline__ double symbol_div<double>(double num, double den) { return num / den; }
template <> __device__ __forceinline__ fpair symbol_div<fpair>(fpair num, fpair den) { return num / den; }

template <typename T, int LOGN, int E, class L, typename C>
__device__ __forceinline__ void apply_symbol(C (&v)[E], const ColArgs<T> &a, int col, int by, int t) {
    constexpr int P = (1 << LOGN) / E;
    const int hn = a.n0 / 2;
    const bool live = col <= a.n0 + hn;
    const T sx = live ? a.tx[col < a.n0 ? col : col - a.n0] : (T)0;
    const T sb = a.tb ? a.tb[by] : (T)0;
    const T base = sx + sb;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const T d = a.sa + a.sb * (base + ldg_ro(&a.tl[t + P * q]));
        const T mult = live ? (a.sinv ? symbol_div<T>(a.sscale, d) : a.sscale * d) : (T)0;
        v[q] = cscale(v[q], mult);
    }
}

// one axis pass over a tile of TW adjacent spectral columns of batch by; thread
// (c, t) owns elements t + P q of column c.  DB: two exchange buffers of N x TW.
template <typename T, int LOGN, int E, int TW, int MODE, bool DB>
__device__ __forceinline__ void col_ct_body(const ColArgs<T> &a, int bx, int by, unsigned char *smraw) {
    using C = cplx<T>;
    using L = ColL<TW>;
    constexpr int N = 1 << LOGN, P = N / E;
    C *buf0 = reinterpret_cast<C *>(smraw);
    C *buf1 = DB ? buf0 + N * TW : buf0;
    const int c = threadIdx.x % TW, t = threadIdx.x / TW;
    const int col = bx * TW + c;
    C *p = a.spec + (long long)by * a.bs + col + (long long)t * a.ls;
    const long long step = (long long)P * a.ls;
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = p[q * step];
    if constexpr ((MODE & 1) != 0) fft<LOGN, E, -1, L, 0, DB>(v, buf0 + c, buf1 + c, t, a.tw);
    if constexpr ((MODE & 4) != 0) apply_symbol<T, LOGN, E, L>(v, a, col, by, t);
    if constexpr ((MODE & 2) != 0) {
        // after a forward transform, start in the buffer its last stage did not read
        // (single buffer: stage 0 of the inverse opens with a barrier)
        constexpr int PAR = (MODE & 1) ? FreeBuf<LOGN, E, 0>::value : 0;
        fft<LOGN, E, +1, L, PAR, DB>(v, buf0 + c, buf1 + c, t, a.tw);
    }
#pragma unroll
    for (int q = 0; q < E; ++q) p[q * step] = v[q];
}

template <typename T, int THREADS> struct ColMinBlocks {
    static constexpr int value = is_fpair<T>::value ? (THREADS <= 128 ? 6 : (THREADS <= 256 ? 3 : 1))
                                                    : ((sizeof(T) == 4 && THREADS <= 512) ? 2 : 1);
};

template <typename T, int LOGN, int E, int TW, int MODE, bool DB>
__global__ void __launch_bounds__(TW *((1 << LOGN) / E), (ColMinBlocks<T, TW * ((1 << LOGN) / E)>::value))
    col_ct(ColArgs<T> a) {
    pdl_wait();
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    col_ct_body<T, LOGN, E, TW, MODE, DB>(a, blockIdx.x, blockIdx.y, smraw);
}

// FP32 axis pass with two adjacent columns per thread (TW columns per tile, TW/2 threads
// per tile row): global loads/stores and every shared-memory exchange are 16-byte words.
template <int LOGN, int TW, int MODE, bool DB>
__global__ void __launch_bounds__((TW / 2) * ((1 << LOGN) / LineE<float, LOGN>::value), 2) col_ct_v2(ColArgs<float> a) {
    pdl_wait();
    if (a.skip && *a.skip) return;
    using C = float2;
    constexpr int N = 1 << LOGN, E = LineE<float, LOGN>::value, P = N / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf0 = reinterpret_cast<C *>(smraw);
    C *buf1 = DB ? buf0 + N * TW : buf0;
    const int c2 = 2 * (threadIdx.x % (TW / 2)), t = threadIdx.x / (TW / 2);
    const int col = blockIdx.x * TW + c2, by = blockIdx.y;
    C *p = a.spec + (long long)by * a.bs + col + (long long)t * a.ls;
    const long long step = (long long)P * a.ls;
    C v[E], w[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const float4 x = *reinterpret_cast<const float4 *>(&p[q * step]);
        v[q] = make_float2(x.x, x.y);
        w[q] = make_float2(x.z, x.w);
    }
    if constexpr ((MODE & 1) != 0) fft2<LOGN, E, -1, TW, 0, DB>(v, w, buf0 + c2, buf1 + c2, t, a.tw);
    if constexpr ((MODE & 4) != 0) {
        apply_symbol<float, LOGN, E, ColL<TW>>(v, a, col, by, t);
        apply_symbol<float, LOGN, E, ColL<TW>>(w, a, col + 1, by, t);
    }
    if constexpr ((MODE & 2) != 0) {
        constexpr int PAR = (MODE & 1) ? FreeBuf<LOGN, E, 0>::value : 0;
        fft2<LOGN, E, +1, TW, PAR, DB>(v, w, buf0 + c2, buf1 + c2, t, a.tw);
    }
#pragma unroll
    for (int q = 0; q < E; ++q) *reinterpret_cast<float4 *>(&p[q * step]) = pack2(v[q], w[q]);
}

// staged FP32 axis pass (see col_staged_kernel): the whole tile of TWL columns is
// copied to shared memory with 16-byte asynchronous copies; CB columns at a time are
// transformed in place in the tile (single exchange buffer: the column itself).
template <int LOGN, int TWL, int CB, int MODE>
__global__ void __launch_bounds__(CB *((1 << LOGN) / 8)) col_staged_ct(ColArgs<float> a, int live) {
    pdl_wait();
    if (a.skip && *a.skip) return;
    using C = float2;
    constexpr int N = 1 << LOGN, E = 8, P = N / E;
    constexpr int SROW = StagedRow<TWL>::value;
    constexpr int CPR = TWL / 2;
    using L = ColL<SROW>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int col0 = blockIdx.x * TWL;
    C *g = a.spec + (long long)blockIdx.y * a.bs + col0;
    constexpr int total = N * CPR;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int e = q / CPR, cc = q % CPR;
        if (col0 + 2 * cc < live) cp_async16(&sm[e * SROW + 2 * cc], g + (long long)e * a.ls + 2 * cc);
    }
    cp_async_wait_all();
    __syncthreads();
    const int c = threadIdx.x % CB, t = threadIdx.x / CB;
#pragma unroll 1
    for (int b = 0; b < TWL / CB; ++b) {
        const int cl = b * CB + c, col = col0 + cl;
        C v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = sm[(t + P * q) * SROW + cl];
        if constexpr ((MODE & 1) != 0) fft<LOGN, E, -1, L, 0, false>(v, sm + cl, sm + cl, t, a.tw);
        if constexpr ((MODE & 4) != 0) apply_symbol<float, LOGN, E, L>(v, a, col, blockIdx.y, t);
        if constexpr ((MODE & 2) != 0) fft<LOGN, E, +1, L, 0, false>(v, sm + cl, sm + cl, t, a.tw);
        __syncthreads();   // every load of this column's last stage precedes the write-back
#pragma unroll
        for (int q = 0; q < E; ++q) sm[(t + P * q) * SROW + cl] = v[q];
    }
    __syncthreads();   // the tile is complete
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int e = q / CPR, cc = q % CPR;
        if (col0 + 2 * cc < live)
            *reinterpret_cast<float4 *>(g + (long long)e * a.ls + 2 * cc) =
                *reinterpret_cast<const float4 *>(&sm[e * SROW + 2 * cc]);
    }
}

}  // namespace ct
}  // namespace llg
