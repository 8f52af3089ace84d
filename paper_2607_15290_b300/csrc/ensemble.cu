// ensemble.cu -- many independent 2D problems advanced by projected-Euler steps in
// ONE persistent cooperative launch.
//
// All problems move through the same sequence of phases in lockstep (right-hand
// side, flexible-GMRES Arnoldi steps with the FP32 FFT--HSS application and inner
// matvec and FP64 Gram--Schmidt, cycle end with the FP64 true residual, the Euler
// update); a grid-wide barrier separates phases.  The barrier is our own (arrival counter
// and generation word); every wait is bounded by a clock budget, after which the block
// raises an error flag and the whole grid returns (no wait can hang the device).  Inside a phase every block takes
// work items (row-pair groups, column tiles, vector chunks, whole problems) of all
// problems in a grid-stride loop, so small and large problems share the machine and
// no per-problem launch is needed.  Each problem carries its own convergence flags:
// a problem that has converged skips all later items, and the loops end when no
// problem needs another Arnoldi step or cycle.
//
// The per-pass code is the same as the context path (spectral_kernels.cuh): the
// ensemble only supplies per-problem arguments.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>
#include <map>
#include <algorithm>
#include "spectral_ct.cuh"
#include "reduce.cuh"
#include "convert.cuh"

using namespace llg;

namespace {

constexpr int ENS_THREADS = 256;
constexpr int ENS_MAXM = 32;          // restart length limit
constexpr int ENS_CHUNK = 8192;       // elements of a 4N vector per chunk item
constexpr int ENS_SMEM = 36864;       // dynamic shared memory (largest pass)

struct EnsClass {
    int n0, n1, ln0, ln1, S, G, TW, nthr_row;
    double L0, L1;
    int exchange;
    double2 *tw64[2];
    float2 *tw32[2];
    double *sig64[2];
    float *sig32[2];
};

struct EnsProb {
    int cls;
    long long N, rows, n4;     // nodes, rows (= n1), 4N
    int nch;                    // chunks of a 4N vector
    long long ch0;              // first global chunk index of this problem
    long long rg0, tile0;       // first row-pair group / column tile of this problem in its class
    double alpha, k, chat, lam, h[3];
    double *m, *x, *b, *V, *W, *T;
    float *Z, *m32;
    double2 *spec64;
    float2 *spec32;
};

// Krylov and step state of one problem (device resident)
struct EnsState {
    int active;       // still solving in this step
    int cyc_done;     // current cycle finished
    int jd, iters, cycles, status;
    int tot_iters, tot_cycles, worst_status, pad;
    double nb, beta, target, rel, drift, worst_rel;
    double H[(ENS_MAXM + 1) * ENS_MAXM];
    double cs[ENS_MAXM], sn[ENS_MAXM], g[ENS_MAXM + 1], y[ENS_MAXM], scale[ENS_MAXM + 1];
    double h1[ENS_MAXM], h2[ENS_MAXM];
};

// grid barrier state (reset before every launch)
struct EnsBarrier {
    unsigned count;   // blocks arrived at the current barrier
    unsigned gen;     // barrier generation
    int err;          // 1: a wait ran out of budget (or the launch was not co-resident)
    int where;        // source line of the barrier that gave up
};

constexpr long long BARRIER_BUDGET = 4000000000LL;   // clock64 cycles (about 2 s)

// Bounded grid-wide barrier.  Thread 0 of each block arrives on the counter; the last
// arrival resets it and advances the generation; the others wait for the generation to
// change, giving up after `budget` cycles.  Returns false (for the whole block) once any
// block has given up.  Memory written before the barrier is visible after it (fences on
// both sides of the arrival).  Block `hold` (diagnostics; -1 in normal runs) does not
// arrive and returns false at once, so the others' waits run out: every block still
// returns, and the host reads the error flag.
__device__ __forceinline__ bool bar_wait(EnsBarrier *b, int where, long long budget, int hold) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x == hold) {
        s_ok = 0;
    } else if (threadIdx.x == 0) {
        volatile unsigned *vgen = &b->gen;
        volatile int *verr = &b->err;
        const unsigned g0 = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&b->count, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g0) {
                if (*verr) { ok = 0; break; }
                if (clock64() - t0 > budget) {
                    atomicExch(&b->err, 1);
                    atomicMax(&b->where, where);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*verr) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct EnsArgs {
    int nprob, ncls, steps, m, max_iters;
    double rtol, eta;
    const EnsClass *cls;
    const EnsProb *prob;
    EnsState *st;
    double *partials;          // [chunk][32]
    int *flags;                // [0]: any problem active, [1], [2]: any cycle still running (parity slots)
    EnsBarrier *bar;
    const long long *rowoff;   // [nprob + 1] prefix sums of x-pass items
    const long long *coloff;   // [nprob + 1] prefix sums of axis-pass items
    unsigned *cnt;             // [nprob] chunk-arrival counters (last-block reductions)
    double *partB, *partC;     // second and third partial-sum buffers ([chunk][32])
    long long nchunks;
    long long row_items[3], col_items[3];   // per class item counts
    int cls_of_group_offset;   // unused
    long long budget;          // barrier wait limit (clock64 cycles)
    int hold_block;            // diagnostics: block that withholds its arrival (-1: none)
};

__device__ __forceinline__ bool bar_sync(const EnsArgs &A, int where) {
    return bar_wait(A.bar, where, A.budget, A.hold_block);
}

// ---------------------------------------------------------------- item decoding

// problem index and local item within a class; problems of a class are contiguous
// in their ordering of prob[], and every problem of a class has the same item count
struct ClassItems {
    int first_prob, count;
};

__device__ __forceinline__ const EnsClass &CL(const EnsArgs &A, int p) { return A.cls[A.prob[p].cls]; }

template <typename T> __device__ __forceinline__ cplx<T> *spec_of(const EnsProb &P);
template <> __device__ __forceinline__ double2 *spec_of<double>(const EnsProb &P) { return P.spec64; }
template <> __device__ __forceinline__ float2 *spec_of<float>(const EnsProb &P) { return P.spec32; }
template <typename T> __device__ __forceinline__ const cplx<T> *tw_of(const EnsClass &C, int ax);
template <> __device__ __forceinline__ const double2 *tw_of<double>(const EnsClass &C, int ax) { return C.tw64[ax]; }
template <> __device__ __forceinline__ const float2 *tw_of<float>(const EnsClass &C, int ax) { return C.tw32[ax]; }
template <typename T> __device__ __forceinline__ const T *sig_of(const EnsClass &C, int ax);
template <> __device__ __forceinline__ const double *sig_of<double>(const EnsClass &C, int ax) { return C.sig64[ax]; }
template <> __device__ __forceinline__ const float *sig_of<float>(const EnsClass &C, int ax) { return C.sig32[ax]; }

// largest p with off[p] <= it (off has nprob + 1 entries, off[0] = 0)
__device__ __forceinline__ int find_prob(const long long *off, int nprob, long long it) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// x-pass items: (problem, row-pair group), over all problems
template <typename F>
__device__ __forceinline__ void for_row_items(const EnsArgs &A, F f) {
    const long long total = A.rowoff[A.nprob];
    for (long long it = blockIdx.x; it < total; it += gridDim.x) {
        const int p = find_prob(A.rowoff, A.nprob, it);
        f(p, it - A.rowoff[p]);
    }
}

// axis-pass items: (problem, column tile)
template <typename F>
__device__ __forceinline__ void for_col_items(const EnsArgs &A, F f) {
    const long long total = A.coloff[A.nprob];
    for (long long it = blockIdx.x; it < total; it += gridDim.x) {
        const int p = find_prob(A.coloff, A.nprob, it);
        f(p, (int)(it - A.coloff[p]));
    }
}

// vector-chunk items: (problem, chunk); problems' chunks are consecutive from ch0
__device__ __forceinline__ int find_chunk_prob(const EnsArgs &A, long long it) {
    int lo = 0, hi = A.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.prob[mid].ch0 <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename F>
__device__ __forceinline__ void for_chunk_items(const EnsArgs &A, F f) {
    for (long long it = blockIdx.x; it < A.nchunks; it += gridDim.x) {
        const int p = find_chunk_prob(A, it);
        f(p, (int)(it - A.prob[p].ch0));
    }
}

// ---------------------------------------------------------------- Fourier passes

template <typename T, typename TIn, typename TOut>
__device__ __forceinline__ RowArgs<T, TIn, TOut> row_args(const EnsProb &P, const EnsClass &C, const TIn *x, TOut *y,
                                                          const T *m, const double *scale) {
    RowArgs<T, TIn, TOut> a;
    a.spec = spec_of<T>(P);
    a.tw0 = tw_of<T>(C, 0);
    a.n0 = C.n0; a.logn0 = C.ln0; a.S = C.S; a.G = C.G;
    a.rows = P.rows; a.N = P.N;
    memset(&a.io, 0, sizeof(a.io));
    a.io.m = m; a.io.x = x; a.io.y = y; a.io.scale = scale; a.io.lam = (T)P.lam;
    return a;
}

template <typename T>
__device__ __forceinline__ ColArgs<T> col_args(const EnsProb &P, const EnsClass &C, double sa, double sb, int inv) {
    ColArgs<T> c{};
    c.spec = spec_of<T>(P);
    c.tw = tw_of<T>(C, 1);
    c.ls = C.S; c.bs = 0;
    c.nl = C.n1; c.logn = C.ln1; c.n0 = C.n0; c.S = C.S;
    c.tx = sig_of<T>(C, 0); c.tl = sig_of<T>(C, 1); c.tb = nullptr;
    c.sa = (T)sa; c.sb = (T)sb; c.sscale = (T)(1.0 / (double)P.N); c.sinv = inv;
    return c;
}

template <typename T>
__device__ __forceinline__ void col_dispatch(const ColArgs<T> &c, int TW, int tile, unsigned char *sm) {
    if (TW == 4) col_body<T, 8, 4, 7>(c, tile, 0, sm);
    else if (TW == 8) col_body<T, 8, 8, 7>(c, tile, 0, sm);
    else col_body<T, 8, 16, 7>(c, tile, 0, sm);
}

// FP32 phases on the compile-time-length bodies (lines of 128, 256, 512 points, 8 points a
// thread).  Every class fills the block exactly: a row item is G = 5, 2, 1 row pairs (with
// one, two, one spare lines of the 256 threads), a column tile is 16, 8, 4 columns wide;
// two exchange buffers of either shape take the 36 KB of dynamic shared memory.
template <typename TIn, typename TOut, int IN>
__device__ __forceinline__ void row_fwd32(const RowArgs<float, TIn, TOut> &a, int ln0, long long grp, unsigned char *sm) {
    if (ln0 == 7) ct::row_fwd_ct_body<float, TIn, TOut, 7, IN>(a, grp, sm);
    else if (ln0 == 8) ct::row_fwd_ct_body<float, TIn, TOut, 8, IN>(a, grp, sm);
    else ct::row_fwd_ct_body<float, TIn, TOut, 9, IN>(a, grp, sm);
}

template <typename TIn, typename TOut, int OUT>
__device__ __forceinline__ void row_inv32(const RowArgs<float, TIn, TOut> &a, int ln0, long long grp, unsigned char *sm) {
    if (ln0 == 7) ct::row_inv_ct_body<float, TIn, TOut, 7, OUT>(a, grp, sm);
    else if (ln0 == 8) ct::row_inv_ct_body<float, TIn, TOut, 8, OUT>(a, grp, sm);
    else ct::row_inv_ct_body<float, TIn, TOut, 9, OUT>(a, grp, sm);
}

__device__ __forceinline__ void col32(const ColArgs<float> &c, int ln1, int tile, unsigned char *sm) {
    if (ln1 == 7) ct::col_ct_body<float, 7, 8, 16, 7, true>(c, tile, 0, sm);
    else if (ln1 == 8) ct::col_ct_body<float, 8, 8, 8, 7, true>(c, tile, 0, sm);
    else ct::col_ct_body<float, 9, 8, 4, 7, true>(c, tile, 0, sm);
}

// ---------------------------------------------------------------- Arnoldi chunks

__device__ __forceinline__ void chunk_range(const EnsProb &P, int ch, long long &lo, long long &hi) {
    lo = (long long)ch * ENS_CHUNK;
    hi = lo + ENS_CHUNK;
    if (hi > P.n4) hi = P.n4;
}

// sum of partials[ch0 .. ch0+nch)[i] for i < cnt, one warp per output
__device__ __forceinline__ void sum_chunks(const EnsArgs &A, const EnsProb &P, int cnt, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < cnt; i += ENS_THREADS / 32) {
        double s = 0.0;
        for (int c = lane; c < P.nch; c += 32) s += A.partials[(P.ch0 + c) * 32 + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = s;
    }
}

__device__ __forceinline__ void store_partials(const EnsArgs &A, const EnsProb &P, int ch, double (&acc)[ENS_MAXM], int nv) {
    block_reduce_store<ENS_MAXM>(acc, nv, A.partials + (P.ch0 + ch) * 32);
}

// After a block has stored its chunk partials in buf: count the arrival; returns true (for
// the whole block) in the block that completes problem p's count, which then owns the
// final reduction; the counter is reset for the next pass.
__device__ __forceinline__ bool last_chunk(const EnsArgs &A, int p) {
    __shared__ int s_last;
    __threadfence();   // every thread's partials are visible device-wide before the count
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned c = atomicAdd(&A.cnt[p], 1u) + 1u;
        s_last = c == (unsigned)A.prob[p].nch;
        if (s_last) {
            A.cnt[p] = 0u;
            __threadfence();
        }
    }
    __syncthreads();
    return s_last != 0;
}

// sum over the chunks of problem p of buf[chunk][i], i < cnt, read through L2
__device__ __forceinline__ void sum_chunks_buf(const EnsProb &P, const double *buf, int cnt, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < cnt; i += ENS_THREADS / 32) {
        double s = 0.0;
        for (int c = lane; c < P.nch; c += 32) s += __ldcg(&buf[(P.ch0 + c) * 32 + i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = s;
    }
}

// ---------------------------------------------------------------- exact-count FP64 loops

// The FP64 loops over the basis are compiled for the exact number of vectors NV: a loop
// compiled for ENS_MAXM with the surplus predicated off still spends FP64 issue slots
// on the skipped multiply-adds.  ENS_NV(nv, CALL) runs CALL with constexpr NVC = nv.
#define ENS_NV(nv, CALL)                                                                              \
    do {                                                                                              \
        switch (nv) {                                                                                 \
            ENS_NV_CASES(CALL)                                                                        \
            default: break;                                                                           \
        }                                                                                             \
    } while (0)
#define ENS_NV_CASES(CALL_)                                                                           \
    ENS_NV_C(1, CALL_) ENS_NV_C(2, CALL_) ENS_NV_C(3, CALL_) ENS_NV_C(4, CALL_) ENS_NV_C(5, CALL_)     \
    ENS_NV_C(6, CALL_) ENS_NV_C(7, CALL_) ENS_NV_C(8, CALL_) ENS_NV_C(9, CALL_) ENS_NV_C(10, CALL_)    \
    ENS_NV_C(11, CALL_) ENS_NV_C(12, CALL_) ENS_NV_C(13, CALL_) ENS_NV_C(14, CALL_) ENS_NV_C(15, CALL_) \
    ENS_NV_C(16, CALL_) ENS_NV_C(17, CALL_) ENS_NV_C(18, CALL_) ENS_NV_C(19, CALL_) ENS_NV_C(20, CALL_) \
    ENS_NV_C(21, CALL_) ENS_NV_C(22, CALL_) ENS_NV_C(23, CALL_) ENS_NV_C(24, CALL_) ENS_NV_C(25, CALL_) \
    ENS_NV_C(26, CALL_) ENS_NV_C(27, CALL_) ENS_NV_C(28, CALL_) ENS_NV_C(29, CALL_) ENS_NV_C(30, CALL_) \
    ENS_NV_C(31, CALL_) ENS_NV_C(32, CALL_)
#define ENS_NV_C(K, CALL_) case K: { constexpr int NVC = K; CALL_; } break;

// per-block sums of acc[0..NV) into part[0..NV) (warp shuffles, then the warps in order;
// red: ENS_THREADS / 32 rows of ENS_MAXM shared doubles)
template <int NV>
__device__ __forceinline__ void ens_reduce_store(double (&acc)[NV], double *part, double (*red)[ENS_MAXM]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NV; i += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < ENS_THREADS / 32; ++w) t += red[w][i];
        part[i] = t;
    }
    __syncthreads();
}

// part[i] = this block's share of V_i . w
template <int NV>
__device__ __forceinline__ void ens_dots(const EnsProb &P, long long lo, long long hi, double *part, double (*red)[ENS_MAXM]) {
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (long long e = lo + threadIdx.x; e < hi; e += ENS_THREADS) {
        const double w = P.W[e];
        double vv[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) vv[i] = __ldcs(&P.V[(long long)i * P.n4 + e]);
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += vv[i] * w;
    }
    ens_reduce_store<NV>(acc, part, red);
}

// w <- w - V cf written to out; part = this block's share of V^T w (DOT) or of |w|^2
template <int NV, bool DOT>
__device__ __forceinline__ void ens_update(const EnsProb &P, long long lo, long long hi, const double *cf, double *out,
                                           double *part, double (*red)[ENS_MAXM]) {
    constexpr int NA = DOT ? NV : 1;
    double acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.0;
    for (long long e = lo + threadIdx.x; e < hi; e += ENS_THREADS) {
        double w = P.W[e];
        double vv[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) vv[i] = P.V[(long long)i * P.n4 + e];
#pragma unroll
        for (int i = 0; i < NV; ++i) w -= cf[i] * vv[i];
        out[e] = w;
        if (DOT) {
#pragma unroll
            for (int i = 0; i < NA; ++i) acc[i] += vv[i] * w;
        } else {
            acc[0] += w * w;
        }
    }
    ens_reduce_store<NA>(acc, part, red);
}

// x += Z y over the NV basis vectors of the cycle
template <int NV>
__device__ __forceinline__ void ens_xupdate(const EnsProb &P, long long lo, long long hi, const double *ys) {
    for (long long e = lo + threadIdx.x; e < hi; e += ENS_THREADS) {
        double v = P.x[e];
#pragma unroll
        for (int i = 0; i < NV; ++i) v += ys[i] * f2d_exact(P.Z[(long long)i * P.n4 + e]);
        P.x[e] = v;
    }
}

// ---------------------------------------------------------------- the persistent kernel

// Four blocks per SM (64 registers a thread).  The FP64 loops over large bases spill at that
// size, but those passes stay bound by FP64 multiply-adds, while the Fourier phases, bound
// by memory latency, gain from twice the resident warps: the 96-problem run measured
// 2.24 s at two blocks per SM, 1.99 s at three, 1.90 s at four and 2.06 s at five.
__global__ void __launch_bounds__(ENS_THREADS, 4) ens_kernel(EnsArgs A) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double s_red[ENS_THREADS / 32][ENS_MAXM];   // block sums of the Gram-Schmidt passes
    EnsState *S = A.st;
    const int tid = threadIdx.x;

    for (int step = 0; step < A.steps; ++step) {
        // ---- right-hand side b = Chat Lap m + (1 + alpha^2) h (FP64 Fourier round trip)
        for_row_items(A, [&](int p, long long grp) {
            const EnsProb &P = A.prob[p];
            const EnsClass &C = A.cls[P.cls];
            auto a = row_args<double, double, double>(P, C, P.m, (double *)nullptr, P.m, nullptr);
            row_fwd_body<double, double, double, 8, IN_M>(a, grp, C.nthr_row, smraw);
            __syncthreads();
        });
        if (!bar_sync(A, __LINE__)) return;
        for_col_items(A, [&](int p, int tile) {
            const EnsProb &P = A.prob[p];
            const EnsClass &C = A.cls[P.cls];
            col_dispatch<double>(col_args<double>(P, C, 0.0, -P.chat, 0), C.TW, tile, smraw);
            __syncthreads();
        });
        if (!bar_sync(A, __LINE__)) return;
        for_row_items(A, [&](int p, long long grp) {
            const EnsProb &P = A.prob[p];
            const EnsClass &C = A.cls[P.cls];
            auto a = row_args<double, double, double>(P, C, P.m, P.b, P.m, nullptr);
            const double s = 1.0 + P.alpha * P.alpha;
            a.io.fld[0] = s * P.h[0]; a.io.fld[1] = s * P.h[1]; a.io.fld[2] = s * P.h[2];
            row_inv_body<double, double, double, 8, OUT_FIELD>(a, grp, C.nthr_row, smraw);
            __syncthreads();
        });
        if (!bar_sync(A, __LINE__)) return;
        // ---- x = 0, V_0 = b, ||b||^2, FP32 copy of m
        for_chunk_items(A, [&](int p, int ch) {
            const EnsProb &P = A.prob[p];
            long long lo, hi;
            chunk_range(P, ch, lo, hi);
            double acc[ENS_MAXM];
            acc[0] = 0.0;
            for (long long e = lo + tid; e < hi; e += ENS_THREADS) {
                const double bv = P.b[e];
                P.x[e] = 0.0;
                P.V[e] = bv;
                acc[0] += bv * bv;
                if (e < 3 * P.N) P.m32[e] = d2f_rn(P.m[e]);
            }
            store_partials(A, P, ch, acc, 1);
            __syncthreads();
        });
        if (blockIdx.x == 0 && tid == 0) { A.flags[0] = 0; A.flags[1] = 0; A.flags[2] = 0; }
        if (!bar_sync(A, __LINE__)) return;
        for (int p = blockIdx.x; p < A.nprob; p += gridDim.x) {
            const EnsProb &P = A.prob[p];
            __shared__ double tot[ENS_MAXM];
            sum_chunks(A, P, 1, tot);
            __syncthreads();
            if (tid == 0) {
                EnsState &s = S[p];
                if (step == 0) { s.tot_iters = 0; s.tot_cycles = 0; s.worst_status = LLG_OK; s.worst_rel = 0.0; }
                const double nb = sqrt(tot[0]);
                s.nb = nb;
                s.iters = 0;
                s.cycles = 0;
                s.rel = nb > 0.0 ? 1.0 : 0.0;
                s.status = LLG_OK;
                s.active = nb > 0.0 ? 1 : 0;
                s.beta = nb;
                s.jd = 0;
                s.cyc_done = s.active ? 0 : 1;
                s.scale[0] = nb > 0.0 ? 1.0 / nb : 0.0;
                for (int i = 0; i <= A.m; ++i) s.g[i] = 0.0;
                s.g[0] = nb;
                s.target = fmax(0.5 * A.rtol, A.eta) * nb;
                if (s.active) atomicOr(&A.flags[0], 1);
            }
            __syncthreads();
        }
        if (!bar_sync(A, __LINE__)) return;

        // ---- flexible GMRES cycles
        for (int cyc = 0; cyc < 1000; ++cyc) {
            if (*(volatile int *)&A.flags[0] == 0) break;
            for (int j = 0; j < A.m; ++j) {
                // flag slot of this step j.  Slots alternate with the parity of j; the slot of
                // step j+1 (the one read at the end of step j-1) is reset only after the first
                // barrier of step j, i.e. once every block has finished reading it.
                int *cyc_flag = &A.flags[1 + (j & 1)];
                // z_j = M^{-1}(s_j V_j) in FP32
                for_row_items(A, [&](int p, long long grp) {
                    const EnsProb &P = A.prob[p];
                    const EnsClass &C = A.cls[P.cls];
                    if (S[p].cyc_done) return;
                    auto a = row_args<float, double, float>(P, C, P.V + (long long)j * P.n4, P.Z + (long long)j * P.n4,
                                                           P.m32, &S[p].scale[j]);
                    row_fwd32<double, float, IN_V>(a, C.ln0, grp, smraw);
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                if (blockIdx.x == 0 && tid == 0) A.flags[1 + ((j + 1) & 1)] = 0;
                for_col_items(A, [&](int p, int tile) {
                    const EnsProb &P = A.prob[p];
                    const EnsClass &C = A.cls[P.cls];
                    if (S[p].cyc_done) return;
                    col32(col_args<float>(P, C, P.alpha + P.lam, P.k * P.chat, 1), C.ln1, tile, smraw);
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                for_row_items(A, [&](int p, long long grp) {
                    const EnsProb &P = A.prob[p];
                    const EnsClass &C = A.cls[P.cls];
                    if (S[p].cyc_done) return;
                    auto a = row_args<float, double, float>(P, C, P.V + (long long)j * P.n4, P.Z + (long long)j * P.n4,
                                                           P.m32, &S[p].scale[j]);
                    row_inv32<double, float, OUT_APPLY>(a, C.ln0, grp, smraw);
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                // w = A z_j in FP32 (stored FP64)
                for_row_items(A, [&](int p, long long grp) {
                    const EnsProb &P = A.prob[p];
                    const EnsClass &C = A.cls[P.cls];
                    if (S[p].cyc_done) return;
                    auto a = row_args<float, float, double>(P, C, P.Z + (long long)j * P.n4, P.W, P.m32, nullptr);
                    row_fwd32<float, double, IN_V>(a, C.ln0, grp, smraw);
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                for_col_items(A, [&](int p, int tile) {
                    const EnsProb &P = A.prob[p];
                    const EnsClass &C = A.cls[P.cls];
                    if (S[p].cyc_done) return;
                    col32(col_args<float>(P, C, P.alpha, P.k * P.chat, 0), C.ln1, tile, smraw);
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                for_row_items(A, [&](int p, long long grp) {
                    const EnsProb &P = A.prob[p];
                    const EnsClass &C = A.cls[P.cls];
                    if (S[p].cyc_done) return;
                    auto a = row_args<float, float, double>(P, C, P.Z + (long long)j * P.n4, P.W, P.m32, nullptr);
                    row_inv32<float, double, OUT_MATVEC>(a, C.ln0, grp, smraw);
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                // CGS2 in FP64, three passes; the block that completes a problem's chunks
                // performs that problem's reduction (no separate reduce phases)
                const int nv = j + 1;
                // pass A: h1 = V^T w
                for_chunk_items(A, [&](int p, int ch) {
                    const EnsProb &P = A.prob[p];
                    if (S[p].cyc_done) return;
                    long long lo, hi;
                    chunk_range(P, ch, lo, hi);
                    ENS_NV(nv, (ens_dots<NVC>(P, lo, hi, A.partials + (P.ch0 + ch) * 32, s_red)));
                    if (last_chunk(A, p)) {
                        __shared__ double tot1[ENS_MAXM];
                        sum_chunks_buf(P, A.partials, nv, tot1);
                        __syncthreads();
                        if (tid < nv) S[p].h1[tid] = tot1[tid] * S[p].scale[tid];
                    }
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                // pass B: w <- w - V h1 ; h2 = V^T w
                for_chunk_items(A, [&](int p, int ch) {
                    const EnsProb &P = A.prob[p];
                    if (S[p].cyc_done) return;
                    long long lo, hi;
                    chunk_range(P, ch, lo, hi);
                    __shared__ double cf[ENS_MAXM];
                    if (tid < nv) cf[tid] = S[p].h1[tid] * S[p].scale[tid];
                    __syncthreads();
                    ENS_NV(nv, (ens_update<NVC, true>(P, lo, hi, cf, P.W, A.partB + (P.ch0 + ch) * 32, s_red)));
                    if (last_chunk(A, p)) {
                        __shared__ double tot2[ENS_MAXM];
                        sum_chunks_buf(P, A.partB, nv, tot2);
                        __syncthreads();
                        if (tid < nv) S[p].h2[tid] = tot2[tid] * S[p].scale[tid];
                    }
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                // pass C: V_{j+1} = w - V h2 (unnormalised), ||V_{j+1}||^2, then the Hessenberg
                // column, Givens rotation and stopping test by the completing block
                for_chunk_items(A, [&](int p, int ch) {
                    const EnsProb &P = A.prob[p];
                    if (S[p].cyc_done) return;
                    long long lo, hi;
                    chunk_range(P, ch, lo, hi);
                    __shared__ double cf2[ENS_MAXM];
                    if (tid < nv) cf2[tid] = S[p].h2[tid] * S[p].scale[tid];
                    __syncthreads();
                    double *vn = P.V + (long long)(j + 1) * P.n4;
                    ENS_NV(nv, (ens_update<NVC, false>(P, lo, hi, cf2, vn, A.partC + (P.ch0 + ch) * 32, s_red)));
                    if (last_chunk(A, p)) {
                        __shared__ double tot3[ENS_MAXM];
                        sum_chunks_buf(P, A.partC, 1, tot3);
                        __syncthreads();
                        if (tid == 0) {
                            EnsState &s = S[p];
                            const int ld = ENS_MAXM + 1;
                            double *H = s.H;
                            for (int i = 0; i <= j; ++i) H[i + ld * j] = s.h1[i] + s.h2[i];
                            const double hn = sqrt(tot3[0]);
                            H[j + 1 + ld * j] = hn;
                            s.scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
                            for (int i = 0; i < j; ++i) {
                                const double a = H[i + ld * j], b = H[i + 1 + ld * j];
                                H[i + ld * j] = s.cs[i] * a + s.sn[i] * b;
                                H[i + 1 + ld * j] = -s.sn[i] * a + s.cs[i] * b;
                            }
                            const double a = H[j + ld * j], b = H[j + 1 + ld * j], rr = hypot(a, b);
                            const double cs = rr > 0.0 ? a / rr : 1.0, sn = rr > 0.0 ? b / rr : 0.0;
                            s.cs[j] = cs;
                            s.sn[j] = sn;
                            H[j + ld * j] = rr;
                            H[j + 1 + ld * j] = 0.0;
                            s.g[j + 1] = -sn * s.g[j];
                            s.g[j] = cs * s.g[j];
                            s.jd = j + 1;
                            s.iters++;
                            const double est = fabs(s.g[j + 1]);
                            if (!isfinite(est)) {
                                s.status = LLG_ERR_BREAKDOWN;
                                s.cyc_done = 1;
                            } else if (est <= s.target || hn == 0.0 || j + 1 == A.m || s.iters >= A.max_iters) {
                                s.cyc_done = 1;
                            }
                            if (!s.cyc_done) atomicOr(cyc_flag, 1);
                        }
                    }
                    __syncthreads();
                });
                if (!bar_sync(A, __LINE__)) return;
                if (*(volatile int *)cyc_flag == 0) break;
            }
            // ---- cycle end: y = H^{-1} g, x += Z y
            for (int p = blockIdx.x; p < A.nprob; p += gridDim.x) {
                if (tid == 0 && S[p].active) {
                    EnsState &s = S[p];
                    const int ld = ENS_MAXM + 1, jd = s.jd;
                    for (int i = jd - 1; i >= 0; --i) {
                        double v = s.g[i];
                        for (int q = i + 1; q < jd; ++q) v -= s.H[i + ld * q] * s.y[q];
                        s.y[i] = v / s.H[i + ld * i];
                    }
                    s.cycles++;
                }
            }
            if (!bar_sync(A, __LINE__)) return;
            for_chunk_items(A, [&](int p, int ch) {
                const EnsProb &P = A.prob[p];
                if (!S[p].active) return;
                long long lo, hi;
                chunk_range(P, ch, lo, hi);
                const int jd = S[p].jd;
                __shared__ double ys[ENS_MAXM];
                if (tid < jd) ys[tid] = S[p].y[tid];
                __syncthreads();
                ENS_NV(jd, (ens_xupdate<NVC>(P, lo, hi, ys)));
                __syncthreads();
            });
            if (!bar_sync(A, __LINE__)) return;
            // ---- FP64 true residual r = b - A x
            for_row_items(A, [&](int p, long long grp) {
                const EnsProb &P = A.prob[p];
                const EnsClass &C = A.cls[P.cls];
                if (!S[p].active) return;
                auto a = row_args<double, double, double>(P, C, P.x, P.T, P.m, nullptr);
                row_fwd_body<double, double, double, 8, IN_V>(a, grp, C.nthr_row, smraw);
                __syncthreads();
            });
            if (!bar_sync(A, __LINE__)) return;
            for_col_items(A, [&](int p, int tile) {
                const EnsProb &P = A.prob[p];
                const EnsClass &C = A.cls[P.cls];
                if (!S[p].active) return;
                col_dispatch<double>(col_args<double>(P, C, P.alpha, P.k * P.chat, 0), C.TW, tile, smraw);
                __syncthreads();
            });
            if (!bar_sync(A, __LINE__)) return;
            for_row_items(A, [&](int p, long long grp) {
                const EnsProb &P = A.prob[p];
                const EnsClass &C = A.cls[P.cls];
                if (!S[p].active) return;
                auto a = row_args<double, double, double>(P, C, P.x, P.T, P.m, nullptr);
                row_inv_body<double, double, double, 8, OUT_MATVEC>(a, grp, C.nthr_row, smraw);
                __syncthreads();
            });
            if (!bar_sync(A, __LINE__)) return;
            for_chunk_items(A, [&](int p, int ch) {
                const EnsProb &P = A.prob[p];
                if (!S[p].active) return;
                long long lo, hi;
                chunk_range(P, ch, lo, hi);
                double acc[ENS_MAXM];
                acc[0] = 0.0;
                for (long long e = lo + tid; e < hi; e += ENS_THREADS) {
                    const double r = P.b[e] - P.T[e];
                    P.V[e] = r;
                    acc[0] += r * r;
                }
                store_partials(A, P, ch, acc, 1);
                __syncthreads();
            });
            if (blockIdx.x == 0 && tid == 0) { A.flags[0] = 0; A.flags[1] = 0; A.flags[2] = 0; }
            if (!bar_sync(A, __LINE__)) return;
            for (int p = blockIdx.x; p < A.nprob; p += gridDim.x) {
                if (!S[p].active) continue;
                __shared__ double tot4[ENS_MAXM];
                sum_chunks(A, A.prob[p], 1, tot4);
                __syncthreads();
                if (tid == 0) {
                    EnsState &s = S[p];
                    const double rn = sqrt(tot4[0]);
                    s.rel = rn / s.nb;
                    if (!isfinite(s.rel) || s.status == LLG_ERR_BREAKDOWN) {
                        s.status = LLG_ERR_BREAKDOWN;
                        s.active = 0;
                    } else if (s.rel <= A.rtol) {
                        s.active = 0;
                    } else if (s.iters >= A.max_iters || s.jd == 0) {
                        s.status = LLG_ERR_NOT_CONVERGED;
                        s.active = 0;
                    } else {
                        s.beta = rn;
                        s.scale[0] = 1.0 / rn;
                        for (int i = 0; i <= A.m; ++i) s.g[i] = 0.0;
                        s.g[0] = rn;
                        s.target = fmax(0.5 * A.rtol / s.rel, A.eta) * rn;
                        s.jd = 0;
                    }
                    s.cyc_done = s.active ? 0 : 1;
                    if (s.active) {
                        atomicOr(&A.flags[0], 1);
                    } else {
                        s.tot_iters += s.iters;
                        s.tot_cycles += s.cycles;
                        s.worst_rel = fmax(s.worst_rel, s.rel);
                        if (s.status != LLG_OK) s.worst_status = s.status;
                    }
                }
                __syncthreads();
            }
            if (!bar_sync(A, __LINE__)) return;
        }
        // ---- projected Euler update m <- (m + k v) / |m + k v|
        for (long long it = blockIdx.x; it < A.nchunks; it += gridDim.x) {
            int p = 0;
            while (p + 1 < A.nprob && A.prob[p + 1].ch0 <= it) ++p;
            const EnsProb &P = A.prob[p];
            const long long lo = (it - P.ch0) * ENS_CHUNK / 4, hi = min(lo + ENS_CHUNK / 4, P.N);
            for (long long q = lo + tid; q < hi; q += ENS_THREADS) {
                const double a = P.m[q] + P.k * P.x[q], b = P.m[P.N + q] + P.k * P.x[P.N + q];
                const double c = P.m[2 * P.N + q] + P.k * P.x[2 * P.N + q];
                const double s = sqrt(a * a + b * b + c * c);
                P.m[q] = a / s;
                P.m[P.N + q] = b / s;
                P.m[2 * P.N + q] = c / s;
            }
        }
        if (!bar_sync(A, __LINE__)) return;
    }
}

bool ens_size_ok(int n) { return n == 128 || n == 256 || n == 512; }
int ilog2i(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

}  // namespace

struct llg_ensemble {
    cudaStream_t stream = nullptr;
    int nprob = 0, restart = 30, max_iters = 300, blocks = 0;
    double rtol = 1e-10;
    std::vector<EnsClass> cls;
    std::vector<EnsProb> prob;
    std::vector<void *> allocs;
    EnsClass *dcls = nullptr;
    EnsProb *dprob = nullptr;
    EnsState *dst = nullptr;
    double *partials = nullptr;
    int *flags = nullptr;
    EnsBarrier *bar = nullptr;
    long long *rowoff = nullptr, *coloff = nullptr;
    unsigned *cnt = nullptr;
    double *partB = nullptr, *partC = nullptr;
    long long nchunks = 0;
    EnsState *hst = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_steps = -1;
    std::vector<int> caller;   // descriptor order -> caller's problem index
    std::string err;
    long long budget = BARRIER_BUDGET;   // barrier wait limit (llg_ensemble_set_barrier_test)
    int hold_block = -1;
};

namespace {
template <typename P> cudaError_t ens_alloc(llg_ensemble *e, P **p, size_t bytes) {
    cudaError_t r = cudaMalloc((void **)p, bytes);
    if (r == cudaSuccess) e->allocs.push_back((void *)*p);
    return r;
}
}  // namespace

extern "C" {

llg_status llg_ensemble_destroy(llg_ensemble *e) {
    if (!e) return LLG_ERR_INVALID_ARG;
    if (e->stream) cudaStreamSynchronize(e->stream);
    else cudaDeviceSynchronize();
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    for (void *p : e->allocs) cudaFree(p);
    if (e->hst) cudaFreeHost(e->hst);
    cudaGetLastError();
    delete e;
    return LLG_OK;
}

const char *llg_ensemble_last_error(const llg_ensemble *e) { return e ? e->err.c_str() : "null ensemble"; }

llg_status llg_ensemble_create(const llg_problem *probs, int count, const llg_opts *opts, void *stream,
                               llg_ensemble **out) {
    if (!out || !probs || count < 1 || !opts) return LLG_ERR_INVALID_ARG;
    *out = nullptr;
    if (opts->restart < 1 || opts->restart > ENS_MAXM - 1 || opts->max_iters < 1 || !(opts->rtol > 0))
        return LLG_ERR_INVALID_ARG;
    llg_ensemble *e = new llg_ensemble();
    e->stream = static_cast<cudaStream_t>(stream);
    e->restart = opts->restart;
    e->max_iters = opts->max_iters;
    e->rtol = opts->rtol;
    auto fail = [&](llg_status s, const char *msg) {
        (void)msg;
        cudaGetLastError();
        llg_ensemble_destroy(e);
        return s;
    };
    // classes: problems sharing grid, cell and exchange discretisation
    std::map<std::vector<double>, int> key_to_cls;
    std::vector<int> cls_of(count);
    for (int i = 0; i < count; ++i) {
        const llg_problem &q = probs[i];
        if (!ens_size_ok(q.n[0]) || !ens_size_ok(q.n[1])) return fail(LLG_ERR_UNSUPPORTED_SIZE, "size");
        if (!q.m || !q.x) return fail(LLG_ERR_INVALID_ARG, "null array");
        const llg_params &p = q.prm;
        if (!(p.alpha > 0) || !(p.c_ex > 0) || !(p.lambda > 0) || p.k < 0 || !(q.L[0] > 0) || !(q.L[1] > 0))
            return fail(LLG_ERR_INVALID_ARG, "params");
        if (p.exchange != LLG_EX_SPECTRAL && p.exchange != LLG_EX_FD2) return fail(LLG_ERR_INVALID_ARG, "exchange");
        if (p.h_field || p.demag || p.k_an != 0.0)
            return fail(LLG_ERR_INVALID_ARG, "ensembles take exchange and uniform applied fields only");
        std::vector<double> key = {(double)q.n[0], (double)q.n[1], q.L[0], q.L[1], (double)p.exchange};
        auto it = key_to_cls.find(key);
        if (it == key_to_cls.end()) {
            const int c = (int)e->cls.size();
            key_to_cls[key] = c;
            EnsClass C{};
            C.n0 = q.n[0]; C.n1 = q.n[1]; C.ln0 = ilog2i(C.n0); C.ln1 = ilog2i(C.n1);
            C.S = ((C.n0 + C.n0 / 2 + 1) + 15) / 16 * 16;
            const int P0 = C.n0 / 8, P1 = C.n1 / 8;
            C.G = ENS_THREADS / (3 * P0);
            C.nthr_row = 3 * C.G * P0;
            C.TW = ENS_THREADS / P1;
            C.L0 = q.L[0]; C.L1 = q.L[1];
            C.exchange = p.exchange;
            for (int ax = 0; ax < 2; ++ax) {
                const int n = ax == 0 ? C.n0 : C.n1;
                const double L = ax == 0 ? C.L0 : C.L1;
                std::vector<double2> t64(n);
                std::vector<float2> t32(n);
                std::vector<double> s64(n);
                std::vector<float> s32(n);
                const long double tp = 6.283185307179586476925286766559L;
                for (int j = 0; j < n; ++j) {
                    const long double ang = tp * j / n;
                    t64[j] = make_double2((double)cosl(ang), (double)-sinl(ang));
                    t32[j] = make_float2((float)cosl(ang), (float)-sinl(ang));
                    const int kw = j < n / 2 ? j : j - n;
                    long double v;
                    if (p.exchange == LLG_EX_FD2) {
                        const long double h = (long double)L / n, sn = sinl(3.14159265358979323846264338327950L * kw / n);
                        v = 4.0L / (h * h) * sn * sn;
                    } else {
                        const long double xi = tp * kw / (long double)L;
                        v = xi * xi;
                    }
                    s64[j] = (double)v;
                    s32[j] = (float)v;
                }
                if (ens_alloc(e, &C.tw64[ax], sizeof(double2) * n) != cudaSuccess ||
                    ens_alloc(e, &C.tw32[ax], sizeof(float2) * n) != cudaSuccess ||
                    ens_alloc(e, &C.sig64[ax], sizeof(double) * n) != cudaSuccess ||
                    ens_alloc(e, &C.sig32[ax], sizeof(float) * n) != cudaSuccess)
                    return fail(LLG_ERR_OOM, "tables");
                cudaMemcpy(C.tw64[ax], t64.data(), sizeof(double2) * n, cudaMemcpyHostToDevice);
                cudaMemcpy(C.tw32[ax], t32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
                cudaMemcpy(C.sig64[ax], s64.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
                cudaMemcpy(C.sig32[ax], s32.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
            }
            e->cls.push_back(C);
            cls_of[i] = c;
        } else {
            cls_of[i] = it->second;
        }
    }
    // problems ordered by class (chunk indices follow this order)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cls_of[a] < cls_of[b]; });
    e->nprob = count;
    long long ch = 0;
    const int m = e->restart;
    for (int oi = 0; oi < count; ++oi) {
        const int i = order[oi];
        const llg_problem &q = probs[i];
        const EnsClass &C = e->cls[cls_of[i]];
        EnsProb P{};
        P.cls = cls_of[i];
        P.N = (long long)C.n0 * C.n1;
        P.rows = C.n1;
        P.n4 = 4 * P.N;
        P.nch = (int)((P.n4 + ENS_CHUNK - 1) / ENS_CHUNK);
        P.ch0 = ch;
        ch += P.nch;
        P.alpha = q.prm.alpha;
        P.k = q.prm.k;
        P.chat = (1.0 + q.prm.alpha * q.prm.alpha) * q.prm.c_ex;
        P.lam = q.prm.lambda;
        for (int c = 0; c < 3; ++c) P.h[c] = q.prm.h_ext[c];
        P.m = q.m;
        P.x = q.x;
        const size_t spec_el = (size_t)C.n1 * C.S;
        if (ens_alloc(e, &P.b, sizeof(double) * P.n4) != cudaSuccess ||
            ens_alloc(e, &P.V, sizeof(double) * P.n4 * (m + 1)) != cudaSuccess ||
            ens_alloc(e, &P.W, sizeof(double) * P.n4) != cudaSuccess ||
            ens_alloc(e, &P.T, sizeof(double) * P.n4) != cudaSuccess ||
            ens_alloc(e, &P.Z, sizeof(float) * P.n4 * m) != cudaSuccess ||
            ens_alloc(e, &P.m32, sizeof(float) * 3 * P.N) != cudaSuccess ||
            ens_alloc(e, &P.spec64, sizeof(double2) * spec_el) != cudaSuccess ||
            ens_alloc(e, &P.spec32, sizeof(float2) * spec_el) != cudaSuccess)
            return fail(LLG_ERR_OOM, "problem buffers");
        cudaMemset(P.spec64, 0, sizeof(double2) * spec_el);
        cudaMemset(P.spec32, 0, sizeof(float2) * spec_el);
        e->prob.push_back(P);
    }
    e->nchunks = ch;
    if (ens_alloc(e, &e->dcls, sizeof(EnsClass) * e->cls.size()) != cudaSuccess ||
        ens_alloc(e, &e->dprob, sizeof(EnsProb) * count) != cudaSuccess ||
        ens_alloc(e, &e->dst, sizeof(EnsState) * count) != cudaSuccess ||
        ens_alloc(e, &e->partials, sizeof(double) * 32 * (size_t)ch) != cudaSuccess ||
        ens_alloc(e, &e->flags, sizeof(int) * 4) != cudaSuccess ||
        ens_alloc(e, &e->bar, sizeof(EnsBarrier)) != cudaSuccess ||
        ens_alloc(e, &e->rowoff, sizeof(long long) * (count + 1)) != cudaSuccess ||
        ens_alloc(e, &e->coloff, sizeof(long long) * (count + 1)) != cudaSuccess ||
        ens_alloc(e, &e->cnt, sizeof(unsigned) * count) != cudaSuccess ||
        ens_alloc(e, &e->partB, sizeof(double) * 32 * (size_t)ch) != cudaSuccess ||
        ens_alloc(e, &e->partC, sizeof(double) * 32 * (size_t)ch) != cudaSuccess)
        return fail(LLG_ERR_OOM, "descriptors");
    if (cudaMallocHost(&e->hst, sizeof(EnsState) * count) != cudaSuccess) return fail(LLG_ERR_OOM, "host state");
    cudaMemcpy(e->dcls, e->cls.data(), sizeof(EnsClass) * e->cls.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(e->dprob, e->prob.data(), sizeof(EnsProb) * count, cudaMemcpyHostToDevice);
    cudaMemset(e->dst, 0, sizeof(EnsState) * count);
    cudaMemset(e->cnt, 0, sizeof(unsigned) * count);
    {
        std::vector<long long> ro(count + 1, 0), co(count + 1, 0);
        for (int q = 0; q < count; ++q) {
            const EnsClass &C = e->cls[e->prob[q].cls];
            ro[q + 1] = ro[q] + (e->prob[q].rows / 2 + C.G - 1) / C.G;
            co[q + 1] = co[q] + C.S / C.TW;
        }
        cudaMemcpy(e->rowoff, ro.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice);
        cudaMemcpy(e->coloff, co.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice);
    }
    // co-resident blocks for the cooperative launch
    cudaError_t r = cudaFuncSetAttribute(ens_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ENS_SMEM);
    int per_sm = 0, dev = 0, sms = 0;
    if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ens_kernel, ENS_THREADS, ENS_SMEM);
    if (r == cudaSuccess) r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (r != cudaSuccess || per_sm < 1) return fail(LLG_ERR_CUDA, "occupancy");
    e->blocks = per_sm * sms;
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(LLG_ERR_CUDA, "create");
    e->caller = order;
    *out = e;
    return LLG_OK;
}

llg_status llg_ensemble_set_blocks(llg_ensemble *e, int blocks) {
    if (!e || blocks < 1) return LLG_ERR_INVALID_ARG;
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ens_kernel, ENS_THREADS, ENS_SMEM);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks > per_sm * sms) return LLG_ERR_INVALID_ARG;   // would not be co-resident
    e->blocks = blocks;
    if (e->gexec) { cudaGraphExecDestroy(e->gexec); e->gexec = nullptr; }
    e->graph_steps = -1;
    return LLG_OK;
}

llg_status llg_ensemble_set_barrier_test(llg_ensemble *e, long long budget_cycles, int hold_block) {
    if (!e || budget_cycles < 0 || hold_block < -1) return LLG_ERR_INVALID_ARG;
    e->budget = budget_cycles > 0 ? budget_cycles : BARRIER_BUDGET;
    e->hold_block = hold_block;
    if (e->gexec) { cudaGraphExecDestroy(e->gexec); e->gexec = nullptr; }   // the arguments changed
    e->graph_steps = -1;
    return LLG_OK;
}

int llg_ensemble_max_blocks(const llg_ensemble *e) {
    if (!e) return 0;
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ens_kernel, ENS_THREADS, ENS_SMEM);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

llg_status llg_ensemble_run(llg_ensemble *e, int steps, llg_info *infos, int *used_graph);

llg_status llg_ensemble_autotune(llg_ensemble *e, int *blocks_out) {
    if (!e) return LLG_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int maxb = llg_ensemble_max_blocks(e);
    // save every problem's m, try each candidate on the same start, restore
    std::vector<double *> saved;
    for (const EnsProb &P : e->prob) {
        double *s = nullptr;
        if (cudaMalloc(&s, sizeof(double) * 3 * P.N) != cudaSuccess) {
            for (double *q : saved) cudaFree(q);
            cudaGetLastError();
            return LLG_ERR_OOM;
        }
        cudaMemcpyAsync(s, P.m, sizeof(double) * 3 * P.N, cudaMemcpyDeviceToDevice, e->stream);
        saved.push_back(s);
    }
    auto restore = [&]() {
        for (size_t i = 0; i < saved.size(); ++i)
            cudaMemcpyAsync(e->prob[i].m, saved[i], sizeof(double) * 3 * e->prob[i].N, cudaMemcpyDeviceToDevice, e->stream);
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = e->blocks;
    float best_ms = 1e30f;
    llg_status st = LLG_OK;
    for (int b = sms; b <= maxb; b += sms) {
        if (llg_ensemble_set_blocks(e, b) != LLG_OK) continue;
        restore();
        cudaEventRecord(e0, e->stream);
        st = llg_ensemble_run(e, 1, nullptr, nullptr);
        cudaEventRecord(e1, e->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st != LLG_OK && st != LLG_ERR_NOT_CONVERGED) break;
        if (ms < best_ms) { best_ms = ms; best = b; }
    }
    restore();
    cudaStreamSynchronize(e->stream);
    for (double *q : saved) cudaFree(q);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    llg_ensemble_set_blocks(e, best);
    if (blocks_out) *blocks_out = best;
    return (st == LLG_OK || st == LLG_ERR_NOT_CONVERGED) ? LLG_OK : st;
}

llg_status llg_ensemble_run(llg_ensemble *e, int steps, llg_info *infos, int *used_graph) {
    if (!e || steps < 1) return LLG_ERR_INVALID_ARG;
    EnsArgs A;
    std::memset(&A, 0, sizeof(A));
    A.nprob = e->nprob;
    A.ncls = (int)e->cls.size();
    A.steps = steps;
    A.m = e->restart;
    A.max_iters = e->max_iters;
    A.rtol = e->rtol;
    A.eta = 1e-5;
    A.cls = e->dcls;
    A.prob = e->dprob;
    A.st = e->dst;
    A.partials = e->partials;
    A.flags = e->flags;
    A.bar = e->bar;
    A.rowoff = e->rowoff;
    A.coloff = e->coloff;
    A.cnt = e->cnt;
    A.partB = e->partB;
    A.partC = e->partC;
    A.nchunks = e->nchunks;
    A.budget = e->budget;
    A.hold_block = e->hold_block;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(e->blocks);
    cfg.blockDim = dim3(ENS_THREADS);
    cfg.dynamicSmemBytes = ENS_SMEM;
    cfg.stream = e->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int graph = 0;
    if (e->graph_steps != steps) {
        if (e->gexec) { cudaGraphExecDestroy(e->gexec); e->gexec = nullptr; }
        e->graph_steps = -1;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaMemsetAsync(e->bar, 0, sizeof(EnsBarrier), e->stream);
            cudaError_t r1 = cudaLaunchKernelEx(&cfg, ens_kernel, A);
            cudaError_t r2 = cudaStreamEndCapture(e->stream, &g);
            if (r1 == cudaSuccess && r2 == cudaSuccess && g &&
                cudaGraphInstantiate(&e->gexec, g, 0) == cudaSuccess)
                e->graph_steps = steps;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
    }
    cudaError_t r;
    if (e->gexec) {
        r = cudaGraphLaunch(e->gexec, e->stream);
        graph = 1;
    } else {
        r = cudaMemsetAsync(e->bar, 0, sizeof(EnsBarrier), e->stream);
        if (r == cudaSuccess) r = cudaLaunchKernelEx(&cfg, ens_kernel, A);
    }
    EnsBarrier hb{};
    if (r == cudaSuccess) r = cudaMemcpyAsync(&hb, e->bar, sizeof(EnsBarrier), cudaMemcpyDeviceToHost, e->stream);
    if (r == cudaSuccess) r = cudaMemcpyAsync(e->hst, e->dst, sizeof(EnsState) * e->nprob, cudaMemcpyDeviceToHost, e->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
    if (r != cudaSuccess) {
        e->err = std::string("ensemble launch: ") + cudaGetErrorString(r);
        cudaGetLastError();
        return LLG_ERR_CUDA;
    }
    if (used_graph) *used_graph = graph;
    if (hb.err) {
        e->err = "ensemble grid barrier gave up (blocks not co-resident?) at source line " + std::to_string(hb.where);
        // a wait that gave up inside a phase can leave a last-block arrival counter raised
        if (cudaMemsetAsync(e->cnt, 0, sizeof(unsigned) * e->nprob, e->stream) != cudaSuccess ||
            cudaStreamSynchronize(e->stream) != cudaSuccess) {
            cudaGetLastError();
            return LLG_ERR_CUDA;
        }
        return LLG_ERR_TIMEOUT;
    }
    llg_status worst = LLG_OK;
    for (int oi = 0; oi < e->nprob; ++oi) {
        const EnsState &s = e->hst[oi];
        if (infos) {
            llg_info inf = llg_info();
            inf.iters = s.tot_iters;
            inf.restarts = s.tot_cycles;
            inf.applies = s.tot_iters;
            inf.picard_iters = steps;
            inf.rel_res_true = s.worst_rel;
            inf.status = s.worst_status;
            infos[e->caller[oi]] = inf;
        }
        if (s.worst_status != LLG_OK && worst == LLG_OK) worst = (llg_status)s.worst_status;
    }
    return worst;
}

}  // extern "C"
