// krylov.cu -- restarted GMRES (left preconditioned, all FP64) and flexible
// GMRES (FP32 preconditioner + inner matvec, FP64 Arnoldi) on the device.
//
// Arnoldi uses classical Gram--Schmidt applied twice (CGS2), as three passes
// over the basis: (A) h1 = V^T w; (B) w <- w - V h1 fused with h2 = V^T w;
// (C) w <- w - V h2 fused with ||w||^2, written straight into V_{j+1}.  Basis
// vectors are stored unnormalised with a device-side scale factor, so no extra
// normalisation pass is needed.  Dot products reduce per block; the block that
// finishes a pass last sums the partials in a fixed order (deterministic) and
// updates the Arnoldi state, so a step is three launches.  The Hessenberg column, Givens
// rotations, residual estimate and stopping flag live on the device, which also writes
// the completed step count and the flag into host-mapped memory; the host follows them
// without synchronising the stream, keeps one step queued behind the running one, and
// synchronises once per cycle.  Kernels of a step issued after the flag was set return
// immediately.
#include <cmath>
#include <algorithm>
#include <vector>
#include "llg_internal.h"
#include "krylov.h"
#include "reduce.cuh"
#include "convert.cuh"
#include "f32pair.cuh"
#include "krylov_dev.cuh"
#include "gs_tma.h"

namespace llg {

int reduction_blocks(llg_ctx *c) { return 2 * c->sm_count; }
int partial_capacity(llg_ctx *c) { return 8 * c->sm_count; }

// ------------------------------------------------------------------ Arnoldi passes

template <int MAXV, int MODE>
__global__ void __launch_bounds__(RB_THREADS) arnoldi_pass(const double *__restrict__ V, long long ldv, int nv,
                                                                GmresDev *gd, const double *win, double *wout, long long n,
                                                                double *__restrict__ partials) {
    pdl_wait();
    if (gd->done) return;
    __shared__ double coef[MAXV];
    if (threadIdx.x < nv) {
        const double h = (MODE == PASS_UPD_DOT) ? gd->h1[threadIdx.x] : ((MODE == PASS_UPD_NRM) ? gd->h2[threadIdx.x] : 0.0);
        coef[threadIdx.x] = h * gd->scale[threadIdx.x];
    }
    __syncthreads();
    double acc[MAXV];
#pragma unroll
    for (int i = 0; i < MAXV; ++i) acc[i] = 0.0;
    long long lo, hi;
    block_chunk(n, lo, hi);
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        double w = win[e];
        if (MODE == PASS_DOT) {
            // all basis loads of this element first, then the multiply-adds: the loads
            // must be in flight together, or the FP64 pipe waits on memory latency
            double vv[MAXV];
#pragma unroll
            for (int i = 0; i < MAXV; ++i) vv[i] = (i < nv) ? __ldg(&V[i * ldv + e]) : 0.0;
#pragma unroll
            for (int i = 0; i < MAXV; ++i)
                if (i < nv) acc[i] += vv[i] * w;
        } else {
            double vv[MAXV];
#pragma unroll
            for (int i = 0; i < MAXV; ++i) vv[i] = (i < nv) ? __ldg(&V[i * ldv + e]) : 0.0;
#pragma unroll
            for (int i = 0; i < MAXV; ++i)
                if (i < nv) w -= coef[i] * vv[i];
            wout[e] = w;
            if (MODE == PASS_UPD_DOT) {
#pragma unroll
                for (int i = 0; i < MAXV; ++i)
                    if (i < nv) acc[i] += vv[i] * w;
            } else {
                acc[0] += w * w;
            }
        }
    }
    block_reduce_store<MAXV>(acc, MODE == PASS_UPD_NRM ? 1 : nv, partials + (long long)blockIdx.x * RB_STRIDE);
    if (last_block_arrived(&gd->arrived)) arnoldi_finish(partials, gridDim.x, nv, gd, MODE, nv - 1);
}

// Passes A and C (one multiply-add per loaded basis value) for up to 16 basis
// vectors, software-pipelined: the basis values of the thread's next element are
// loaded before the multiply-adds of the current one, so memory latency overlaps
// the FP64 pipe instead of alternating with it (pass B has twice the arithmetic per
// load and saturates the pipe without this).
template <int MAXV, int MODE>
__global__ void __launch_bounds__(RB_THREADS, MAXV <= 8 ? 2 : 1) arnoldi_pass_pipe(const double *__restrict__ V, long long ldv, int nv,
                                                                                     GmresDev *gd, const double *win, double *wout,
                                                                                     long long n, double *__restrict__ partials) {
    pdl_wait();
    static_assert(MODE == PASS_DOT || MODE == PASS_UPD_NRM, "pipelined form covers passes A and C");
    if (gd->done) return;
    __shared__ double coef[MAXV];
    if (threadIdx.x < nv) coef[threadIdx.x] = MODE == PASS_UPD_NRM ? gd->h2[threadIdx.x] * gd->scale[threadIdx.x] : 0.0;
    __syncthreads();
    double acc[MAXV];
#pragma unroll
    for (int i = 0; i < MAXV; ++i) acc[i] = 0.0;
    long long lo, hi;
    block_chunk(n, lo, hi);
    const long long bd = blockDim.x;
    double va[MAXV], vb[MAXV], wa = 0.0, wb = 0.0;
    auto load = [&](double (&vv)[MAXV], double &w, long long e) {
        if (e < hi) {
            w = win[e];
#pragma unroll
            for (int i = 0; i < MAXV; ++i) vv[i] = (i < nv) ? __ldg(&V[i * ldv + e]) : 0.0;
        }
    };
    auto work = [&](const double (&vv)[MAXV], double w, long long e) {
        if (e >= hi) return;
        if (MODE == PASS_DOT) {
#pragma unroll
            for (int i = 0; i < MAXV; ++i)
                if (i < nv) acc[i] += vv[i] * w;
        } else {
#pragma unroll
            for (int i = 0; i < MAXV; ++i)
                if (i < nv) w -= coef[i] * vv[i];
            wout[e] = w;
            acc[0] += w * w;
        }
    };
    long long e = lo + threadIdx.x;
    load(va, wa, e);
    for (; e < hi; e += 2 * bd) {
        load(vb, wb, e + bd);
        work(va, wa, e);
        load(va, wa, e + 2 * bd);
        work(vb, wb, e + bd);
    }
    block_reduce_store<MAXV>(acc, MODE == PASS_UPD_NRM ? 1 : nv, partials + (long long)blockIdx.x * RB_STRIDE);
    if (last_block_arrived(&gd->arrived)) arnoldi_finish(partials, gridDim.x, nv, gd, MODE, nv - 1);
}

// The three passes of a flexible solve with FP32-pair arithmetic (f32pair.cuh).  The
// first basis vector V_0 is the FP64 true residual; every later basis vector and w are
// planar FP32 pairs (a hi plane of n floats, then a lo plane, in the same 8 bytes per
// value), so only V_0 is split on the integer pipes.  w as the FP32 inner matvec leaves
// it is its hi plane alone (lo = 0); pass B writes w - V h1 as a pair, pass C writes
// V_{j+1} as a pair.  Products and sums are error-free FP32 transformations; only the
// per-thread totals return to FP64.  The FP64 unit is then out of the loop, and the
// passes are bound by memory.  With PIPE, the next element's loads are issued before the
// current element's arithmetic.
template <int MAXV, int MODE, bool PIPE>
__global__ void __launch_bounds__(RB_THREADS, MAXV <= 16 ? 2 : 1) arnoldi_pass_pair(const double *__restrict__ V, long long ldv,
                                                                                     int nv, GmresDev *gd, const float *w_hi,
                                                                                     const float *w_lo, float *o_hi, float *o_lo,
                                                                                     long long n, double *__restrict__ partials) {
    pdl_wait();
    if (gd->done) return;
    constexpr bool WLO = MODE == PASS_UPD_NRM;   // w carries a lo plane only after pass B
    __shared__ f32x2 coef[MAXV];
    if (threadIdx.x < nv) {
        const double h = (MODE == PASS_UPD_DOT) ? gd->h1[threadIdx.x] : ((MODE == PASS_UPD_NRM) ? gd->h2[threadIdx.x] : 0.0);
        coef[threadIdx.x] = split_f64(h * gd->scale[threadIdx.x]);
    }
    __syncthreads();
    f32x2 acc[MAXV];
#pragma unroll
    for (int i = 0; i < MAXV; ++i) acc[i] = f32x2{0.0f, 0.0f};
    long long lo, hi;
    block_chunk(n, lo, hi);
    const long long bd = blockDim.x;
    struct Ld { double v0; float2 v[MAXV > 1 ? MAXV - 1 : 1]; float wh, wl; };
    auto load = [&](Ld &d, long long e) {
        if (e < hi) {
            d.wh = w_hi[e];
            d.wl = WLO ? w_lo[e] : 0.0f;
            d.v0 = __ldg(&V[e]);
#pragma unroll
            for (int i = 1; i < MAXV; ++i) {
                if (i < nv) {
                    const float *b = reinterpret_cast<const float *>(V + i * ldv);
                    d.v[i - 1] = make_float2(__ldg(&b[e]), __ldg(&b[n + e]));
                }
            }
        }
    };
    auto work = [&](const Ld &d, long long e) {
        if (e >= hi) return;
        const f32x2 w{d.wh, d.wl};
        f32x2 v[MAXV];
        v[0] = split_f64(d.v0);
#pragma unroll
        for (int i = 1; i < MAXV; ++i)
            if (i < nv) v[i] = f32x2{d.v[i - 1].x, d.v[i - 1].y};
        if (MODE == PASS_DOT) {
#pragma unroll
            for (int i = 0; i < MAXV; ++i)
                if (i < nv) fma_acc(v[i], w, acc[i]);
        } else {
            f32x2 u{0.0f, 0.0f};
#pragma unroll
            for (int i = 0; i < MAXV; ++i)
                if (i < nv) fma_acc(coef[i], v[i], u);
            const f32x2 wn = sub_pair(w, u);
            o_hi[e] = wn.hi;
            o_lo[e] = wn.lo;
            if (MODE == PASS_UPD_DOT) {
#pragma unroll
                for (int i = 0; i < MAXV; ++i)
                    if (i < nv) fma_acc(v[i], wn, acc[i]);
            } else {
                fma_acc(wn, wn, acc[0]);
            }
        }
    };
    if (PIPE) {
        Ld a, b;
        long long e = lo + threadIdx.x;
        load(a, e);
        for (; e < hi; e += 2 * bd) {
            load(b, e + bd);
            work(a, e);
            load(a, e + 2 * bd);
            work(b, e + bd);
        }
    } else {
        for (long long e = lo + threadIdx.x; e < hi; e += bd) {
            Ld d;
            load(d, e);
            work(d, e);
        }
    }
    double accd[MAXV];
#pragma unroll
    for (int i = 0; i < MAXV; ++i) accd[i] = pair_to_f64(acc[i]);
    block_reduce_store<MAXV>(accd, MODE == PASS_UPD_NRM ? 1 : nv, partials + (long long)blockIdx.x * RB_STRIDE);
    if (last_block_arrived(&gd->arrived)) arnoldi_finish(partials, gridDim.x, nv, gd, MODE, nv - 1);
}

// partial sums of a . b over n values of two basis vectors, each FP64 or a planar FP32
// pair (widened exactly), products and sums in FP64 (a measurement, not the hot path)
__global__ void __launch_bounds__(RB_THREADS) dot_mixed_partials(const double *a, int a_pair, const double *b, int b_pair,
                                                                 long long n, double *partials) {
    double acc[1] = {0.0};
    long long lo, hi;
    block_chunk(n, lo, hi);
    const float *ap = reinterpret_cast<const float *>(a), *bp = reinterpret_cast<const float *>(b);
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        const double x = a_pair ? f2d_exact(ap[e]) + f2d_exact(ap[n + e]) : a[e];
        const double y = b_pair ? f2d_exact(bp[e]) + f2d_exact(bp[n + e]) : b[e];
        acc[0] += x * y;
    }
    block_reduce_store<1>(acc, 1, partials + (long long)blockIdx.x * 64);
}

// start cycle `epoch`: beta = sqrt(red), g = beta e1, scale[0] = 1/beta, target = rel_factor * beta
__global__ void cycle_init(GmresDev *gd, const double *red_dev, double rel_factor, int m, int epoch) {
    pdl_wait();
    if (threadIdx.x != 0) return;
    const double beta = sqrt(*red_dev);
    gd->m = m;
    gd->done = 0;
    gd->jd = 0;
    gd->breakdown = 0;
    for (int i = 0; i <= m; ++i) gd->g[i] = 0.0;
    gd->g[0] = beta;
    gd->scale[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    gd->target = rel_factor * beta;
    if (!(beta > 0.0) || !isfinite(beta)) {
        gd->done = 1;
        gd->breakdown = !isfinite(beta);
    }
    gd->epoch = epoch;
    if (gd->prog) {
        // the counters first, then the epoch that makes them current
        gd->prog[1] = 0;
        gd->prog[2] = gd->done;
        __threadfence_system();
        gd->prog[0] = epoch;
        __threadfence_system();
    }
}

// y = H^{-1} g (upper triangular, jd x jd); coef_i = y_i * (flexible ? 1 : scale_i)
__global__ void cycle_backsolve(GmresDev *gd, int flexible) {
    pdl_wait();
    if (threadIdx.x != 0) return;
    const int jd = gd->jd, ld = GmresDev::LD;
    for (int i = jd - 1; i >= 0; --i) {
        double s = gd->g[i];
        for (int k = i + 1; k < jd; ++k) s -= gd->H[i + ld * k] * gd->y[k];
        gd->y[i] = s / gd->H[i + ld * i];
    }
    for (int i = 0; i < jd; ++i) gd->coef[i] = flexible ? gd->y[i] : gd->y[i] * gd->scale[i];
}

template <typename TB>
__global__ void __launch_bounds__(RB_THREADS) cycle_update(double *x, const TB *__restrict__ B, long long ldb,
                                                           const GmresDev *__restrict__ gd, long long n) {
    pdl_wait();
    __shared__ double cf[64];
    const int jd = gd->jd;
    if (threadIdx.x < jd) cf[threadIdx.x] = gd->coef[threadIdx.x];
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double s = x[e];
        // FP32 basis: widened on the integer pipes (the hardware conversion would take an
        // FP64 issue slot per element, as many as the multiply-adds)
        for (int i = 0; i < jd; ++i) s += cf[i] * to_f64(B[i * ldb + e]);
        x[e] = s;
    }
}

// x += Z y over an FP32 basis with FP32-pair arithmetic: each z value is exact in FP32, the
// coefficient a pair, the products error-free and the per-element sum a two-sum chain; one
// FP64 addition per element puts it into x (the FP64 form spends one FP64 multiply-add per
// basis value, the bound of this pass)
__global__ void __launch_bounds__(RB_THREADS) cycle_update_pair(double *x, const float *__restrict__ B, long long ldb,
                                                                const GmresDev *__restrict__ gd, long long n) {
    pdl_wait();
    __shared__ f32x2 cf[64];
    const int jd = gd->jd;
    if (threadIdx.x < jd) cf[threadIdx.x] = split_f64(gd->coef[threadIdx.x]);
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        f32x2 s{0.0f, 0.0f};
        for (int i = 0; i < jd; ++i) fma_acc(cf[i], f32x2{B[i * ldb + e], 0.0f}, s);
        x[e] += pair_to_f64(s);
    }
}

// The same update four elements a thread: 16-byte loads of every basis vector (eight vectors
// in flight at a time), the FP32-pair sums of two elements per packed instruction; per
// element the operations, their order and so the result are those of cycle_update_pair.
// x 16-byte aligned, n and ldb multiples of 4.
__global__ void __launch_bounds__(RB_THREADS) cycle_update_pair4(double *x, const float *__restrict__ B, long long ldb,
                                                                 const GmresDev *__restrict__ gd, long long n) {
    pdl_wait();
    __shared__ f32x2v2 cf[GmresDev::MAXM];
    const int jd = gd->jd;
    if (threadIdx.x < jd) {
        const f32x2 c = split_f64(gd->coef[threadIdx.x]);
        cf[threadIdx.x].hi = v2_pack(c.hi, c.hi);
        cf[threadIdx.x].lo = v2_pack(c.lo, c.lo);
    }
    __syncthreads();
    const long long n4 = n >> 2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
        f32x2v2 s01{0ull, 0ull}, s23{0ull, 0ull};
        for (int i0 = 0; i0 < jd; i0 += 8) {
            float4 bv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (i0 + k < jd) bv[k] = __ldg(reinterpret_cast<const float4 *>(B + (long long)(i0 + k) * ldb) + q);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (i0 + k < jd) {
                    const f32x2v2 b01{v2_pack(bv[k].x, bv[k].y), 0ull}, b23{v2_pack(bv[k].z, bv[k].w), 0ull};
                    fma_acc_v2(cf[i0 + k], b01, s01);
                    fma_acc_v2(cf[i0 + k], b23, s23);
                }
        }
        double2 *xp = reinterpret_cast<double2 *>(x) + 2 * q;
        double2 x01 = xp[0], x23 = xp[1];
        float h0, h1, l0, l1;
        v2_unpack(s01.hi, h0, h1);
        v2_unpack(s01.lo, l0, l1);
        x01.x += f2d_exact(h0) + f2d_exact(l0);
        x01.y += f2d_exact(h1) + f2d_exact(l1);
        v2_unpack(s23.hi, h0, h1);
        v2_unpack(s23.lo, l0, l1);
        x23.x += f2d_exact(h0) + f2d_exact(l0);
        x23.y += f2d_exact(h1) + f2d_exact(l1);
        xp[0] = x01;
        xp[1] = x23;
    }
}

// out = b - t, partial sums of out^2 (two elements a thread per 16-byte access when all three
// arrays are 16-byte aligned: the blocks' chunks start at even elements)
template <bool V2>
__global__ void __launch_bounds__(RB_THREADS) residual_partials(const double *__restrict__ b, const double *t,
                                                                double *out, long long n, double *partials) {
    pdl_wait();
    double acc[1] = {0.0};
    long long lo, hi;
    block_chunk(n, lo, hi);
    if constexpr (V2) {
        // the squares summed in FP32-pair arithmetic (off the FP64 unit, which the subtraction
        // alone then loads): about 47 bits, far more than the convergence test needs
        f32x2 s0{0.0f, 0.0f}, s1{0.0f, 0.0f};
        for (long long e = lo + 2 * threadIdx.x; e + 1 < hi; e += 2 * blockDim.x) {
            const double2 bb = *reinterpret_cast<const double2 *>(b + e), tt = *reinterpret_cast<const double2 *>(t + e);
            const double2 r = make_double2(bb.x - tt.x, bb.y - tt.y);
            *reinterpret_cast<double2 *>(out + e) = r;
            const f32x2 px = split_f64(r.x), py = split_f64(r.y);
            fma_acc(px, px, s0);
            fma_acc(py, py, s1);
        }
        if (((hi - lo) & 1) && threadIdx.x == 0) {   // an odd chunk (the last one)
            const double r = b[hi - 1] - t[hi - 1];
            out[hi - 1] = r;
            const f32x2 pr = split_f64(r);
            fma_acc(pr, pr, s1);
        }
        acc[0] = pair_to_f64(s0) + pair_to_f64(s1);
    } else {
        for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
            const double r = b[e] - t[e];
            out[e] = r;
            acc[0] += r * r;
        }
    }
    block_reduce_store<1>(acc, 1, partials + (long long)blockIdx.x * 64);
}

__global__ void __launch_bounds__(RB_THREADS) dot_partials(const double *__restrict__ a, const double *__restrict__ b,
                                                           long long n, double *partials) {
    pdl_wait();
    double acc[1] = {0.0};
    long long lo, hi;
    block_chunk(n, lo, hi);
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) acc[0] += a[e] * b[e];
    block_reduce_store<1>(acc, 1, partials + (long long)blockIdx.x * 64);
}

__global__ void sum_partials(const double *__restrict__ partials, int nb, double *dst) {
    pdl_wait();
    __shared__ double tot[1];
    block_sum_partials(partials, nb, 1, tot);
    __syncthreads();
    if (threadIdx.x == 0) *dst = tot[0];
}

// ------------------------------------------------------------------ host helpers

llg_status dot_async(llg_ctx *c, const double *a, const double *b, long long n, double *dst_dev) {
    const int nb = reduction_blocks(c);
    launch_pdl(dot_partials, dim3(nb), dim3(RB_THREADS), 0, c->stream, a, b, n, c->red);
    launch_pdl(sum_partials, dim3(1), dim3(RB_THREADS), 0, c->stream, c->red, nb, dst_dev);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "dot");
}

static llg_status residual_async(llg_ctx *c, const double *b, const double *t, double *out, long long n, double *dst_dev) {
    const int nb = reduction_blocks(c);
    const bool v2 = (((uintptr_t)b | (uintptr_t)t | (uintptr_t)out) & 15u) == 0;
    if (v2) launch_pdl(residual_partials<true>, dim3(nb), dim3(RB_THREADS), 0, c->stream, b, t, out, n, c->red);
    else launch_pdl(residual_partials<false>, dim3(nb), dim3(RB_THREADS), 0, c->stream, b, t, out, n, c->red);
    launch_pdl(sum_partials, dim3(1), dim3(RB_THREADS), 0, c->stream, c->red, nb, dst_dev);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "residual");
}

// blocks of an Arnoldi pass: every SM filled to the kernel's occupancy (one wave),
// capped by the capacity of the partial-sum buffer
template <typename K> static int arnoldi_grid(llg_ctx *c, K kern) {
    for (const auto &p : c->occ)
        if (p.first == (const void *)kern) return p.second;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, RB_THREADS, 0) != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 1;
    }
    const int nb = std::min(per * c->sm_count, partial_capacity(c));
    c->occ.push_back({(const void *)kern, nb});
    return nb;
}

// One instantiation per basis count up to 32 (restart 30 needs 31): a kernel compiled
// for more vectors than it uses still spends FP64 issue slots on the predicated-off
// multiply-adds, which costs up to half of a pass.  Above 32, buckets of 8.
template <int MAXV>
static void launch_pass(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const double *win, double *wout,
                        long long n) {
    GmresDev *gd = c->gdev;
#define LLG_AP(KERN)                                                                      \
    {                                                                                     \
        auto k = KERN;                                                                    \
        const int nb = arnoldi_grid(c, k);                                                \
        launch_pdl(k, dim3(nb), dim3(RB_THREADS), 0, c->stream, V, ldv, nv, gd, win, wout, n, c->red);        \
        return;                                                                           \
    }
    if constexpr (MAXV <= 16) {
        if (mode == PASS_DOT) LLG_AP((arnoldi_pass_pipe<MAXV, PASS_DOT>))
        if (mode == PASS_UPD_NRM) LLG_AP((arnoldi_pass_pipe<MAXV, PASS_UPD_NRM>))
    }
    if (mode == PASS_DOT) LLG_AP((arnoldi_pass<MAXV, PASS_DOT>))
    if (mode == PASS_UPD_DOT) LLG_AP((arnoldi_pass<MAXV, PASS_UPD_DOT>))
    LLG_AP((arnoldi_pass<MAXV, PASS_UPD_NRM>))
#undef LLG_AP
}

template <int MAXV>
static void launch_pass_pair(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const float *wh,
                             const float *wl, float *oh, float *ol, long long n) {
    GmresDev *gd = c->gdev;
    // passes A and C (one multiply-add term per loaded value) load the next element ahead;
    // pass B, with two terms per value, runs at higher occupancy instead (beyond 8 vectors the
    // second set of loads would spill registers anyway)
    constexpr bool pipe = MAXV <= 8;
#define LLG_APP(KERN)                                                                                      \
    {                                                                                                      \
        auto k = KERN;                                                                                     \
        const int nb = arnoldi_grid(c, k);                                                                 \
        launch_pdl(k, dim3(nb), dim3(RB_THREADS), 0, c->stream, V, ldv, nv, gd, wh, wl, oh, ol, n, c->red); \
        return;                                                                                            \
    }
    if (mode == PASS_DOT) LLG_APP((arnoldi_pass_pair<MAXV, PASS_DOT, pipe>))
    if (mode == PASS_UPD_DOT) LLG_APP((arnoldi_pass_pair<MAXV, PASS_UPD_DOT, false>))
    LLG_APP((arnoldi_pass_pair<MAXV, PASS_UPD_NRM, pipe>))
#undef LLG_APP
}

// the pair passes are compiled for 1..32 basis vectors (restart <= 32)
static void pass_dispatch_pair(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const float *wh,
                               const float *wl, float *oh, float *ol, long long n) {
#define LLG_NVP(K) case K: return launch_pass_pair<K>(c, mode, V, ldv, nv, wh, wl, oh, ol, n);
    switch (nv) {
        LLG_NVP(1) LLG_NVP(2) LLG_NVP(3) LLG_NVP(4) LLG_NVP(5) LLG_NVP(6) LLG_NVP(7) LLG_NVP(8)
        LLG_NVP(9) LLG_NVP(10) LLG_NVP(11) LLG_NVP(12) LLG_NVP(13) LLG_NVP(14) LLG_NVP(15) LLG_NVP(16)
        LLG_NVP(17) LLG_NVP(18) LLG_NVP(19) LLG_NVP(20) LLG_NVP(21) LLG_NVP(22) LLG_NVP(23) LLG_NVP(24)
        LLG_NVP(25) LLG_NVP(26) LLG_NVP(27) LLG_NVP(28) LLG_NVP(29) LLG_NVP(30) LLG_NVP(31) LLG_NVP(32)
        default: break;
    }
#undef LLG_NVP
}

static void pass_dispatch_raw(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const double *win, double *wout,
                              long long n) {
#define LLG_NV(K) case K: return launch_pass<K>(c, mode, V, ldv, nv, win, wout, n);
    switch (nv) {
        LLG_NV(1) LLG_NV(2) LLG_NV(3) LLG_NV(4) LLG_NV(5) LLG_NV(6) LLG_NV(7) LLG_NV(8)
        LLG_NV(9) LLG_NV(10) LLG_NV(11) LLG_NV(12) LLG_NV(13) LLG_NV(14) LLG_NV(15) LLG_NV(16)
        LLG_NV(17) LLG_NV(18) LLG_NV(19) LLG_NV(20) LLG_NV(21) LLG_NV(22) LLG_NV(23) LLG_NV(24)
        LLG_NV(25) LLG_NV(26) LLG_NV(27) LLG_NV(28) LLG_NV(29) LLG_NV(30) LLG_NV(31) LLG_NV(32)
        default: break;
    }
#undef LLG_NV
    if (nv <= 40) launch_pass<40>(c, mode, V, ldv, nv, win, wout, n);
    else if (nv <= 48) launch_pass<48>(c, mode, V, ldv, nv, win, wout, n);
    else if (nv <= 56) launch_pass<56>(c, mode, V, ldv, nv, win, wout, n);
    else launch_pass<64>(c, mode, V, ldv, nv, win, wout, n);
}

// one Arnoldi step j on w = W (CGS2); writes the unnormalised V_{j+1} (a planar FP32 pair
// with `pairs`, where W holds the matvec's FP32 output in its hi plane)
static llg_status arnoldi_step(llg_ctx *c, int j, bool pairs) {
    Workspace &w = c->ws;
    const long long n = w.n;
    const int nv = j + 1;
    // algorithmic bytes and flops of the three passes: (nv + 1) + 2 (nv + 2) words and
    // nv + 2 nv + (nv + 1) multiply-adds per unknown (FP64 multiply-adds, or their FP32-pair
    // equivalents); profiled as one interval of 3 launches
    const double nd = (double)n;
    prof_begin(c, K_ARNOLDI, 8.0 * nd * (3.0 * nv + 5.0), nd * (8.0 * nv + 2.0), j, 3);
    if (pairs) {
        float *wh = reinterpret_cast<float *>(w.W), *wl = wh + n;
        float *vh = reinterpret_cast<float *>(w.V + (long long)(j + 1) * n), *vl = vh + n;
        if (gst::available(c, n)) {
            // operands staged in shared memory by bulk copies
            cudaError_t e = gst::pass(c, PASS_DOT, w.V, n, nv, wh, nullptr, nullptr, nullptr, n);
            if (e == cudaSuccess) e = gst::pass(c, PASS_UPD_DOT, w.V, n, nv, wh, nullptr, wh, wl, n);
            if (e == cudaSuccess) e = gst::pass(c, PASS_UPD_NRM, w.V, n, nv, wh, wl, vh, vl, n);
            if (e != cudaSuccess) { prof_end(c); return cuda_check(c, e, "Gram-Schmidt pass"); }
        } else {
            pass_dispatch_pair(c, PASS_DOT, w.V, n, nv, wh, nullptr, nullptr, nullptr, n);
            pass_dispatch_pair(c, PASS_UPD_DOT, w.V, n, nv, wh, nullptr, wh, wl, n);
            pass_dispatch_pair(c, PASS_UPD_NRM, w.V, n, nv, wh, wl, vh, vl, n);
        }
    } else {
        pass_dispatch_raw(c, PASS_DOT, w.V, n, nv, w.W, nullptr, n);
        pass_dispatch_raw(c, PASS_UPD_DOT, w.V, n, nv, w.W, w.W, n);
        pass_dispatch_raw(c, PASS_UPD_NRM, w.V, n, nv, w.W, w.V + (long long)(j + 1) * n, n);
    }
    prof_end(c);
    c->launches += 3;
    return cuda_check(c, cudaGetLastError(), "arnoldi");
}

llg_status ensure_workspace(llg_ctx *c, int restart, bool flexible) {
    Workspace &w = c->ws;
    const long long n = 4 * c->geo.N;
    if (w.restart >= restart && w.n == n && (!flexible || w.Z)) return LLG_OK;
    cudaFree(w.V); cudaFree(w.Z); cudaFree(w.W); cudaFree(w.T); cudaFree(w.R);
    w = Workspace();
    const int m = std::max(restart, 1);
    cudaError_t e = cudaMalloc(&w.V, sizeof(double) * n * (m + 1));
    if (e == cudaSuccess) e = cudaMalloc(&w.W, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&w.T, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&w.R, sizeof(double) * n);
    if (e == cudaSuccess && flexible) e = cudaMalloc(&w.Z, sizeof(float) * n * m);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(w.V); cudaFree(w.Z); cudaFree(w.W); cudaFree(w.T); cudaFree(w.R);
        w = Workspace();
        return set_error(c, LLG_ERR_OOM, "GMRES workspace allocation failed");
    }
    w.restart = m;
    w.n = n;
    return LLG_OK;
}

static llg_status sync_read(llg_ctx *c, void *dst_host, const void *src_dev, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst_host, src_dev, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "device->host read");
}

// Wait until the running cycle (number `epoch`) has completed `need` Arnoldi steps or set
// its stopping flag (*done = 1), reading the progress words the kernels write into host
// memory; the stream is not synchronised.  Should the stream drain without the words
// showing either (they are written before each step's last kernel ends), the device
// header decides.
static llg_status wait_progress(llg_ctx *c, int epoch, int need, int *done) {
    volatile int *pw = c->hprog;
    *done = 0;
    for (;;) {
        if (pw[0] == epoch) {
            const int jd = pw[1], dn = pw[2];
            if (dn) { *done = 1; return LLG_OK; }
            if (jd >= need) return LLG_OK;
        } else if (need <= 0) {
            return LLG_OK;
        }
        const cudaError_t q = cudaStreamQuery(c->stream);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return cuda_check(c, q, "GMRES cycle");
        // idle stream: every issued step has finished and written its words
        if (pw[0] == epoch && (pw[2] || pw[1] >= need)) continue;
        GmresDev *gh = static_cast<GmresDev *>(c->ghost);
        const llg_status st = sync_read(c, gh, c->gdev, GMRES_HEADER_BYTES);
        if (st != LLG_OK) return st;
        *done = gh->done;
        return LLG_OK;
    }
}

llg_status gmres_run(llg_ctx *c, const SolveOps &ops, bool flexible, const llg_opts *o, const double *b, double *x,
                     llg_info *info, const double *r0) {
    llg_status st = ensure_workspace(c, o->restart, flexible);
    if (st != LLG_OK) return st;
    Workspace &w = c->ws;
    w.last_res = nullptr;
    const long long n = w.n;
    const int m = o->restart;
    // FP32-pair Gram-Schmidt: flexible solves with at most 32 basis vectors
    const bool pairs = flexible && o->gs_arith == LLG_GS_F32X2 && m <= 32 && ops.fprec32 && ops.fmatvec32;
    w.pairs = pairs;
    double *dsc = c->dsc, *hsc = c->hsc;
    GmresDev *gh = static_cast<GmresDev *>(c->ghost);

    // ||b||^2 -> dsc[0]; with a caller's initial residual r0 (copied into V_0 or T), ||r0||^2
    // -> dsc[2] in the same round trip
    if (ops.bnorm_slot < 0 && (st = dot_async(c, b, b, n, dsc)) != LLG_OK) return st;
    if (r0) {
        double *dst = flexible ? w.V : w.T;
        if (!(ops.r0_ready && dst == r0)) {
            cudaError_t ce = cudaMemcpyAsync(dst, r0, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream);
            if ((st = cuda_check(c, ce, "initial residual")) != LLG_OK) return st;
            if ((st = dot_async(c, dst, dst, n, dsc + 2)) != LLG_OK) return st;
        }
    }
    const int nread = std::max(std::max(ops.node_check ? SolveOps::NODE_CHECK_SLOT + 1 : 1, r0 ? 3 : 1), ops.bnorm_slot + 1);
    if ((st = sync_read(c, hsc, dsc, nread * sizeof(double))) != LLG_OK) return st;
    if (ops.node_check) {
        const double minn2 = -hsc[SolveOps::NODE_CHECK_SLOT];
        if (!(minn2 > 0.0) || !std::isfinite(minn2))
            return set_error(c, LLG_ERR_DEGENERATE_NODE, "some node has |m_i| = 0 (or non-finite): the saddle matrix is singular");
    }
    const double nb = std::sqrt(hsc[ops.bnorm_slot < 0 ? 0 : ops.bnorm_slot]);
    llg_info inf = llg_info();
    if (nb == 0.0) {
        cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream);
        inf.status = LLG_OK;
        if (info) *info = inf;
        return LLG_OK;
    }
    // the true residual r = b - A x: into T (left) or V_0 (flexible: v_0 = r / ||r||), ||r||^2
    // into dsc[0]; the caller reads it
    auto issue_true_residual = [&]() -> llg_status {
        llg_status s2 = ops.matvec(x, w.T);
        if (s2 != LLG_OK) return s2;
        return residual_async(c, b, w.T, flexible ? w.V : w.T, n, dsc);
    };
    double rel;
    // device location of ||V_0||^2 for the flexible cycle start (V_0 holds the residual itself)
    const double *v0sq = dsc;
    if (r0) {
        rel = std::sqrt(hsc[2]) / nb;
        v0sq = dsc + 2;
    } else {
        if ((st = issue_true_residual()) != LLG_OK) return st;
        if ((st = sync_read(c, hsc, dsc, sizeof(double))) != LLG_OK) return st;
        rel = std::sqrt(hsc[0]) / nb;
    }
    w.last_res = flexible ? w.V : w.T;
    const double eta = flexible ? 1e-5 : 0.0;
    llg_status result = LLG_OK;
    for (;;) {
        inf.rel_res_true = rel;
        if (!std::isfinite(rel)) { result = LLG_ERR_BREAKDOWN; break; }
        if (rel <= o->rtol) { result = LLG_OK; break; }
        if (inf.iters >= o->max_iters) { result = LLG_ERR_NOT_CONVERGED; break; }
        // v_0
        if (!flexible) {
            if ((st = ops.prec(w.T, nullptr, w.V)) != LLG_OK) return st;
            inf.applies++;
        }
        if (!flexible && (st = dot_async(c, w.V, w.V, n, dsc + 1)) != LLG_OK) return st;
        const double rel_factor = std::max(0.5 * o->rtol / rel, eta);
        const int epoch = ++c->cycle_epoch;
        launch_pdl(cycle_init, dim3(1), dim3(32), 0, c->stream, c->gdev, flexible ? v0sq : dsc + 1, std::min(rel_factor, 1.0), m, epoch);
        c->launches++;
        const int jmax = std::min(m, o->max_iters - inf.iters);
        const size_t prof_first = c->prof_used;
        for (int j = 0; j < jmax; ++j) {
            const double *scale_j = &c->gdev->scale[j];
            double *vj = w.V + (long long)j * n;
            if (!flexible) {
                st = ops.pop(vj, scale_j, w.W);
            } else if (pairs) {
                float *zj = w.Z + (long long)j * n;
                float *w32 = reinterpret_cast<float *>(w.W);
                // V_0 is FP64; V_j (j >= 1) a planar pair whose hi plane the FP32 preconditioner reads
                if (ops.fpm && ops.fpm32) {
                    st = j == 0 ? ops.fpm(vj, scale_j, zj, w32)
                                : ops.fpm32(reinterpret_cast<const float *>(vj), scale_j, zj, w32);
                } else {
                    st = j == 0 ? ops.fprec(vj, scale_j, zj) : ops.fprec32(reinterpret_cast<const float *>(vj), scale_j, zj);
                    if (st == LLG_OK) st = ops.fmatvec32(zj, w32);
                }
            } else {
                float *zj = w.Z + (long long)j * n;
                st = ops.fprec(vj, scale_j, zj);
                if (st == LLG_OK) st = ops.fmatvec(zj, w.W);
            }
            if (st != LLG_OK) return st;
            if ((st = arnoldi_step(c, j, pairs)) != LLG_OK) return st;
            if (j + 1 == jmax) break;
            if (c->hprog) {
                // keep one step queued behind the running one: wait for steps 0..j-1, stop once
                // the cycle's flag is up (at most step j+1 is then issued in vain, and returns
                // at once)
                int done = 0;
                if ((st = wait_progress(c, epoch, j, &done)) != LLG_OK) return st;
                if (done) break;
            } else if ((j + 1) % c->sync_every == 0) {
                if ((st = sync_read(c, gh, c->gdev, GMRES_HEADER_BYTES)) != LLG_OK) return st;
                if (gh->done) break;
            }
        }
        launch_pdl(cycle_backsolve, dim3(1), dim3(32), 0, c->stream, c->gdev, flexible ? 1 : 0);
        const int ub = reduction_blocks(c) * 2;
        if (flexible && pairs && ((uintptr_t)x & 15u) == 0 && n % 4 == 0)
            launch_pdl(cycle_update_pair4, dim3(ub), dim3(RB_THREADS), 0, c->stream, x, (const float *)w.Z, n,
                       (const GmresDev *)c->gdev, n);
        else if (flexible && pairs)
            launch_pdl(cycle_update_pair, dim3(ub), dim3(RB_THREADS), 0, c->stream, x, (const float *)w.Z, n,
                       (const GmresDev *)c->gdev, n);
        else if (flexible)
            launch_pdl(cycle_update<float>, dim3(ub), dim3(RB_THREADS), 0, c->stream, x, w.Z, n, c->gdev, n);
        else
            launch_pdl(cycle_update<double>, dim3(ub), dim3(RB_THREADS), 0, c->stream, x, w.V, n, c->gdev, n);
        c->launches += 2;
        if ((st = cuda_check(c, cudaGetLastError(), "cycle update")) != LLG_OK) return st;
        // the true residual is queued behind the update before the cycle's header is read,
        // so one host round trip serves both
        if ((st = issue_true_residual()) != LLG_OK) return st;
        cudaError_t ce = cudaMemcpyAsync(gh, c->gdev, GMRES_HEADER_BYTES, cudaMemcpyDeviceToHost, c->stream);
        if ((st = cuda_check(c, ce, "cycle header")) != LLG_OK) return st;
        if ((st = sync_read(c, hsc, dsc, sizeof(double))) != LLG_OK) return st;
        prof_discard(c, prof_first, gh->jd);
        inf.iters += gh->jd;
        inf.applies += gh->jd;
        inf.restarts++;
        if (gh->breakdown) { result = LLG_ERR_BREAKDOWN; break; }
        rel = std::sqrt(hsc[0]) / nb;
        v0sq = dsc;
        if (gh->jd == 0) { inf.rel_res_true = rel; result = rel <= o->rtol ? LLG_OK : LLG_ERR_NOT_CONVERGED; break; }
    }
    inf.status = result;
    if (info) *info = inf;
    if (result != LLG_OK) {
        if (result == LLG_ERR_NOT_CONVERGED) set_error(c, result, "GMRES reached max_iters");
        else set_error(c, result, "GMRES breakdown (non-finite residual)");
    }
    return result;
}

// Orthogonality of the last GMRES cycle's basis: max_{i,k} |delta_ik - (s_i V_i).(s_k V_k)|
// over the stored vectors (s_i the device-side scales), the dot products in FP64.  In a
// flexible solve V_0 holds the final true residual once the solve has returned, so the
// measurement starts at V_1 there.
llg_status krylov_orthogonality(llg_ctx *c, double *max_dev, int *nvec) {
    Workspace &w = c->ws;
    if (!w.V) return set_error(c, LLG_ERR_INVALID_ARG, "no GMRES solve has run on this context");
    GmresDev *gh = static_cast<GmresDev *>(c->ghost);
    llg_status st = sync_read(c, gh, c->gdev, sizeof(GmresDev));
    if (st != LLG_OK) return st;
    const int first = w.last_res == w.V ? 1 : 0;
    const int last = gh->jd;   // V_0 .. V_jd were written by the cycle
    const int cnt = last - first + 1;
    if (cnt < 1) return set_error(c, LLG_ERR_INVALID_ARG, "the last cycle stored no basis vector");
    double *dots = nullptr;
    cudaError_t e = cudaMalloc(&dots, sizeof(double) * cnt * cnt);
    if (e != cudaSuccess) { cudaGetLastError(); return set_error(c, LLG_ERR_OOM, "orthogonality buffer"); }
    const long long n = w.n;
    const int nb = reduction_blocks(c);
    for (int i = 0; i < cnt && st == LLG_OK; ++i)
        for (int k = i; k < cnt; ++k) {
            // in a solve with FP32-pair Gram-Schmidt every vector after V_0 is a planar pair
            const int ia = first + i, ib = first + k;
            launch_pdl(dot_mixed_partials, dim3(nb), dim3(RB_THREADS), 0, c->stream, (const double *)(w.V + (long long)ia * n),
                       (int)(w.pairs && ia > 0), (const double *)(w.V + (long long)ib * n), (int)(w.pairs && ib > 0), n, c->red);
            launch_pdl(sum_partials, dim3(1), dim3(RB_THREADS), 0, c->stream, (const double *)c->red, nb, dots + i * cnt + k);
            c->launches += 2;
        }
    if (st == LLG_OK) st = cuda_check(c, cudaGetLastError(), "orthogonality");
    std::vector<double> hd((size_t)cnt * cnt);
    if (st == LLG_OK) st = sync_read(c, hd.data(), dots, sizeof(double) * cnt * cnt);
    cudaFree(dots);
    if (st != LLG_OK) return st;
    double worst = 0.0;
    for (int i = 0; i < cnt; ++i)
        for (int k = i; k < cnt; ++k) {
            const double g = hd[(size_t)i * cnt + k] * gh->scale[first + i] * gh->scale[first + k];
            worst = std::max(worst, std::fabs((i == k ? 1.0 : 0.0) - g));
        }
    *max_dev = worst;
    *nvec = cnt;
    return LLG_OK;
}

}  // namespace llg
