// krylov.cu -- restarted GMRES (left preconditioned, all FP64) and flexible
// GMRES (FP32 preconditioner + inner matvec, FP64 Arnoldi) on the device.
//
// Arnoldi uses classical Gram--Schmidt applied twice (CGS2), as three passes
// over the basis: (A) h1 = V^T w; (B) w <- w - V h1 fused with h2 = V^T w;
// (C) w <- w - V h2 fused with ||w||^2, written straight into V_{j+1}.  Basis
// vectors are stored unnormalised with a device-side scale factor, so no extra
// normalisation pass is needed.  Dot products reduce per block and then in one
// block in a fixed order (deterministic).  The Hessenberg column, Givens
// rotations, residual estimate and stopping flag live on the device; kernels of
// later iterations return immediately once the flag is set, so the host only
// synchronises every few iterations and once per cycle.
#include <cmath>
#include <algorithm>
#include "llg_internal.h"
#include "krylov.h"
#include "reduce.cuh"

namespace llg {

int reduction_blocks(llg_ctx *c) { return 2 * c->sm_count; }

// ------------------------------------------------------------------ Arnoldi passes

enum { PASS_DOT = 0, PASS_UPD_DOT = 1, PASS_UPD_NRM = 2 };

template <int MAXV, int MODE>
__global__ void __launch_bounds__(RB_THREADS) arnoldi_pass(const double *__restrict__ V, long long ldv, int nv,
                                                                const GmresDev *__restrict__ gd,
                                                                const double *win, double *wout, long long n,
                                                                double *__restrict__ partials) {
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
    block_reduce_store<MAXV>(acc, MODE == PASS_UPD_NRM ? 1 : nv, partials + (long long)blockIdx.x * 64);
}

// Sum the per-block partials (fixed order) and finish the Arnoldi step.
// MODE 0: h1 = scale .* sums; MODE 1: h2 = scale .* sums; MODE 2: ||w||^2 -> Givens update.
__global__ void __launch_bounds__(RB_THREADS) arnoldi_reduce(const double *__restrict__ partials, int nb, int nv,
                                                             GmresDev *gd, int mode, int j) {
    if (gd->done) return;
    __shared__ double tot[64];
    block_sum_partials(partials, nb, mode == 2 ? 1 : nv, tot);
    __syncthreads();
    if (mode == 0) {
        for (int i = threadIdx.x; i < nv; i += blockDim.x) gd->h1[i] = tot[i] * gd->scale[i];
        return;
    }
    if (mode == 1) {
        for (int i = threadIdx.x; i < nv; i += blockDim.x) gd->h2[i] = tot[i] * gd->scale[i];
        return;
    }
    if (threadIdx.x != 0) return;
    const int ld = GmresDev::LD;
    double *H = gd->H;
    for (int i = 0; i <= j; ++i) H[i + ld * j] = gd->h1[i] + gd->h2[i];
    const double hn = sqrt(tot[0]);
    H[j + 1 + ld * j] = hn;
    gd->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
        const double a = H[i + ld * j], b = H[i + 1 + ld * j];
        H[i + ld * j] = gd->cs[i] * a + gd->sn[i] * b;
        H[i + 1 + ld * j] = -gd->sn[i] * a + gd->cs[i] * b;
    }
    const double a = H[j + ld * j], b = H[j + 1 + ld * j];
    const double rr = hypot(a, b);
    const double cs = rr > 0.0 ? a / rr : 1.0, sn = rr > 0.0 ? b / rr : 0.0;
    gd->cs[j] = cs;
    gd->sn[j] = sn;
    H[j + ld * j] = rr;
    H[j + 1 + ld * j] = 0.0;
    gd->g[j + 1] = -sn * gd->g[j];
    gd->g[j] = cs * gd->g[j];
    gd->jd = j + 1;
    const double est = fabs(gd->g[j + 1]);
    if (!isfinite(est) || !isfinite(hn)) {
        gd->breakdown = 1;
        gd->done = 1;
    } else if (est <= gd->target || hn == 0.0) {
        gd->done = 1;
    }
}

// start a cycle: beta = sqrt(red), g = beta e1, scale[0] = 1/beta, target = rel_factor * beta
__global__ void cycle_init(GmresDev *gd, const double *red_dev, double rel_factor, int m) {
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
}

// y = H^{-1} g (upper triangular, jd x jd); coef_i = y_i * (flexible ? 1 : scale_i)
__global__ void cycle_backsolve(GmresDev *gd, int flexible) {
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
    __shared__ double cf[64];
    const int jd = gd->jd;
    if (threadIdx.x < jd) cf[threadIdx.x] = gd->coef[threadIdx.x];
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double s = x[e];
        for (int i = 0; i < jd; ++i) s += cf[i] * (double)B[i * ldb + e];
        x[e] = s;
    }
}

// out = b - t, partial sums of out^2
__global__ void __launch_bounds__(RB_THREADS) residual_partials(const double *__restrict__ b, const double *t,
                                                                double *out, long long n, double *partials) {
    double acc[1] = {0.0};
    long long lo, hi;
    block_chunk(n, lo, hi);
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        const double r = b[e] - t[e];
        out[e] = r;
        acc[0] += r * r;
    }
    block_reduce_store<1>(acc, 1, partials + (long long)blockIdx.x * 64);
}

__global__ void __launch_bounds__(RB_THREADS) dot_partials(const double *__restrict__ a, const double *__restrict__ b,
                                                           long long n, double *partials) {
    double acc[1] = {0.0};
    long long lo, hi;
    block_chunk(n, lo, hi);
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) acc[0] += a[e] * b[e];
    block_reduce_store<1>(acc, 1, partials + (long long)blockIdx.x * 64);
}

__global__ void sum_partials(const double *__restrict__ partials, int nb, double *dst) {
    __shared__ double tot[1];
    block_sum_partials(partials, nb, 1, tot);
    __syncthreads();
    if (threadIdx.x == 0) *dst = tot[0];
}

// ------------------------------------------------------------------ host helpers

llg_status dot_async(llg_ctx *c, const double *a, const double *b, long long n, double *dst_dev) {
    const int nb = reduction_blocks(c);
    dot_partials<<<nb, RB_THREADS, 0, c->stream>>>(a, b, n, c->red);
    sum_partials<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, dst_dev);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "dot");
}

static llg_status residual_async(llg_ctx *c, const double *b, const double *t, double *out, long long n, double *dst_dev) {
    const int nb = reduction_blocks(c);
    residual_partials<<<nb, RB_THREADS, 0, c->stream>>>(b, t, out, n, c->red);
    sum_partials<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, dst_dev);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "residual");
}

template <int MAXV>
static void launch_pass(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const double *win, double *wout,
                        long long n) {
    const int nb = reduction_blocks(c);
    GmresDev *gd = c->gdev;
    if (mode == PASS_DOT)
        arnoldi_pass<MAXV, PASS_DOT><<<nb, RB_THREADS, 0, c->stream>>>(V, ldv, nv, gd, win, wout, n, c->red);
    else if (mode == PASS_UPD_DOT)
        arnoldi_pass<MAXV, PASS_UPD_DOT><<<nb, RB_THREADS, 0, c->stream>>>(V, ldv, nv, gd, win, wout, n, c->red);
    else
        arnoldi_pass<MAXV, PASS_UPD_NRM><<<nb, RB_THREADS, 0, c->stream>>>(V, ldv, nv, gd, win, wout, n, c->red);
}

static void pass_dispatch_raw(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const double *win, double *wout,
                              long long n) {
    if (nv <= 4) launch_pass<4>(c, mode, V, ldv, nv, win, wout, n);
    else if (nv <= 8) launch_pass<8>(c, mode, V, ldv, nv, win, wout, n);
    else if (nv <= 16) launch_pass<16>(c, mode, V, ldv, nv, win, wout, n);
    else if (nv <= 32) launch_pass<32>(c, mode, V, ldv, nv, win, wout, n);
    else launch_pass<64>(c, mode, V, ldv, nv, win, wout, n);
}

static void pass_dispatch(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const double *win, double *wout,
                          long long n, int j) {
    const double nd = (double)n;
    const double bytes = 8.0 * nd * (mode == PASS_DOT ? nv + 1 : nv + 2);
    const double flops = nd * (mode == PASS_DOT ? 2.0 * nv : (mode == PASS_UPD_DOT ? 4.0 * nv : 2.0 * nv + 2.0));
    prof_begin(c, K_ARNOLDI, bytes, flops, j);
    pass_dispatch_raw(c, mode, V, ldv, nv, win, wout, n);
    prof_end(c);
}

// one Arnoldi step j on w = W (CGS2); writes the unnormalised V_{j+1}
static llg_status arnoldi_step(llg_ctx *c, int j) {
    Workspace &w = c->ws;
    const long long n = w.n;
    const int nb = reduction_blocks(c), nv = j + 1;
    pass_dispatch(c, PASS_DOT, w.V, n, nv, w.W, nullptr, n, j);
    arnoldi_reduce<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, nv, c->gdev, 0, j);
    pass_dispatch(c, PASS_UPD_DOT, w.V, n, nv, w.W, w.W, n, j);
    arnoldi_reduce<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, nv, c->gdev, 1, j);
    pass_dispatch(c, PASS_UPD_NRM, w.V, n, nv, w.W, w.V + (long long)(j + 1) * n, n, j);
    arnoldi_reduce<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, nv, c->gdev, 2, j);
    c->launches += 6;
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

llg_status gmres_run(llg_ctx *c, const SolveOps &ops, bool flexible, const llg_opts *o, const double *b, double *x,
                     llg_info *info, const double *r0) {
    llg_status st = ensure_workspace(c, o->restart, flexible);
    if (st != LLG_OK) return st;
    Workspace &w = c->ws;
    w.last_res = nullptr;
    const long long n = w.n;
    const int m = o->restart;
    double *dsc = c->dsc, *hsc = c->hsc;
    GmresDev *gh = static_cast<GmresDev *>(c->ghost);

    if ((st = dot_async(c, b, b, n, dsc)) != LLG_OK) return st;
    if ((st = sync_read(c, hsc, dsc, sizeof(double))) != LLG_OK) return st;
    const double nb = std::sqrt(hsc[0]);
    llg_info inf = llg_info();
    if (nb == 0.0) {
        cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream);
        inf.status = LLG_OK;
        if (info) *info = inf;
        return LLG_OK;
    }
    auto true_residual = [&](double *rel) -> llg_status {
        llg_status s2 = ops.matvec(x, w.T);
        if (s2 != LLG_OK) return s2;
        // the residual overwrites T (left) or lands in V_0 (flexible: v_0 = r / ||r||)
        if ((s2 = residual_async(c, b, w.T, flexible ? w.V : w.T, n, dsc)) != LLG_OK) return s2;
        if ((s2 = sync_read(c, hsc, dsc, sizeof(double))) != LLG_OK) return s2;
        *rel = std::sqrt(hsc[0]) / nb;
        return LLG_OK;
    };
    double rel;
    if (r0) {
        // the caller's exact initial residual replaces the first matvec
        double *dst = flexible ? w.V : w.T;
        cudaError_t ce = cudaMemcpyAsync(dst, r0, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream);
        if ((st = cuda_check(c, ce, "initial residual")) != LLG_OK) return st;
        if ((st = dot_async(c, dst, dst, n, dsc)) != LLG_OK) return st;
        if ((st = sync_read(c, hsc, dsc, sizeof(double))) != LLG_OK) return st;
        rel = std::sqrt(hsc[0]) / nb;
    } else if ((st = true_residual(&rel)) != LLG_OK) {
        return st;
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
        if ((st = dot_async(c, w.V, w.V, n, dsc + 1)) != LLG_OK) return st;
        const double rel_factor = std::max(0.5 * o->rtol / rel, eta);
        cycle_init<<<1, 32, 0, c->stream>>>(c->gdev, dsc + 1, std::min(rel_factor, 1.0), m);
        c->launches++;
        const int jmax = std::min(m, o->max_iters - inf.iters);
        const size_t prof_first = c->prof_used;
        for (int j = 0; j < jmax; ++j) {
            const double *scale_j = &c->gdev->scale[j];
            double *vj = w.V + (long long)j * n;
            if (!flexible) {
                st = ops.pop(vj, scale_j, w.W);
            } else {
                float *zj = w.Z + (long long)j * n;
                st = ops.fprec(vj, scale_j, zj);
                if (st == LLG_OK) st = ops.fmatvec(zj, w.W);
            }
            if (st != LLG_OK) return st;
            if ((st = arnoldi_step(c, j)) != LLG_OK) return st;
            if ((j + 1) % c->sync_every == 0 && j + 1 < jmax) {
                if ((st = sync_read(c, gh, c->gdev, GMRES_HEADER_BYTES)) != LLG_OK) return st;
                if (gh->done) break;
            }
        }
        cycle_backsolve<<<1, 32, 0, c->stream>>>(c->gdev, flexible ? 1 : 0);
        const int ub = reduction_blocks(c) * 2;
        if (flexible)
            cycle_update<float><<<ub, RB_THREADS, 0, c->stream>>>(x, w.Z, n, c->gdev, n);
        else
            cycle_update<double><<<ub, RB_THREADS, 0, c->stream>>>(x, w.V, n, c->gdev, n);
        c->launches += 2;
        if ((st = cuda_check(c, cudaGetLastError(), "cycle update")) != LLG_OK) return st;
        if ((st = sync_read(c, gh, c->gdev, GMRES_HEADER_BYTES)) != LLG_OK) return st;
        prof_discard(c, prof_first, gh->jd);
        inf.iters += gh->jd;
        inf.applies += gh->jd;
        inf.restarts++;
        if (gh->breakdown) { result = LLG_ERR_BREAKDOWN; break; }
        if ((st = true_residual(&rel)) != LLG_OK) return st;
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

}  // namespace llg
