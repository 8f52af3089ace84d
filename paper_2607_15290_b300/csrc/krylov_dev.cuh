// krylov_dev.cuh -- device parts of the Gram-Schmidt passes shared by the kernels of
// krylov.cu and gs_tma.cu: the pass modes and the finish that the last block of a pass runs.
#pragma once
#include "krylov.h"
#include "reduce.cuh"

namespace llg {

enum { PASS_DOT = 0, PASS_UPD_DOT = 1, PASS_UPD_NRM = 2 };

// Finish of Arnoldi pass `mode` of step j, run by the block that completes the pass
// last: sums the per-block partials in a fixed order, then
//   mode 0: h1 = scale .* sums;  mode 1: h2 = scale .* sums;
//   mode 2: ||w||^2 -> Hessenberg column h1 + h2 and h_{j+1,j}, previous Givens
//           rotations applied, new rotation, residual estimate, stopping flag.
// The state the sequential part needs is first gathered into shared memory by all
// threads, so the single-thread part runs on shared memory, not on a chain of
// dependent global loads.
static __device__ __noinline__ void arnoldi_finish(const double *partials, int nb, int nv, GmresDev *gd, int mode, int j) {
    __shared__ double tot[64];
    __shared__ double col[GmresDev::LD + 1], cs_s[GmresDev::MAXM], sn_s[GmresDev::MAXM];
    __shared__ double gj;
    block_sum_partials_l2(partials, nb, mode == PASS_UPD_NRM ? 1 : nv, tot);
    __syncthreads();
    if (mode != PASS_UPD_NRM) {
        double *h = mode == PASS_DOT ? gd->h1 : gd->h2;
        for (int i = threadIdx.x; i < nv; i += blockDim.x) h[i] = tot[i] * gd->scale[i];
        return;
    }
    for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = gd->h1[i] + gd->h2[i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        cs_s[i] = gd->cs[i];
        sn_s[i] = gd->sn[i];
    }
    if (threadIdx.x == 0) gj = gd->g[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        const double hn = sqrt(tot[0]);
        col[j + 1] = hn;
        for (int i = 0; i < j; ++i) {
            const double a = col[i], b = col[i + 1];
            col[i] = cs_s[i] * a + sn_s[i] * b;
            col[i + 1] = -sn_s[i] * a + cs_s[i] * b;
        }
        const double a = col[j], b = col[j + 1];
        const double rr = hypot(a, b);
        const double cs = rr > 0.0 ? a / rr : 1.0, sn = rr > 0.0 ? b / rr : 0.0;
        col[j] = rr;
        col[j + 1] = 0.0;
        gd->cs[j] = cs;
        gd->sn[j] = sn;
        gd->scale[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
        gd->g[j + 1] = -sn * gj;
        gd->g[j] = cs * gj;
        gd->jd = j + 1;
        const double est = fabs(sn * gj);
        if (!isfinite(est) || !isfinite(hn)) {
            gd->breakdown = 1;
            gd->done = 1;
        } else if (est <= gd->target || hn == 0.0) {
            gd->done = 1;
        }
        if (gd->prog) {
            gd->prog[1] = j + 1;
            gd->prog[2] = gd->done;
            __threadfence_system();
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) gd->H[i + GmresDev::LD * j] = col[i];
}

}  // namespace llg
