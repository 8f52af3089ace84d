// krylov.h -- device-side Arnoldi state and the GMRES driver interface.
#pragma once
#include <functional>
#include "llg_internal.h"

namespace llg {

// Arnoldi state of one GMRES cycle, resident in device memory.  The small
// header (flags, counters) comes first so the host can poll it cheaply.
struct GmresDev {
    static constexpr int MAXM = 64;
    static constexpr int LD = MAXM + 1;
    int done;        // cycle finished (converged estimate, breakdown or happy breakdown)
    int jd;          // Arnoldi steps completed in this cycle
    int breakdown;   // non-finite value met
    int m;           // restart length of the cycle
    double target;   // stop when |g_{j+1}| <= target
    double pad[3];
    double H[LD * MAXM];   // Hessenberg, column-major, rotated in place
    double cs[MAXM], sn[MAXM];
    double g[LD];          // rotated right-hand side beta e1
    double y[MAXM], coef[MAXM];
    double scale[LD];      // 1 / ||V_i|| of the stored (unnormalised) basis vectors
    double h1[MAXM], h2[MAXM];
    unsigned int arrived;  // blocks of the running Arnoldi pass that have stored their partial sums
    int epoch;             // number of the running cycle (set by cycle_init)
    // progress words in host-mapped memory, written as the cycle advances:
    // [0] epoch of the cycle they describe, [1] Arnoldi steps completed, [2] stopping flag.
    // NULL when mapped memory is unavailable (the host then polls the header).
    volatile int *prog;
};
static constexpr size_t GMRES_HEADER_BYTES = 32;

struct SolveOps {
    // y = A x in FP64 (true residual)
    std::function<llg_status(const double *x, double *y)> matvec;
    // y = M^{-1} (s x) in FP64, s = *scale (NULL: 1)
    std::function<llg_status(const double *x, const double *scale, double *y)> prec;
    // y = M^{-1} A (s x) in FP64 (left-preconditioned operator)
    std::function<llg_status(const double *x, const double *scale, double *y)> pop;
    // flexible GMRES: z = P(s x) stored FP32, then w = A z stored FP64
    std::function<llg_status(const double *x, const double *scale, float *z)> fprec;
    std::function<llg_status(const float *z, double *w)> fmatvec;
    // flexible GMRES with FP32-pair Gram-Schmidt: z = P(s x) from an FP32 input (the hi plane
    // of a planar-pair basis vector), and w = A z stored FP32 (the hi plane of w)
    std::function<llg_status(const float *x, const double *scale, float *z)> fprec32;
    std::function<llg_status(const float *z, float *w)> fmatvec32;
    // the same two operators as one fused sequence (z written, then w = A z), from the FP64
    // first basis vector or from the hi plane of a later one; empty when unavailable
    std::function<llg_status(const double *x, const double *scale, float *z, float *w)> fpm;
    std::function<llg_status(const float *x, const double *scale, float *z, float *w)> fpm32;
    // the caller has queued max_i -|m_i|^2 into device scalar NODE_CHECK_SLOT: gmres_run reads
    // it with its first scalars and fails with LLG_ERR_DEGENERATE_NODE unless |m_i| > 0
    static constexpr int NODE_CHECK_SLOT = 3;
    bool node_check = false;
    // the initial residual passed to gmres_run already sits in the workspace buffer the
    // cycle starts from (V_0, or T for left preconditioning) and its squared norm in device
    // scalar 2: no copy, no dot product
    bool r0_ready = false;
    // >= 0: ||b||^2 already sits in this device scalar (the right-hand side is shared by the
    // solves of a step): no dot product
    int bnorm_slot = -1;
};

llg_status ensure_workspace(llg_ctx *c, int restart, bool flexible);
// r0 (optional, FP64, 4N): the exact initial residual b - A x of the given x, when the
// caller can form it without a matvec.  On return c->ws.last_res points at the final
// FP64 true residual b - A x (NULL when b = 0); it stays valid until the next solve.
llg_status gmres_run(llg_ctx *c, const SolveOps &ops, bool flexible, const llg_opts *o, const double *b, double *x,
                     llg_info *info, const double *r0 = nullptr);

// max |I - V^T V| over the last cycle's normalised basis vectors (HOST outputs)
llg_status krylov_orthogonality(llg_ctx *c, double *max_dev, int *nvec);

}  // namespace llg
