/*
 * llg.h -- C ABI of the B300 (sm_103a) FFT--HSS preconditioned GMRES library
 * for the periodic tangent-plane Landau--Lifshitz--Gilbert saddle system.
 *
 * Problem (paper Sec. 2.4, eqs. "total system 2" and "saddle point system";
 * Sec. 3.3, eq. "C-N"): on a periodic grid with N_g nodes, find the velocity
 * v (3 components per node) and multiplier r (1 per node) with
 *
 *   [ A(m)  B(m)^T ] [v]   [f]      A = alpha I + theta k Chat (-Lap_N) + [m]x,
 *   [ -B(m)   0    ] [r] = [0],     B v = (m_i . v_i)_i,  Chat = (1 + alpha^2) c_ex.
 *
 * The second block row is negated as in the paper; the solution is the same.
 *
 * Memory layout (all calls): structure-of-arrays planes, node index
 * j = ix + n0 * (iy + n1 * iz) (x fastest).  m has 3 planes (m1|m2|m3);
 * a saddle vector x has 4 planes (v1|v2|v3|r).  Every array argument is a
 * caller-owned DEVICE pointer (cudaMalloc or torch) on the device current when
 * the context was created, unless stated otherwise; inputs and outputs must not
 * alias.  Pointers must be 16-byte aligned.
 *
 * Execution: every call is enqueued on the context's stream.  Calls that
 * return an llg_info (solves, steps, adjoint) synchronise that stream before
 * returning; the others are asynchronous.  Argument errors are detected on the
 * host before any launch.  A context is not thread-safe: one context per
 * stream.  Errors are returned as status codes; llg_last_error() gives text.
 */
#ifndef LLG_H
#define LLG_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LLG_OK = 0,
    LLG_ERR_INVALID_ARG = 1,      /* null pointer, bad parameter value */
    LLG_ERR_UNSUPPORTED_SIZE = 2, /* grid axis not a power of two in [2, 1024] */
    LLG_ERR_NOT_CONVERGED = 3,    /* iteration cap reached; outputs hold the last iterate */
    LLG_ERR_BREAKDOWN = 4,        /* non-finite residual in GMRES */
    LLG_ERR_DEGENERATE_NODE = 5,  /* |m_i| = 0 at some node: the saddle matrix is singular */
    LLG_ERR_TIMEOUT = 6,          /* a bounded device wait gave up */
    LLG_ERR_OOM = 7,              /* device allocation failed */
    LLG_ERR_CUDA = 8              /* CUDA runtime error */
} llg_status;

enum { LLG_EX_SPECTRAL = 0, LLG_EX_FD2 = 1 };
/* precision of a solve: all FP64 (left-preconditioned GMRES on M^{-1}A), or flexible GMRES
   with the FFT--HSS application and its inner matvec in FP32 (Arnoldi, least squares,
   true residual and the solution update stay FP64) */
enum { LLG_PREC_FP64 = 0, LLG_PREC_FP32_FLEX = 1 };
/* left preconditioner of GMRES (Sec. 4.3 comparison): the split FFT--HSS preconditioner
   (lambda I + S)^{-1} (lambda I + H)^{-1} of Sec. 3.2; the shifted symmetric part
   (lambda I + H)^{-1} alone (Algorithm 1 on the velocity, r / lambda on the multiplier); none */
enum { LLG_PC_FFTHSS = 0, LLG_PC_HERMITIAN = 1, LLG_PC_NONE = 2 };
/* arithmetic of the Gram--Schmidt passes (llg_opts.gs_arith) */
enum { LLG_GS_FP64 = 0, LLG_GS_F32X2 = 1 };
/* arithmetic of the FP64-accurate Fourier chains outside the Krylov cycles (llg_opts.chain_arith) */
enum { LLG_CHAIN_FP64 = 0, LLG_CHAIN_F32X2 = 1 };
/* pass plan of 3D FP32 Fourier round trips (llg_set_pass_plan) */
enum { LLG_PLAN_FIVE = 0, LLG_PLAN_CLUSTER = 1 };

typedef struct llg_ctx llg_ctx;

/* periodic cell prod_l (0, L_l); n[l] points per axis, a power of two in [2, 1024];
   dim = 2 uses n[0], n[1] (n[2] ignored) */
typedef struct {
    int dim;
    int n[3];
    double L[3];
} llg_grid;

/* alpha > 0 damping; c_ex > 0 normalised exchange coefficient (paper: 1);
   k >= 0 time step; theta in {1, 1/2} (Euler / midpoint; steps set it themselves);
   lambda > 0 HSS shift; h_ext uniform applied field; exchange = LLG_EX_*;
   h_field: optional per-node applied field added to h_ext in the lower-order field h_low
   (DEVICE, 3 FP64 planes, caller-owned, read by the right-hand side and the energy; NULL =
   none).  A time-dependent field (e.g. a manufactured-solution forcing, Sec. 4.2) is passed
   per step, sampled where the scheme samples h_low: t_{n+1} (Euler), t_{n+1/2} (midpoint).
   The ensemble rejects a non-NULL h_field.
   k_an, e_an: uniaxial anisotropy energy k_an (1 - (e_an.m)^2) (field 2 k_an (e_an.m) e_an;
   e_an a unit vector; k_an = 0: none); demag = 1: the periodic zero-mean demagnetising field
   h^(xi) = -xi'(xi'.m^)/|xi|^2 (xi' = xi with Nyquist components zeroed), Sec. 2.2, 4.6.
   Both enter h_low, evaluated at m^n (Euler) or at the Picard midpoint field (midpoint),
   and the energy; the ensemble and the adjoint reject them. */
typedef struct {
    double alpha, c_ex, k, theta, lambda;
    double h_ext[3];
    int exchange;
    const double *h_field;
    double k_an;
    double e_an[3];
    int demag;
} llg_params;

typedef struct {
    int restart;        /* GMRES restart length, 1..64 */
    int max_iters;      /* cap on total Arnoldi steps per solve */
    double rtol;        /* stop when ||b - A x|| <= rtol ||b|| (true residual, FP64) */
    int precision;      /* LLG_PREC_* */
    int picard_max;     /* midpoint: cap on Picard iterations */
    double picard_tol;  /* midpoint: stop when ||v^p - v^{p-1}|| <= picard_tol ||v^p|| */
    int diagnostics;    /* steps: 1 = also compute energies and the dissipation residual */
    int preconditioner; /* forward solves: LLG_PC_FFTHSS (default), LLG_PC_HERMITIAN, LLG_PC_NONE;
                           transposed (adjoint) solves always use FFT--HSS */
    int gs_arith;       /* arithmetic of the Gram--Schmidt passes of flexible solves (no counterpart
                           in the paper): LLG_GS_FP64 = FP64 multiply-adds on FP64 data;
                           LLG_GS_F32X2 = FP32-pair arithmetic (error-free FP32 products, Dekker
                           1971, and two-sums, Knuth 4.2.2) on a basis whose vectors after the
                           first are stored as planar FP32 pairs (about 47 significant bits), so
                           the passes run on the FP32 pipes; the correction Z y of each cycle is
                           summed the same way and added to the FP64 solution.  The first basis
                           vector, the true residual, the Hessenberg least squares and the
                           solution stay FP64.
                           Used by FP32_FLEX solves with restart <= 32; other solves run FP64. */
    int chain_arith;    /* arithmetic of the Fourier chains that the method needs to FP64 accuracy
                           outside the Krylov cycles: the true residual b - A x of every cycle
                           (Sec. 3.3) and the step's right-hand side (no counterpart in the
                           paper): LLG_CHAIN_FP64 = FP64; LLG_CHAIN_F32X2 = FP32-pair arithmetic
                           (sums by two-sum, products by Dekker's exact product; about 47
                           significant bits, errors a few 2^-48 of the operands' magnitudes),
                           which runs the FFTs on the FP32 pipes.  FP64 inputs and outputs
                           either way.  Grids with an axis length outside 64..1024 run FP64. */
} llg_opts;

typedef struct {
    int iters;                    /* Arnoldi steps (all cycles, all Picard iterations) */
    int restarts;                 /* GMRES cycles */
    int picard_iters;             /* linear solves in a midpoint step */
    int applies;                  /* FFT--HSS applications (fused operator counts one) */
    double rel_res_true;          /* final ||b - A x|| / ||b|| (worst over Picard solves) */
    double max_len_drift;         /* steps: max_i | |m^{n+1}_i| - |m^n_i| | */
    double energy_before, energy_after;   /* diagnostics: volume-averaged exchange + Zeeman energy */
    double dissipation_residual;  /* g(m^{n+1}) - g(m^n) + alpha k/(1+alpha^2) ||v||_N^2 (volume avg) */
    int status;                   /* llg_status of the call */
} llg_info;

/* Create a context for one grid; cuda_stream is a cudaStream_t (NULL = legacy default stream).
   Allocates twiddle/symbol tables and spectral scratch on the current device, and 64 bytes
   of host-mapped memory in which the Arnoldi kernels publish a GMRES cycle's progress, so
   that the host can follow the cycle without synchronising the stream.  Where mapped memory
   cannot be had, or when the environment variable LLG_HOST_POLL is "1" at creation, the
   host instead synchronises every fourth Arnoldi step; results are identical either way.
   Errors: INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA. */
llg_status llg_create(const llg_grid *grid, void *cuda_stream, llg_ctx **out);
/* Free every device and host resource of the context (synchronises its stream). */
llg_status llg_destroy(llg_ctx *ctx);
/* Text of the last error on this context (never NULL; empty after success). */
const char *llg_last_error(const llg_ctx *ctx);
/* Re-target the context at another stream of the same device. */
llg_status llg_set_stream(llg_ctx *ctx, void *cuda_stream);
/* Number of kernels this context has launched so far (for launch accounting). */
long long llg_launch_count(const llg_ctx *ctx);
/* Nodes of the context's grid. */
long long llg_nodes(const llg_ctx *ctx);

/* Saddle matvec y = A x, or y = A^T x when transpose != 0 (Sec. 2.4 eq. "saddle point
   system"; Sec. 3.2: the forward action uses the Fourier symbol without inversion plus the
   nodal formulas of eqs. (S), (Lambda)).  m: 3 planes; x, y: 4 planes; FP64. */
llg_status llg_saddle_apply(llg_ctx *ctx, const llg_params *prm, const double *m, const double *x,
                            double *y, int transpose);
/* The same matvec with its Fourier chain in FP32-pair arithmetic (llg_opts.chain_arith =
   LLG_CHAIN_F32X2; no counterpart in the paper): FP64 inputs and outputs, same layout, errors a
   few 2^-48 of the operands' magnitudes per operation instead of 2^-53.  Returns
   LLG_ERR_UNSUPPORTED_SIZE when an axis length is outside 64..1024. */
llg_status llg_saddle_apply_f32x2(llg_ctx *ctx, const llg_params *prm, const double *m, const double *x,
                                  double *y, int transpose);

/* FFT--HSS preconditioner z = M^{-1} p with M = (H + lambda I)(S + lambda I) (Sec. 3.2):
   Algorithm 1 (Fourier solve of the shifted exchange block, multiplier / lambda) followed by
   the closed-form 4x4 nodal inverse, eq. (inverse S).  transpose != 0 applies
   M^{-T} = (H + lambda I)^{-1} (S + lambda I)^{-T}.  FP64. */
llg_status llg_ffthss_apply(llg_ctx *ctx, const llg_params *prm, const double *m, const double *p,
                            double *z, int transpose);
/* The same in FP32 (m, p, z float planes). */
llg_status llg_ffthss_apply_f32(llg_ctx *ctx, const llg_params *prm, const float *m, const float *p,
                                float *z, int transpose);
/* Maximum spectral scratch of llg_ffthss_apply_noalloc, in complex FP64 slots (4 MiB):
   a grid fits when n1 * n2 * S <= this, with S = 1.5 n0 + 1 rounded up to a multiple of 16
   (for example 256 x 256 or 512 x 256 in 2D, 32^3 or 64 x 64 x 32 in 3D). */
#define LLG_NOALLOC_MAX_SPECTRAL 262144
/* The paper has no counterpart to this call: it is llg_ffthss_apply for callers that cannot
   allocate device memory and therefore cannot create a context -- a time-critical loop that
   has promised no allocation after start-up, an application whose device memory is fully
   reserved by another allocator (where an extra cudaMalloc fails or fragments), or a plug-in
   environment that may not create device allocations.  It calls no cudaMalloc, cudaFree or
   other allocating routine: its spectral scratch and tables live in one static device array
   (about 4.1 MiB) that every GPU loading the library holds until the process exits.
   Same operation, layout and precision as llg_ffthss_apply (FP64; transpose != 0 applies
   M^{-T}); m, p, z are caller-owned device pointers; cuda_stream is a cudaStream_t (NULL =
   legacy default stream).  Grids beyond LLG_NOALLOC_MAX_SPECTRAL return
   LLG_ERR_UNSUPPORTED_SIZE before any launch.  Every call fetches the array's device address
   for the current device (cudaGetSymbolAddress, which allocates nothing), so nothing stale
   survives a device reset; the first call on a device also loads the module there, so make
   that first call before any stream capture.  All calls share the array (each rewrites its tables and
   clears the scratch it uses), so calls that overlap on the GPU -- on other streams or host
   threads -- race on it and must be serialised by the caller. */
llg_status llg_ffthss_apply_noalloc(const llg_grid *grid, const llg_params *prm, const double *m,
                                    const double *p, double *z, int transpose, void *cuda_stream);
/* Left-preconditioned operator z = M^{-1} A x in one Fourier round trip, using
   (H + lambda I)^{-1} A = I + (H + lambda I)^{-1}(S - lambda I) (consequence of Sec. 3.2's
   splitting; the operator GMRES iterates on).  FP64. */
llg_status llg_precond_saddle_apply(llg_ctx *ctx, const llg_params *prm, const double *m,
                                    const double *x, double *z);

/* Solve A(m) x = b by FFT--HSS preconditioned GMRES(restart) (Sec. 3.2, Sec. 4.1).
   x: on entry the initial guess, on exit the solution.  Precision per opts->precision.
   Convergence is declared on the FP64 true residual.  Returns NOT_CONVERGED (x holds the
   last iterate) when max_iters is reached; DEGENERATE_NODE if some |m_i| = 0. */
llg_status llg_gmres_solve(llg_ctx *ctx, const llg_params *prm, const llg_opts *opts,
                           const double *m, const double *b, double *x, llg_info *info);

/* Projected implicit Euler tangent-plane step (Sec. 2.4 eq. "total system", Sec. 3.2):
   f = Chat Lap_N m^n + (1 + alpha^2) h_ext; solve with theta = 1 and blocks from m^n;
   m^{n+1}_i = (m^n_i + k v_i) / |m^n_i + k v_i|.  x_out receives (v | r). */
llg_status llg_step_euler(llg_ctx *ctx, const llg_params *prm, const llg_opts *opts,
                          const double *m_n, double *m_next, double *x_out, llg_info *info);

/* Crank--Nicolson-type midpoint step with Picard iteration (Sec. 3.3 eqs. "C-N", "hatm"):
   mhat^0 = m^n + (k/2) v_prev (v_prev may be NULL: zero); each Picard step solves the
   saddle system with theta = 1/2 and blocks from mhat^p; mhat^{p+1} = m^n + (k/2) v^p;
   m^{n+1} = m^n + k v.  x_out receives (v^{n+1/2} | r) and also serves as the warm start. */
llg_status llg_step_midpoint(llg_ctx *ctx, const llg_params *prm, const llg_opts *opts,
                             const double *m_n, const double *v_prev, double *m_next,
                             double *x_out, llg_info *info);

/* Adjoint of one converged midpoint step (derived from Sec. 3.3 eqs. "C-N", "hatm"; the paper
   has no adjoint): with R(v, r; m^n, alpha, h) = 0 the step's residual and J its Jacobian in
   (v, r), solves J^T y = (k mbar_next, 0) by GMRES preconditioned with M(mhat)^{-T}, then
   mbar_n = mbar_next - (dR/dm^n)^T y, *dalpha -= y^T dR/dalpha, dh[c] -= y^T dR/dh_c.
   m_n: 3 planes; x: the step's (v | r) (4 planes); mbar_next, mbar_n: 3 planes (device).
   dalpha, dh: HOST pointers, accumulated (+=).  The applied field is h_ext plus the optional
   per-node prm->h_field (the same field the forward step used): both enter dR_v/dalpha through
   -2 alpha (h_ext + h_field_j); dh is the gradient with respect to the uniform h_ext.  Demag
   and anisotropy are refused (INVALID_ARG).  FP64. */
llg_status llg_adjoint_step(llg_ctx *ctx, const llg_params *prm, const llg_opts *opts,
                            const double *m_n, const double *x, const double *mbar_next,
                            double *mbar_n, double *dalpha, double dh[3], llg_info *info);

/* Volume-averaged energy g_N(m) = (1/N_g) sum_j [c_ex/2 m.(-Lap_N m) - h_j.m
   + k_an (1 - (e_an.m)^2) - 1/2 m.h_dem] with h_j = h_ext + h_field_j (Sec. 2.1; the
   quadratic-affine energy of Prop. "nodal constraint and energy law").
   *out is a HOST pointer; synchronises the stream. */
llg_status llg_energy(llg_ctx *ctx, const llg_params *prm, const double *m, double *out);
/* Lower-order field h_low(m) = h_ext + h_field + 2 k_an (e_an.m) e_an + h_dem(m) (Sec. 2.1,
   2.2): the field the steppers add to the exchange term.  m, h: DEVICE, 3 FP64 planes,
   caller-owned, no aliasing.  Asynchronous on the context stream. */
llg_status llg_lower_order_field(llg_ctx *ctx, const llg_params *prm, const double *m, double *h);

/* ---------------------------------------------------------------- ensembles
   Many independent 2D problems advanced together by projected-Euler steps (Sec. 2.4, 3.2)
   in ONE persistent cooperative kernel launch, captured in a CUDA graph when the stream
   allows capture (a batched mode of this library; the paper solves one problem at a time).  Every
   problem has its own grid, damping, time step and field; all advance through the same
   phases in lockstep (right-hand side; flexible GMRES(restart) with the FP32 FFT--HSS
   application and inner matvec, FP64 Arnoldi and least squares; FP64 true residual; the
   Euler update) with per-problem convergence flags, so converged problems idle. */
typedef struct {
    int n[2];          /* grid n0 x n1, each 128, 256 or 512 */
    double L[2];       /* cell lengths */
    llg_params prm;    /* alpha, c_ex, k, lambda, h_ext, exchange (theta is 1: Euler) */
    double *m;         /* device, 3 planes: m^0 on entry, m after the steps on return */
    double *x;         /* device, 4 planes: on return (v | r) of the last step */
} llg_problem;
typedef struct llg_ensemble llg_ensemble;
/* Allocate the per-problem workspace (Krylov bases, spectra) and descriptors.  opts: restart
   (1..31), max_iters per solve, rtol (FP64 true residual); precision is always FP32-flexible,
   and the Gram--Schmidt passes are always FP64 (gs_arith is ignored: in this kernel's
   64-register budget the FP32-pair passes spill and ran slower).
   cuda_stream: a cudaStream_t (a non-default stream allows graph capture). */
llg_status llg_ensemble_create(const llg_problem *probs, int count, const llg_opts *opts, void *cuda_stream,
                               llg_ensemble **out);
/* Run `steps` Euler steps of every problem in one launch (synchronises).  infos (HOST, count
   entries, caller order, may be NULL): iterations and cycles summed over the steps, worst
   final relative residual, worst status.  used_graph (HOST, may be NULL): 1 if the launch ran
   as a captured CUDA graph. */
llg_status llg_ensemble_run(llg_ensemble *ens, int steps, llg_info *infos, int *used_graph);
/* Number of persistent blocks (must not exceed llg_ensemble_max_blocks, the co-resident limit). */
llg_status llg_ensemble_set_blocks(llg_ensemble *ens, int blocks);
int llg_ensemble_max_blocks(const llg_ensemble *ens);
/* Pick the persistent block count by timing one step for each multiple of the SM count up to
   the co-resident limit (problems' m restored afterwards); *blocks (HOST) receives the choice. */
llg_status llg_ensemble_autotune(llg_ensemble *ens, int *blocks);
/* Diagnostics of the persistent kernel's grid barrier (no counterpart in the paper).  Every
   barrier wait gives up after budget_cycles SM clock cycles (0: the default, about 2 s), sets an
   error flag and returns; all blocks then leave the kernel and llg_ensemble_run returns
   LLG_ERR_TIMEOUT with the barrier's source line in llg_ensemble_last_error.  hold_block >= 0
   makes that block withhold its arrival at the first barrier and return (-1: none), so the
   others' waits run out: this exercises the timeout path without any unbounded wait.  The
   ensemble stays usable after a timeout (restore budget 0, hold -1 and run again).
   INVALID_ARG for budget_cycles < 0 or hold_block < -1. */
llg_status llg_ensemble_set_barrier_test(llg_ensemble *ens, long long budget_cycles, int hold_block);
llg_status llg_ensemble_destroy(llg_ensemble *ens);
const char *llg_ensemble_last_error(const llg_ensemble *ens);

/* Pass plan of this context's 3D FP32 Fourier round trips (Algorithm 1's transforms and the
   inner matvec of flexible GMRES; no counterpart in the paper).  LLG_PLAN_FIVE: x, y, z
   (with the multiplier), y, x passes over HBM, 35 words per node for an FFT--HSS
   application (the default).  LLG_PLAN_CLUSTER: the x and y transforms of each z-plane run
   in one thread-block cluster that keeps the plane in its CTAs' shared memory (distributed
   shared memory between them), so the spectrum crosses HBM only around the z pass, 23
   words per node.  The cluster plan is compiled for 128 x 128 and 256 x 256 planes and the
   FFT--HSS application (FP64 or FP32 input) and FP32 matvec; other grids and operators run
   the five-pass plan either way.  Results agree to FP32 rounding.  INVALID_ARG for an
   unknown plan. */
llg_status llg_set_pass_plan(llg_ctx *ctx, int plan);

/* Autotune the launch shapes of the Fourier axis passes for this context's grid (no
   counterpart in the paper): every compiled shape (register kernel with 4/8/16-column
   tiles; shared-memory-staged FP32 kernel with several tile/sub-batch sizes) is run on a
   deterministic spectrum, its result checked against the default shape (candidates that
   disagree beyond 1e-4 FP32 / 1e-11 FP64 relative are rejected), timed with CUDA events
   (median of seven runs), and the fastest kept for each pass, a later candidate replacing an
   earlier one only when at least 3% faster.  precision_mask: 1 = FP64 passes, 2 = FP32 passes, 3 = both.
   report (HOST, may be NULL): text of the timings and choices.  Allocates and frees scratch;
   synchronises the stream.  Without this call the default shapes are used. */
llg_status llg_autotune(llg_ctx *ctx, int precision_mask, char *report, int report_len);

/* Set one axis pass's launch shape by hand, as llg_autotune would (no counterpart in the
   paper; lets a profiler run replay the shapes a live run picked).  fp32: 1 = FP32 passes,
   0 = FP64; slot: 0 = y pass of 2D grids, 1 = y forward, 2 = z (with the multiplier),
   3 = y inverse (3D); kind: 0 = register kernel (E points per thread, TW columns), 1 = staged
   tile (TW columns, CB per sub-batch), 3 = two columns per thread (TW), 4 = TMA-fed persistent
   kernel (TW).  LLG_ERR_INVALID_ARG when the grid has no such pass or the shape is not one the
   tuner would try for its line length.  Other passes keep their shapes (defaults if none). */
llg_status llg_set_axis_shape(llg_ctx *ctx, int fp32, int slot, int kind, int E, int TW, int CB);

/* ---------------------------------------------------------------- measurement support
   (infrastructure for the benchmark; no counterpart in the paper) */

/* kernel classes that can be timed live */
enum {
    LLG_KCLASS_NONE = 0,
    LLG_KCLASS_XFWD = 1,     /* forward x-axis pass with the nodal prologue */
    LLG_KCLASS_AXIS = 2,     /* y/z axis passes (with the Fourier multiplier on the last axis) */
    LLG_KCLASS_XINV = 3,     /* inverse x-axis pass with the nodal epilogue */
    LLG_KCLASS_ARNOLDI = 4   /* Gram--Schmidt passes over the Krylov basis */
};
/* Start timing every launch of one kernel class on this context: a CUDA event pair is
   recorded on the context's stream around each launch (around the three passes of an
   Arnoldi step for that class, counted as three launches), together with the launch's
   algorithmic bytes and flops (inputs read + outputs written once; 5 n log2 n flops per
   complex length-n transform; 2 per multiply-add).  Launches of an Arnoldi step that the
   device-side stopping flag turned into no-ops are discarded. */
llg_status llg_profile_begin(llg_ctx *ctx, int kernel_class);
/* Stop timing, synchronise the stream and return the totals (HOST pointers, any may be NULL). */
llg_status llg_profile_end(llg_ctx *ctx, double *total_ms, long long *launches, double *bytes, double *flops);
/* Orthogonality of the Krylov basis of the context's last GMRES cycle (no counterpart in the
   paper; a measurement of the Gram--Schmidt passes): *max_dev = max_{i,k} |delta_ik -
   v_i . v_k| over the normalised stored vectors v_i = V_i / ||V_i||, each dot product in FP64;
   *nvec the number of vectors compared (HOST pointers).  In a flexible solve the first stored
   vector holds the final true residual once the solve has returned, so the comparison starts
   at the second.  Synchronises the stream; allocates nvec^2 doubles.
   Errors: INVALID_ARG (null pointer, no solve yet), OOM/CUDA. */
llg_status llg_krylov_orthogonality(llg_ctx *ctx, double *max_dev, int *nvec);
/* Measure the device's multiply-add rate with a register-resident FMA loop on the context's
   stream (fp64 != 0: double, else float); *tflops receives 2 * FMAs / s / 1e12 (HOST). */
llg_status llg_probe_fma_rate(llg_ctx *ctx, int fp64, double *tflops);
/* Self-check with no counterpart in the paper.  The mixed-precision path converts between
   float and double with integer operations instead of the hardware conversions (which run
   at the FP64 multiply-add rate on this part) and relies on both giving the same bits.
   This compares them on the device: float -> double on all 2^32 float bit patterns, double
   -> float (round to nearest even) on n_doubles hashed patterns, a quarter each arbitrary,
   in and around the float exponent range, on or beside a rounding tie, and at ties in the
   float subnormal range.  The mismatch counts (NaN against NaN matches) go to the HOST
   pointers.  Runs on the context's stream and synchronises it; allocates 16 bytes.
   Errors: INVALID_ARG (null pointer, n_doubles < 0), OOM/CUDA. */
llg_status llg_check_conversions(llg_ctx *ctx, long long n_doubles, long long *f2d_mismatches,
                                 long long *d2f_mismatches);

#ifdef __cplusplus
}
#endif
#endif
