/*
 * llg_oracle.h -- plain, slow FP64 CPU oracle for the periodic tangent-plane
 * LLG saddle system and its FFT--HSS preconditioned GMRES solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this code; only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no source with the CUDA
 * library (its own grid, symbol, transform and solver code, written from the
 * paper's equations).
 *
 * Conventions (all arrays are caller-owned host double arrays):
 *   grid nodes N_g = n[0]*n[1]*n[2] (n[l] = 1 for l >= dim), node index
 *   j = ix + n0*(iy + n1*iz).  Fields are SoA planes: m = (m1|m2|m3),
 *   x = (v1|v2|v3|r), each plane N_g long.
 *   Saddle matrix (Sec. 2.4, eq. "saddle point system", with the second block
 *   row negated as the paper does):
 *     y_v = alpha v + theta k Chat (-Lap_N) v + m x v + m r
 *     y_r = -(m . v)
 *   Chat = (1 + alpha^2) c_ex  (Sec. 2.4: normalised exchange coefficient).
 */
#ifndef LLG_ORACLE_H
#define LLG_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;        /* 2 or 3 */
    int n[3];       /* points per axis; n[l] = 1 for l >= dim */
    double L[3];    /* periodic cell lengths */
} orc_grid;

enum { ORC_EX_SPECTRAL = 0, ORC_EX_FD2 = 1 };
enum { ORC_TR_DFT = 0, ORC_TR_FFT = 1 };

typedef struct {
    double alpha;   /* Gilbert damping */
    double c_ex;    /* normalised exchange coefficient (paper: one) */
    double k;       /* time step */
    double theta;   /* 1 Euler, 1/2 midpoint */
    double lambda;  /* HSS shift */
    double h[3];    /* uniform applied field */
    int exchange;   /* ORC_EX_SPECTRAL or ORC_EX_FD2 */
    double k_an;    /* anisotropy energy k_an (1 - (e.m)^2), 0 = off */
    double e_an[3]; /* easy axis */
    int demag;      /* 1 = periodic zero-mean demagnetising field */
    const double *h_field; /* optional nodal applied field (3 planes), added to h; NULL = none */
} orc_params;

typedef struct {
    int restart;      /* GMRES restart length */
    int max_iters;    /* cap on total Arnoldi steps */
    double rtol;      /* relative tolerance */
    int picard_max;   /* midpoint Picard cap */
    double picard_tol;/* midpoint Picard relative tolerance */
    int use_dense;    /* 1: solve each linear system by dense LU instead of GMRES */
    int precond;      /* GMRES left preconditioner: ORC_PC_FFTHSS (default), _HERMITIAN, _NONE */
} orc_opts;

/* the split FFT--HSS preconditioner (lambda I + S)^{-1} (lambda I + H)^{-1}; the shifted
   symmetric part (lambda I + H)^{-1} alone; no preconditioner (Sec. 4.3 comparison) */
enum { ORC_PC_FFTHSS = 0, ORC_PC_HERMITIAN = 1, ORC_PC_NONE = 2 };

typedef struct {
    int iters, restarts, picard_iters, converged;
    double rel_res_true, rel_res_prec;
} orc_info;

/* transform selection: naive separable DFT (default) or textbook radix-2 FFT */
void orc_set_transform(int mode);

/* wavenumber integer of index i on an axis of length n; symbol sigma of -Lap_N */
int orc_wavenumber(int n, int i);
double orc_symbol(const orc_grid *g, int exchange, const int kvec[3]);

/* complex transform of all axes in place; sign -1 forward (unnormalised), +1 inverse (unnormalised) */
void orc_transform(const orc_grid *g, double *re, double *im, int sign);

/* w = (-Lap_N) u for one real plane */
void orc_neg_laplacian(const orc_grid *g, int exchange, const double *u, double *w);

/* Alg. 1: (H + lambda I)^{-1} p, p = (v|r) four planes */
void orc_hermitian_solve(const orc_grid *g, const orc_params *p, const double *pin, double *w);
/* (S + lambda I)^{-1} w per node by 4x4 Gaussian elimination; transpose != 0 solves (S + lambda I)^T */
void orc_nodal_solve(const orc_grid *g, const orc_params *p, const double *m, const double *w,
                     double *z, int transpose);
/* FFT--HSS preconditioner M^{-1} = (S+lambda)^{-1}(H+lambda)^{-1}; transpose: M^{-T} */
void orc_ffthss_apply(const orc_grid *g, const orc_params *p, const double *m, const double *pin,
                      double *z, int transpose);
/* saddle matvec y = A x (transpose != 0: y = A^T x) */
void orc_saddle_apply(const orc_grid *g, const orc_params *p, const double *m, const double *x,
                      double *y, int transpose);

/* dense assembly of A (4Ng x 4Ng, row-major) and dense LU solve */
void orc_saddle_dense(const orc_grid *g, const orc_params *p, const double *m, double *A);
int orc_dense_solve(int n, const double *A, const double *b, double *x);

/* left-preconditioned restarted GMRES on A x = b (x: in x0, out solution) */
int orc_gmres_solve(const orc_grid *g, const orc_params *p, const orc_opts *o, const double *m,
                    const double *b, double *x, int transpose, orc_info *info,
                    double *res_hist, int hist_len);

/* lower-order field h_low(m) = h + h_ani(m) + h_dem(m), three planes */
void orc_h_low(const orc_grid *g, const orc_params *p, const double *m, double *hl);
/* volume-averaged energy g_N(m) */
double orc_energy(const orc_grid *g, const orc_params *p, const double *m);

/* projected implicit Euler step (Sec. 2.4 / 3.2): theta forced to 1 */
int orc_step_euler(const orc_grid *g, const orc_params *p, const orc_opts *o, const double *m_n,
                   double *m_next, double *x_out, orc_info *info);
/* midpoint step with Picard iteration (Sec. 3.3): theta forced to 1/2.
   v_prev may be NULL (v^{-1/2} = 0).  x_out = (v^{n+1/2} | r). */
int orc_step_midpoint(const orc_grid *g, const orc_params *p, const orc_opts *o, const double *m_n,
                      const double *v_prev, double *m_next, double *x_out, orc_info *info);

/* adjoint of one converged midpoint step: given m_n, the step's (v, r), and
   mbar_next = dL/dm^{n+1}, return mbar_n = dL/dm^n and accumulate dL/dalpha, dL/dh. */
int orc_adjoint_midpoint(const orc_grid *g, const orc_params *p, const orc_opts *o,
                         const double *m_n, const double *x, const double *mbar_next,
                         double *mbar_n, double *dalpha, double dh[3], orc_info *info);

/* closed forms of Sec. 3.4 */
double orc_beta_N(const orc_grid *g, const orc_params *p);
double orc_q_bar(double lambda, double alpha, double beta);
double orc_lambda_bd(double alpha, double beta);
double orc_gamma_m(double lambda, double m_min, double m_max);
double orc_theta2(double q, double gamma);
double orc_kappa(double lambda, double m_min, double m_max);
int orc_iteration_bound(double kappa, double theta, double eps);

#ifdef __cplusplus
}
#endif
#endif
