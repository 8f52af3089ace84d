/*
 * llg_oracle.c -- plain FP64 CPU oracle (test infrastructure only).
 *
 * Every function follows the paper's statement of the method directly, with
 * no blocking, fusion or reordering:
 *   - grid, discrete Laplacian symbol ........ Sec. 2.3 ("Periodic spectral discretization")
 *   - saddle matrix and nodal blocks ......... Sec. 2.4 eqs. (total system 2), (saddle point system), (Bi);
 *                                              Sec. 3.1 eqs. (HS), (S), (Lambda)
 *   - (H + lambda I)^{-1} .................... Sec. 3.2, Algorithm 1
 *   - (S + lambda I)^{-1} .................... Sec. 3.1/3.2: one 4x4 solve per node, done here by
 *                                              Gaussian elimination (not the closed form of eq.
 *                                              (inverse S), which the tests use as an independent pin)
 *   - left preconditioner M^{-1} ............. Sec. 3.2 (H-solve first, then the nodal solve)
 *   - restarted GMRES ........................ Sec. 3.2 and Sec. 4.1 (textbook MGS + Givens)
 *   - projected Euler step ................... Sec. 2.4 eq. (total system), Sec. 3.2 (update + normalise)
 *   - midpoint step + Picard ................. Sec. 3.3 eqs. (C-N), (hatm)
 *   - energy, lower-order field .............. Sec. 2.1 eq. (heff), Sec. 2.2 eq. (hdem)
 *   - closed-form bounds ..................... Sec. 3.4 Prop. (reduced HSS), Cor. (Fourier enclosure),
 *                                              Thm. (full saddle GMRES), Cor. (uniform bound)
 * The adjoint of a converged midpoint step is derived from eqs. (C-N)/(hatm)
 * by the implicit function theorem; it has no counterpart in the paper.
 *
 * Built with -O2 -ffp-contract=off so that every product is rounded separately.
 */
#include "llg_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double TWO_PI = 6.283185307179586476925286766559;
static int g_transform_mode = ORC_TR_DFT;

void orc_set_transform(int mode) { g_transform_mode = mode; }

static long nodes_of(const orc_grid *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static double dot(long n, const double *a, const double *b) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}
static double nrm2(long n, const double *a) { return sqrt(dot(n, a, a)); }

/* ---------------------------------------------------------------- grid (Sec. 2.3) */

/* integer wavenumber: 0..n/2-1, then -n/2..-1 (the Nyquist index n/2 maps to -n/2) */
int orc_wavenumber(int n, int i) { return (i < n / 2) ? i : i - n; }

/* symbol of -Lap_N: spectral |xi|^2 with xi_l = 2 pi k_l / L_l, or the
   second-order central-difference symbol sum_l (4/h_l^2) sin^2(pi k_l / n_l) */
double orc_symbol(const orc_grid *g, int exchange, const int kvec[3]) {
    double s = 0.0;
    for (int l = 0; l < g->dim; ++l) {
        if (exchange == ORC_EX_FD2) {
            double h = g->L[l] / g->n[l];
            double sn = sin(M_PI * (double)kvec[l] / (double)g->n[l]);
            s += 4.0 / (h * h) * sn * sn;
        } else {
            double xi = TWO_PI * (double)kvec[l] / g->L[l];
            s += xi * xi;
        }
    }
    return s;
}

/* ---------------------------------------------------------------- transforms */

/* naive DFT of one line: out[q] = sum_j in[j] exp(sign 2 pi i j q / n) */
static void dft_line(int n, const double *ire, const double *iim, double *ore, double *oim,
                     int sign, const double *ct, const double *st) {
    for (int q = 0; q < n; ++q) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
            long t = ((long)j * q) % n;
            double c = ct[t], s = sign * st[t];
            sr += ire[j] * c - iim[j] * s;
            si += ire[j] * s + iim[j] * c;
        }
        ore[q] = sr;
        oim[q] = si;
    }
}

/* textbook iterative radix-2 Cooley--Tukey (n a power of two), in place */
static void fft_line(int n, double *re, double *im, int sign, const double *ct, const double *st) {
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int step = n / len;
        for (int i = 0; i < n; i += len) {
            for (int j = 0; j < len / 2; ++j) {
                double c = ct[j * step], s = sign * st[j * step];
                double ur = re[i + j], ui = im[i + j];
                double xr = re[i + j + len / 2], xi = im[i + j + len / 2];
                double vr = xr * c - xi * s, vi = xr * s + xi * c;
                re[i + j] = ur + vr; im[i + j] = ui + vi;
                re[i + j + len / 2] = ur - vr; im[i + j + len / 2] = ui - vi;
            }
        }
    }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

void orc_transform(const orc_grid *g, double *re, double *im, int sign) {
    int n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    int nmax = n0 > n1 ? n0 : n1;
    if (n2 > nmax) nmax = n2;
    double *lr = malloc(sizeof(double) * nmax * 4);
    double *li = lr + nmax, *or_ = li + nmax, *oi = or_ + nmax;
    double *ct = malloc(sizeof(double) * nmax * 2), *st = ct + nmax;
    for (int axis = 0; axis < g->dim; ++axis) {
        int n = g->n[axis];
        if (n == 1) continue;
        for (int t = 0; t < n; ++t) { ct[t] = cos(TWO_PI * t / n); st[t] = sin(TWO_PI * t / n); }
        long stride = axis == 0 ? 1 : (axis == 1 ? n0 : (long)n0 * n1);
        /* enumerate line starts: all nodes whose coordinate along axis is 0 */
        for (int i2 = 0; i2 < (axis == 2 ? 1 : n2); ++i2)
            for (int i1 = 0; i1 < (axis == 1 ? 1 : n1); ++i1)
                for (int i0 = 0; i0 < (axis == 0 ? 1 : n0); ++i0) {
                    long base = i0 + (long)n0 * (i1 + (long)n1 * i2);
                    for (int j = 0; j < n; ++j) { lr[j] = re[base + j * stride]; li[j] = im[base + j * stride]; }
                    if (g_transform_mode == ORC_TR_FFT && is_pow2(n)) {
                        fft_line(n, lr, li, sign, ct, st);
                        memcpy(or_, lr, sizeof(double) * n);
                        memcpy(oi, li, sizeof(double) * n);
                    } else {
                        dft_line(n, lr, li, or_, oi, sign, ct, st);
                    }
                    for (int j = 0; j < n; ++j) { re[base + j * stride] = or_[j]; im[base + j * stride] = oi[j]; }
                }
    }
    free(lr);
    free(ct);
}

static void mode_of(const orc_grid *g, long j, int kvec[3]) {
    int i0 = (int)(j % g->n[0]);
    int i1 = (int)((j / g->n[0]) % g->n[1]);
    int i2 = (int)(j / ((long)g->n[0] * g->n[1]));
    kvec[0] = orc_wavenumber(g->n[0], i0);
    kvec[1] = g->dim > 1 ? orc_wavenumber(g->n[1], i1) : 0;
    kvec[2] = g->dim > 2 ? orc_wavenumber(g->n[2], i2) : 0;
}

/* w = F^{-1}[ s(xi) F[u] ] for a real plane, s = a + b sigma(xi) or 1/(a + b sigma(xi)) */
static void fourier_apply(const orc_grid *g, int exchange, const double *u, double *w,
                          double a, double b, int invert) {
    long N = nodes_of(g);
    double *re = malloc(sizeof(double) * N * 2), *im = re + N;
    for (long j = 0; j < N; ++j) { re[j] = u[j]; im[j] = 0.0; }
    orc_transform(g, re, im, -1);
    for (long j = 0; j < N; ++j) {
        int kv[3];
        mode_of(g, j, kv);
        double s = a + b * orc_symbol(g, exchange, kv);
        if (invert) s = 1.0 / s;
        re[j] *= s;
        im[j] *= s;
    }
    orc_transform(g, re, im, +1);
    for (long j = 0; j < N; ++j) w[j] = re[j] / (double)N;
    free(re);
}

void orc_neg_laplacian(const orc_grid *g, int exchange, const double *u, double *w) {
    fourier_apply(g, exchange, u, w, 0.0, 1.0, 0);
}

/* ---------------------------------------------------------------- operators */

static double chat_of(const orc_params *p) { return (1.0 + p->alpha * p->alpha) * p->c_ex; }

/* Algorithm 1: q3 = iFFT(FFT(v) / (alpha + theta k Chat |xi|^2 + lambda)), q4 = r / lambda */
void orc_hermitian_solve(const orc_grid *g, const orc_params *p, const double *pin, double *w) {
    long N = nodes_of(g);
    double a = p->alpha + p->lambda, b = p->theta * p->k * chat_of(p);
    for (int c = 0; c < 3; ++c) fourier_apply(g, p->exchange, pin + c * N, w + c * N, a, b, 1);
    for (long j = 0; j < N; ++j) w[3 * N + j] = pin[3 * N + j] / p->lambda;
}

/* (S~_i + lambda I) with S~_i = [[Lambda_i, m_i], [-m_i^T, 0]], Lambda_i v = m_i x v (eqs. (S), (Lambda)) */
static void nodal_matrix(double m1, double m2, double m3, double lam, double M[4][4]) {
    double T[4][4] = {
        { lam, -m3,  m2,  m1 },
        {  m3, lam, -m1,  m2 },
        { -m2,  m1, lam,  m3 },
        { -m1, -m2, -m3, lam },
    };
    memcpy(M, T, sizeof(T));
}

/* Gaussian elimination with partial pivoting on a small dense system */
static int ge_solve(int n, double *A, double *b) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

void orc_nodal_solve(const orc_grid *g, const orc_params *p, const double *m, const double *w,
                     double *z, int transpose) {
    long N = nodes_of(g);
    for (long j = 0; j < N; ++j) {
        double M[4][4], A[16], b[4];
        nodal_matrix(m[j], m[N + j], m[2 * N + j], p->lambda, M);
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) A[r * 4 + c] = transpose ? M[c][r] : M[r][c];
        for (int r = 0; r < 4; ++r) b[r] = w[r * N + j];
        ge_solve(4, A, b);
        for (int r = 0; r < 4; ++r) z[r * N + j] = b[r];
    }
}

/* M^{-1} = (S + lambda I)^{-1} (H + lambda I)^{-1}; M^{-T} = (H + lambda I)^{-1} (S + lambda I)^{-T} */
void orc_ffthss_apply(const orc_grid *g, const orc_params *p, const double *m, const double *pin,
                      double *z, int transpose) {
    long N = nodes_of(g);
    double *w = malloc(sizeof(double) * 4 * N);
    if (!transpose) {
        orc_hermitian_solve(g, p, pin, w);
        orc_nodal_solve(g, p, m, w, z, 0);
    } else {
        orc_nodal_solve(g, p, m, pin, w, 1);
        orc_hermitian_solve(g, p, w, z);
    }
    free(w);
}

/* y = A x with A = [[H + S, B^T], [-B, 0]]; A^T = [[H - S, -B^T], [B, 0]] */
void orc_saddle_apply(const orc_grid *g, const orc_params *p, const double *m, const double *x,
                      double *y, int transpose) {
    long N = nodes_of(g);
    double b = p->theta * p->k * chat_of(p);
    for (int c = 0; c < 3; ++c) fourier_apply(g, p->exchange, x + c * N, y + c * N, p->alpha, b, 0);
    double sgn = transpose ? -1.0 : 1.0;
    for (long j = 0; j < N; ++j) {
        double m1 = m[j], m2 = m[N + j], m3 = m[2 * N + j];
        double v1 = x[j], v2 = x[N + j], v3 = x[2 * N + j], r = x[3 * N + j];
        /* m x v */
        double c1 = m2 * v3 - m3 * v2, c2 = m3 * v1 - m1 * v3, c3 = m1 * v2 - m2 * v1;
        y[j] += sgn * (c1 + m1 * r);
        y[N + j] += sgn * (c2 + m2 * r);
        y[2 * N + j] += sgn * (c3 + m3 * r);
        y[3 * N + j] = -sgn * (m1 * v1 + m2 * v2 + m3 * v3);
    }
}

typedef void (*orc_op)(void *ctx, const double *x, double *y);

static void assemble_dense(long n, orc_op op, void *ctx, double *A) {
    double *e = calloc((size_t)n, sizeof(double)), *col = malloc(sizeof(double) * n);
    for (long c = 0; c < n; ++c) {
        e[c] = 1.0;
        op(ctx, e, col);
        e[c] = 0.0;
        for (long r = 0; r < n; ++r) A[r * n + c] = col[r];
    }
    free(e);
    free(col);
}

typedef struct { const orc_grid *g; const orc_params *p; const double *m; int transpose; } saddle_ctx;
static void saddle_op(void *c, const double *x, double *y) {
    saddle_ctx *s = c;
    orc_saddle_apply(s->g, s->p, s->m, x, y, s->transpose);
}
static void saddle_prec(void *c, const double *x, double *y) {
    saddle_ctx *s = c;
    orc_ffthss_apply(s->g, s->p, s->m, x, y, s->transpose);
}
/* (lambda I + H)^{-1}: H = diag(alpha + theta k Chat (-Lap), 0) is symmetric, so also its transpose */
static void hermitian_prec(void *c, const double *x, double *y) {
    saddle_ctx *s = c;
    orc_hermitian_solve(s->g, s->p, x, y);
}
static void identity_prec(void *c, const double *x, double *y) {
    saddle_ctx *s = c;
    memcpy(y, x, sizeof(double) * 4 * nodes_of(s->g));
}

void orc_saddle_dense(const orc_grid *g, const orc_params *p, const double *m, double *A) {
    saddle_ctx s = { g, p, m, 0 };
    assemble_dense(4 * nodes_of(g), saddle_op, &s, A);
}

int orc_dense_solve(int n, const double *A, const double *b, double *x) {
    double *C = malloc(sizeof(double) * (size_t)n * n);
    memcpy(C, A, sizeof(double) * (size_t)n * n);
    memcpy(x, b, sizeof(double) * n);
    int rc = ge_solve(n, C, x);
    free(C);
    return rc;
}

/* ---------------------------------------------------------------- GMRES */

/*
 * Restarted GMRES(restart) with left preconditioner Minv (Saad, Alg. 9.4):
 * modified Gram--Schmidt Arnoldi on Minv A, Givens rotations, x0 given.
 * A cycle stops early once the preconditioned residual estimate has fallen by
 * the factor the true residual still has to fall (with margin 0.5), or at the
 * restart length.  The solve is accepted only when the TRUE relative residual
 * ||b - A x|| / ||b|| <= rtol (computed before every cycle).
 */
static int gmres_core(long n, orc_op A, orc_op Minv, void *ctx, const double *b, double *x,
                      int restart, int max_iters, double rtol, orc_info *info, double *hist, int hist_len) {
    int m = restart;
    double nb = nrm2(n, b);
    orc_info inf = { 0, 0, 0, 0, 0.0, 0.0 };
    if (nb == 0.0) {
        memset(x, 0, sizeof(double) * n);
        inf.converged = 1;
        if (info) *info = inf;
        return 0;
    }
    double *V = malloc(sizeof(double) * (size_t)n * (m + 1));
    double *H = calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = malloc(sizeof(double) * m), *sn = malloc(sizeof(double) * m);
    double *gv = malloc(sizeof(double) * (m + 1)), *y = malloc(sizeof(double) * m);
    double *t = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
    double *mb = malloc(sizeof(double) * n);
    Minv(ctx, b, mb);
    double nmb = nrm2(n, mb);
    free(mb);
#define HH(i, j) H[(i) * m + (j)]
    for (;;) {
        A(ctx, x, t);
        for (long i = 0; i < n; ++i) t[i] = b[i] - t[i];
        double true_rel = nrm2(n, t) / nb;
        inf.rel_res_true = true_rel;
        if (true_rel <= rtol) { inf.converged = 1; break; }
        if (inf.iters >= max_iters) break;
        Minv(ctx, t, w);
        double beta = nrm2(n, w);
        if (beta == 0.0) break;
        double target = beta * (rtol / true_rel) * 0.5;
        for (long i = 0; i < n; ++i) V[i] = w[i] / beta;
        memset(gv, 0, sizeof(double) * (m + 1));
        gv[0] = beta;
        int jd = 0;
        for (int j = 0; j < m; ++j) {
            A(ctx, V + (size_t)j * n, t);
            Minv(ctx, t, w);
            for (int i = 0; i <= j; ++i) {
                double h = dot(n, w, V + (size_t)i * n);
                HH(i, j) = h;
                for (long q = 0; q < n; ++q) w[q] -= h * V[(size_t)i * n + q];
            }
            double hn = nrm2(n, w);
            HH(j + 1, j) = hn;
            if (hn != 0.0)
                for (long q = 0; q < n; ++q) V[(size_t)(j + 1) * n + q] = w[q] / hn;
            for (int i = 0; i < j; ++i) {
                double a = HH(i, j), c = HH(i + 1, j);
                HH(i, j) = cs[i] * a + sn[i] * c;
                HH(i + 1, j) = -sn[i] * a + cs[i] * c;
            }
            double a = HH(j, j), c = HH(j + 1, j), rr = hypot(a, c);
            cs[j] = a / rr;
            sn[j] = c / rr;
            HH(j, j) = rr;
            HH(j + 1, j) = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            inf.iters++;
            jd = j + 1;
            inf.rel_res_prec = fabs(gv[j + 1]) / nmb;
            if (hist && inf.iters - 1 < hist_len) hist[inf.iters - 1] = inf.rel_res_prec;
            if (fabs(gv[j + 1]) <= target || hn == 0.0 || inf.iters >= max_iters) break;
        }
        for (int i = jd - 1; i >= 0; --i) {
            double s = gv[i];
            for (int k = i + 1; k < jd; ++k) s -= HH(i, k) * y[k];
            y[i] = s / HH(i, i);
        }
        for (int i = 0; i < jd; ++i)
            for (long q = 0; q < n; ++q) x[q] += y[i] * V[(size_t)i * n + q];
        inf.restarts++;
    }
#undef HH
    free(V); free(H); free(cs); free(sn); free(gv); free(y); free(t); free(w);
    if (info) *info = inf;
    return inf.converged ? 0 : 1;
}

int orc_gmres_solve(const orc_grid *g, const orc_params *p, const orc_opts *o, const double *m,
                    const double *b, double *x, int transpose, orc_info *info,
                    double *res_hist, int hist_len) {
    saddle_ctx s = { g, p, m, transpose };
    long n = 4 * nodes_of(g);
    if (o->use_dense) {
        double *A = malloc(sizeof(double) * n * n);
        saddle_ctx s2 = { g, p, m, transpose };
        assemble_dense(n, saddle_op, &s2, A);
        int rc = orc_dense_solve((int)n, A, b, x);
        free(A);
        if (info) { memset(info, 0, sizeof(*info)); info->converged = rc == 0; }
        return rc == 0 ? 0 : 1;
    }
    orc_op prec = o->precond == ORC_PC_HERMITIAN ? hermitian_prec : (o->precond == ORC_PC_NONE ? identity_prec : saddle_prec);
    return gmres_core(n, saddle_op, prec, &s, b, x, o->restart, o->max_iters, o->rtol,
                      info, res_hist, hist_len);
}

/* ---------------------------------------------------------------- fields and energy (Sec. 2.1, 2.2) */

/* periodic zero-mean demagnetising field: h^(xi) = -xi'(xi'.m^)/|xi|^2, xi != 0,
   with xi' the first-derivative wavevector (Nyquist component set to zero) */
static void demag_field(const orc_grid *g, const double *m, double *hd) {
    long N = nodes_of(g);
    double *re = malloc(sizeof(double) * N * 6), *im = re + 3 * N;
    for (int c = 0; c < 3; ++c)
        for (long j = 0; j < N; ++j) { re[c * N + j] = m[c * N + j]; im[c * N + j] = 0.0; }
    for (int c = 0; c < 3; ++c) orc_transform(g, re + c * N, im + c * N, -1);
    for (long j = 0; j < N; ++j) {
        int kv[3];
        mode_of(g, j, kv);
        double xi[3] = { 0, 0, 0 }, xp[3] = { 0, 0, 0 };
        for (int l = 0; l < g->dim; ++l) {
            xi[l] = TWO_PI * kv[l] / g->L[l];
            xp[l] = (g->n[l] % 2 == 0 && kv[l] == -g->n[l] / 2) ? 0.0 : xi[l];
        }
        double s = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
        if (s == 0.0) {
            for (int c = 0; c < 3; ++c) { re[c * N + j] = 0.0; im[c * N + j] = 0.0; }
            continue;
        }
        double dr = xp[0] * re[j] + xp[1] * re[N + j] + xp[2] * re[2 * N + j];
        double di = xp[0] * im[j] + xp[1] * im[N + j] + xp[2] * im[2 * N + j];
        for (int c = 0; c < 3; ++c) {
            re[c * N + j] = -xp[c] * dr / s;
            im[c * N + j] = -xp[c] * di / s;
        }
    }
    for (int c = 0; c < 3; ++c) orc_transform(g, re + c * N, im + c * N, +1);
    for (int c = 0; c < 3; ++c)
        for (long j = 0; j < N; ++j) hd[c * N + j] = re[c * N + j] / (double)N;
    free(re);
}

void orc_h_low(const orc_grid *g, const orc_params *p, const double *m, double *hl) {
    long N = nodes_of(g);
    for (int c = 0; c < 3; ++c)
        for (long j = 0; j < N; ++j) hl[c * N + j] = p->h[c] + (p->h_field ? p->h_field[c * N + j] : 0.0);
    if (p->k_an != 0.0) {
        for (long j = 0; j < N; ++j) {
            double em = p->e_an[0] * m[j] + p->e_an[1] * m[N + j] + p->e_an[2] * m[2 * N + j];
            for (int c = 0; c < 3; ++c) hl[c * N + j] += 2.0 * p->k_an * p->e_an[c] * em;
        }
    }
    if (p->demag) {
        double *hd = malloc(sizeof(double) * 3 * N);
        demag_field(g, m, hd);
        for (long i = 0; i < 3 * N; ++i) hl[i] += hd[i];
        free(hd);
    }
}

/* g_N(m) = (1/N_g) sum_j [ c_ex/2 m.(-Lap m) - h_j.m + k_an (1 - (e.m)^2) - 1/2 m.h_dem ], h_j = h + h_field_j */
double orc_energy(const orc_grid *g, const orc_params *p, const double *m) {
    long N = nodes_of(g);
    double *lap = malloc(sizeof(double) * 3 * N);
    for (int c = 0; c < 3; ++c) orc_neg_laplacian(g, p->exchange, m + c * N, lap + c * N);
    double *hd = NULL;
    if (p->demag) {
        hd = malloc(sizeof(double) * 3 * N);
        demag_field(g, m, hd);
    }
    double e = 0.0;
    for (long j = 0; j < N; ++j) {
        double mj[3] = { m[j], m[N + j], m[2 * N + j] };
        double ej = 0.0;
        for (int c = 0; c < 3; ++c) {
            double hc = p->h[c] + (p->h_field ? p->h_field[c * N + j] : 0.0);
            ej += 0.5 * p->c_ex * mj[c] * lap[c * N + j] - hc * mj[c];
        }
        if (p->k_an != 0.0) {
            double em = p->e_an[0] * mj[0] + p->e_an[1] * mj[1] + p->e_an[2] * mj[2];
            ej += p->k_an * (1.0 - em * em);
        }
        if (hd)
            for (int c = 0; c < 3; ++c) ej -= 0.5 * mj[c] * hd[c * N + j];
        e += ej;
    }
    free(lap);
    free(hd);
    return e / (double)N;
}

/* ---------------------------------------------------------------- time steppers */

static int solve_system(const orc_grid *g, const orc_params *p, const orc_opts *o, const double *m,
                        const double *b, double *x, orc_info *inf) {
    return orc_gmres_solve(g, p, o, m, b, x, 0, inf, NULL, 0);
}

/* f = Chat Lap_N m + (1 + alpha^2) h_low(mfield) for the velocity block */
static void rhs_velocity(const orc_grid *g, const orc_params *p, const double *m_ex,
                         const double *m_low, double *f) {
    long N = nodes_of(g);
    double chat = chat_of(p), s = 1.0 + p->alpha * p->alpha;
    double *hl = malloc(sizeof(double) * 3 * N);
    orc_h_low(g, p, m_low, hl);
    for (int c = 0; c < 3; ++c) {
        orc_neg_laplacian(g, p->exchange, m_ex + c * N, f + c * N);
        for (long j = 0; j < N; ++j) f[c * N + j] = -chat * f[c * N + j] + s * hl[c * N + j];
    }
    free(hl);
}

int orc_step_euler(const orc_grid *g, const orc_params *p, const orc_opts *o, const double *m_n,
                   double *m_next, double *x_out, orc_info *info) {
    long N = nodes_of(g);
    orc_params q = *p;
    q.theta = 1.0;
    double *b = calloc((size_t)4 * N, sizeof(double));
    rhs_velocity(g, &q, m_n, m_n, b);
    memset(x_out, 0, sizeof(double) * 4 * N);
    orc_info inf;
    int rc = solve_system(g, &q, o, m_n, b, x_out, &inf);
    for (long j = 0; j < N; ++j) {
        double u[3], s = 0.0;
        for (int c = 0; c < 3; ++c) { u[c] = m_n[c * N + j] + q.k * x_out[c * N + j]; s += u[c] * u[c]; }
        s = sqrt(s);
        for (int c = 0; c < 3; ++c) m_next[c * N + j] = u[c] / s;
    }
    free(b);
    if (info) *info = inf;
    return rc;
}

int orc_step_midpoint(const orc_grid *g, const orc_params *p, const orc_opts *o, const double *m_n,
                      const double *v_prev, double *m_next, double *x_out, orc_info *info) {
    long N = nodes_of(g);
    orc_params q = *p;
    q.theta = 0.5;
    double *mhat = malloc(sizeof(double) * 3 * N), *vold = malloc(sizeof(double) * 3 * N);
    double *b = calloc((size_t)4 * N, sizeof(double));
    for (long i = 0; i < 3 * N; ++i) mhat[i] = m_n[i] + (v_prev ? 0.5 * q.k * v_prev[i] : 0.0);
    memset(x_out, 0, sizeof(double) * 4 * N);
    orc_info tot = { 0, 0, 0, 0, 0.0, 0.0 }, inf;
    int conv = 0, rc_lin = 0;
    for (int pi = 0; pi < o->picard_max; ++pi) {
        rhs_velocity(g, &q, m_n, mhat, b);   /* exchange split: Chat Lap m^n; h_low at the midpoint */
        rc_lin |= solve_system(g, &q, o, mhat, b, x_out, &inf);
        tot.iters += inf.iters;
        tot.restarts += inf.restarts;
        if (inf.rel_res_true > tot.rel_res_true) tot.rel_res_true = inf.rel_res_true;
        tot.picard_iters = pi + 1;
        if (pi >= 1) {
            double d = 0.0, nv = 0.0;
            for (long i = 0; i < 3 * N; ++i) {
                double e = x_out[i] - vold[i];
                d += e * e;
                nv += x_out[i] * x_out[i];
            }
            if (sqrt(d) <= o->picard_tol * sqrt(nv)) { conv = 1; break; }
        }
        memcpy(vold, x_out, sizeof(double) * 3 * N);
        for (long i = 0; i < 3 * N; ++i) mhat[i] = m_n[i] + 0.5 * q.k * x_out[i];
    }
    for (long i = 0; i < 3 * N; ++i) m_next[i] = m_n[i] + q.k * x_out[i];
    tot.converged = conv && !rc_lin;
    free(mhat); free(vold); free(b);
    if (info) *info = tot;
    return tot.converged ? 0 : 1;
}

/* ---------------------------------------------------------------- adjoint of a midpoint step */

/*
 * The converged midpoint step solves R(v, r) = 0 with mhat = m^n + (k/2) v:
 *   R_v = alpha v + (k/2) Chat (-Lap) v + Chat (-Lap) m^n + mhat x v + mhat r - (1+alpha^2) h_j
 *   (h_j = h + h_field_j, the applied field at node j)
 *   R_r = -mhat . v
 * Its Jacobian in (v, r):
 *   J_vv = alpha I + (k/2) Chat (-Lap) + [m^n]x + (k/2) r I,  J_vr = mhat,  J_rv = -(m^n + k v)^T.
 * With m^{n+1} = m^n + k v and y solving J^T y = (k mbar^{n+1}, 0):
 *   mbar^n = mbar^{n+1} - (dR/dm^n)^T y,  dL/dp -= y^T dR/dp.
 */
typedef struct {
    const orc_grid *g; const orc_params *p; const double *mn, *mhat, *mnext, *r;
} adj_ctx;

static void jt_op(void *c, const double *y, double *out) {
    adj_ctx *a = c;
    const orc_grid *g = a->g;
    long N = nodes_of(g);
    double b = 0.5 * a->p->k * chat_of(a->p);
    for (int q = 0; q < 3; ++q) fourier_apply(g, a->p->exchange, y + q * N, out + q * N, a->p->alpha, b, 0);
    for (long j = 0; j < N; ++j) {
        double m1 = a->mn[j], m2 = a->mn[N + j], m3 = a->mn[2 * N + j];
        double y1 = y[j], y2 = y[N + j], y3 = y[2 * N + j], yr = y[3 * N + j];
        double kr = 0.5 * a->p->k * a->r[j];
        /* J_vv^T y = ... - m^n x y + (k/2) r y ; minus m^{n+1} y_r */
        out[j] += -(m2 * y3 - m3 * y2) + kr * y1 - a->mnext[j] * yr;
        out[N + j] += -(m3 * y1 - m1 * y3) + kr * y2 - a->mnext[N + j] * yr;
        out[2 * N + j] += -(m1 * y2 - m2 * y1) + kr * y3 - a->mnext[2 * N + j] * yr;
        out[3 * N + j] = a->mhat[j] * y1 + a->mhat[N + j] * y2 + a->mhat[2 * N + j] * y3;
    }
}
static void jt_prec(void *c, const double *x, double *y) {
    adj_ctx *a = c;
    orc_ffthss_apply(a->g, a->p, a->mhat, x, y, 1);
}

int orc_adjoint_midpoint(const orc_grid *g, const orc_params *p, const orc_opts *o,
                         const double *m_n, const double *x, const double *mbar_next,
                         double *mbar_n, double *dalpha, double dh[3], orc_info *info) {
    long N = nodes_of(g);
    orc_params q = *p;
    q.theta = 0.5;
    if (q.k_an != 0.0 || q.demag) return 2;   /* adjoint covers a uniform applied field only */
    const double *v = x, *r = x + 3 * N;
    double *mhat = malloc(sizeof(double) * 3 * N), *mnext = malloc(sizeof(double) * 3 * N);
    for (long i = 0; i < 3 * N; ++i) { mhat[i] = m_n[i] + 0.5 * q.k * v[i]; mnext[i] = m_n[i] + q.k * v[i]; }
    double *rhs = calloc((size_t)4 * N, sizeof(double)), *y = calloc((size_t)4 * N, sizeof(double));
    for (long i = 0; i < 3 * N; ++i) rhs[i] = q.k * mbar_next[i];
    adj_ctx a = { g, &q, m_n, mhat, mnext, r };
    int rc;
    orc_info inf;
    memset(&inf, 0, sizeof(inf));
    if (o->use_dense) {
        long n = 4 * N;
        double *A = malloc(sizeof(double) * n * n);
        assemble_dense(n, jt_op, &a, A);
        rc = orc_dense_solve((int)n, A, rhs, y);
        free(A);
        inf.converged = rc == 0;
    } else {
        rc = gmres_core(4 * N, jt_op, jt_prec, &a, rhs, y, o->restart, o->max_iters, o->rtol, &inf, NULL, 0);
    }
    double chat = chat_of(&q), s = 1.0 + q.alpha * q.alpha;
    double *lap_y = malloc(sizeof(double) * 3 * N), *lap_v = malloc(sizeof(double) * 3 * N);
    double *lap_m = malloc(sizeof(double) * 3 * N);
    for (int c = 0; c < 3; ++c) {
        orc_neg_laplacian(g, q.exchange, y + c * N, lap_y + c * N);
        orc_neg_laplacian(g, q.exchange, v + c * N, lap_v + c * N);
        orc_neg_laplacian(g, q.exchange, m_n + c * N, lap_m + c * N);
    }
    double da = 0.0, dhx[3] = { 0, 0, 0 };
    for (long j = 0; j < N; ++j) {
        double yv[3] = { y[j], y[N + j], y[2 * N + j] }, yr = y[3 * N + j];
        double vv[3] = { v[j], v[N + j], v[2 * N + j] };
        double vxy[3] = { vv[1] * yv[2] - vv[2] * yv[1], vv[2] * yv[0] - vv[0] * yv[2], vv[0] * yv[1] - vv[1] * yv[0] };
        for (int c = 0; c < 3; ++c) {
            /* (dR/dm^n)^T y = Chat(-Lap) y_v + v x y_v + r y_v - v y_r */
            double t = chat * lap_y[c * N + j] + vxy[c] + r[j] * yv[c] - vv[c] * yr;
            mbar_n[c * N + j] = mbar_next[c * N + j] - t;
            /* dR_v/dalpha = v + alpha k c_ex (-Lap) v + 2 alpha c_ex (-Lap) m^n - 2 alpha h_j,
             * h_j = h + h_field_j: the whole applied field enters R_v through (1+alpha^2) h_low */
            double hj = q.h[c] + (q.h_field ? q.h_field[c * N + j] : 0.0);
            double dra = vv[c] + q.alpha * q.k * q.c_ex * lap_v[c * N + j]
                       + 2.0 * q.alpha * q.c_ex * lap_m[c * N + j] - 2.0 * q.alpha * hj;
            da -= yv[c] * dra;
            dhx[c] += s * yv[c];
        }
    }
    *dalpha += da;
    for (int c = 0; c < 3; ++c) dh[c] += dhx[c];
    free(lap_y); free(lap_v); free(lap_m); free(mhat); free(mnext); free(rhs); free(y);
    if (info) *info = inf;
    return rc == 0 ? 0 : 1;
}

/* ---------------------------------------------------------------- closed forms (Sec. 3.4) */

/* beta_N = alpha + theta k Chat max_xi |xi|^2 (Cor. "computable Fourier spectral enclosure") */
double orc_beta_N(const orc_grid *g, const orc_params *p) {
    double smax = 0.0;
    long N = nodes_of(g);
    for (long j = 0; j < N; ++j) {
        int kv[3];
        mode_of(g, j, kv);
        double s = orc_symbol(g, p->exchange, kv);
        if (s > smax) smax = s;
    }
    return p->alpha + p->theta * p->k * chat_of(p) * smax;
}
double orc_q_bar(double lambda, double alpha, double beta) {
    double a = fabs((lambda - alpha) / (lambda + alpha)), b = fabs((lambda - beta) / (lambda + beta));
    return a > b ? a : b;
}
double orc_lambda_bd(double alpha, double beta) { return sqrt(alpha * beta); }
double orc_gamma_m(double lambda, double m_min, double m_max) {
    double a = 2.0 * lambda * m_min / (lambda * lambda + m_min * m_min);
    double b = 2.0 * lambda * m_max / (lambda * lambda + m_max * m_max);
    return a < b ? a : b;
}
double orc_theta2(double q, double gamma) {
    double g2 = gamma * gamma, q2 = q * q;
    return sqrt(1.0 - (1.0 - q2) * g2 / (g2 + 1.0 + q2));
}
double orc_kappa(double lambda, double m_min, double m_max) {
    return sqrt((lambda * lambda + m_max * m_max) / (lambda * lambda + m_min * m_min));
}
int orc_iteration_bound(double kappa, double theta, double eps) {
    return 2 * (int)ceil(log(kappa / eps) / log(1.0 / theta));
}
