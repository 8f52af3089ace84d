// api.cu -- the C ABI of include/llg.h: context, operators, solves, time steps,
// adjoint.  Host code here only validates arguments, sequences kernels on the
// context's stream and reads back convergence scalars; all arithmetic of the
// method runs in the kernels of spectral.cu, krylov.cu and below.
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <new>
#include <vector>
#include <algorithm>
#include "llg_internal.h"
#include "krylov.h"
#include "reduce.cuh"
#include "convert.cuh"

using namespace llg;

namespace llg {

llg_status set_error(llg_ctx *c, llg_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

llg_status cuda_check(llg_ctx *c, cudaError_t e, const char *what) {
    if (c->hprog && c->hprog[KERR_WORD]) {
        // a kernel's bounded wait ran out (its block returned); the launch itself succeeded
        c->hprog[KERR_WORD] = 0;
        return set_error(c, LLG_ERR_TIMEOUT, std::string(what) + ": a bounded wait on an asynchronous copy ran out");
    }
    if (e == cudaSuccess) return LLG_OK;
    cudaGetLastError();
    return set_error(c, e == cudaErrorMemoryAllocation ? LLG_ERR_OOM : LLG_ERR_CUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

void prof_begin(llg_ctx *c, int cls, double bytes, double flops, int tag, int count) {
    c->prof_open = -1;
    if (c->prof_class == 0 || cls != c->prof_class) return;
    if (c->prof_used == c->prof.size()) {
        if (c->prof.size() >= 65536) return;
        llg_ctx::ProfEntry e{};
        if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        c->prof.push_back(e);
    }
    llg_ctx::ProfEntry &e = c->prof[c->prof_used];
    e.bytes = bytes;
    e.flops = flops;
    e.tag = tag;
    e.valid = 1;
    e.count = count;
    cudaEventRecord(e.a, c->stream);
    c->prof_open = (int)c->prof_used++;
}

void prof_end(llg_ctx *c) {
    if (c->prof_open < 0) return;
    cudaEventRecord(c->prof[c->prof_open].b, c->stream);
    c->prof_open = -1;
}

// drop entries recorded since `first` whose tag (Arnoldi step index) is >= min_tag:
// those launches found the cycle's stopping flag set and did no work
void prof_discard(llg_ctx *c, size_t first, int min_tag) {
    for (size_t i = first; i < c->prof_used; ++i)
        if (c->prof[i].tag >= min_tag) c->prof[i].valid = 0;
}

// ------------------------------------------------------------------ small kernels

// Self-check of the integer-pipe conversions (convert.cuh) against the hardware ones.
// Floats: every bit pattern u in [first, first + count).  Doubles: `count` patterns from a
// counter-based hash, mixed so that a quarter are arbitrary, a quarter have exponents in
// and around the float range, a quarter sit on or next to a rounding tie, and a quarter are
// ties in the float subnormal range.  Mismatches (NaN against NaN counts as a match) are
// added to bad[0] (float -> double) and bad[1] (double -> float).
__device__ __forceinline__ unsigned long long conv_hash(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void k_conv_check_f2d(unsigned long long first, unsigned long long count, unsigned long long *bad) {
    unsigned long long local = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float f = __uint_as_float((unsigned)(first + i));
        const double a = (double)f, b = f2d_exact(f);
        const bool same = __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b);
        local += same ? 0ull : 1ull;
    }
    if (local) atomicAdd(&bad[0], local);
}

__global__ void k_conv_check_d2f(unsigned long long seed, unsigned long long count, unsigned long long *bad) {
    unsigned long long local = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long u = conv_hash(seed + 2 * i);
        const unsigned long long r = conv_hash(seed + 2 * i + 1);
        const unsigned kind = (unsigned)(i & 3);
        if (kind == 1) {
            const unsigned long long ex = 856ull + (r >> 33) % 400ull;
            u = (u & 0x800fffffffffffffull) | (ex << 52);
        } else if (kind == 2) {
            const unsigned long long ex = 866ull + (r >> 40) % 300ull, t = (r >> 20) & 3ull;
            u = (u & 0x800fffffe0000000ull) | (ex << 52) |
                (t == 0 ? 0x10000000ull : (t == 1 ? 0x0fffffffull : 0x10000001ull));
        } else if (kind == 3) {
            const unsigned long long ex = 866ull + (r >> 40) % 31ull;
            const int sh = 926 - (int)ex;
            unsigned long long m = u & 0xfffffffffffffull;
            if (sh >= 1 && sh <= 52) m = (m & ~((1ull << sh) - 1ull)) | (1ull << (sh - 1));
            u = (u & 0x8000000000000000ull) | (ex << 52) | m;
        }
        const double d = __longlong_as_double((long long)u);
        const float a = (float)d, b = d2f_rn(d);
        const bool same = __float_as_uint(a) == __float_as_uint(b) || (a != a && b != b);
        local += same ? 0ull : 1ull;
    }
    if (local) atomicAdd(&bad[1], local);
}

template <typename T>
__global__ void k_fma_probe(T *out, int iters) {
    T a[8];
    for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    const T b = (T)0.9999999, cc = (T)1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, cc);
    }
    T s = 0;
    for (int i = 0; i < 8; ++i) s += a[i];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_min_norm2(const double *__restrict__ m, long long N, double *partials) {
    long long lo, hi;
    block_chunk(N, lo, hi);
    double v = -1e300;
    for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const double a = m[j], b = m[N + j], c = m[2 * N + j];
        const double q = -(a * a + b * b + c * c);
        v = q != q ? 1e308 : fmax(v, q);   // a non-finite node fails the check too
    }
    block_max_store(v, partials + (long long)blockIdx.x * RB_STRIDE);
}

// max over the blocks' partials, the whole block reading them (launch with RB_THREADS)
__global__ void k_max_partials(const double *__restrict__ partials, int nb, double *dst) {
    double s = -1e300;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s = fmax(s, partials[(long long)b * RB_STRIDE]);
    block_max_store(s, dst);
}

__global__ void k_sum_partials_n(const double *__restrict__ partials, int nb, int cnt, double *dst) {
    block_sum_partials(partials, nb, cnt, dst);
}

// the FP32 copy of the nodal field m (3 planes) and, in the same pass, per-block maxima of
// -|m_i|^2 (the degenerate-node check of flexible solves)
__global__ void k_to_f32_minnorm(const double *__restrict__ m, float *__restrict__ m32, long long N, double *partials) {
    long long lo, hi;
    block_chunk(N, lo, hi);
    double v = -1e300;
    for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const double a = m[j], b = m[N + j], c = m[2 * N + j];
        m32[j] = d2f_rn(a);
        m32[N + j] = d2f_rn(b);
        m32[2 * N + j] = d2f_rn(c);
        const double q = -(a * a + b * b + c * c);
        v = q != q ? 1e308 : fmax(v, q);   // a non-finite node fails the check too
    }
    block_max_store(v, partials + (long long)blockIdx.x * RB_STRIDE);
}

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, long long n) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = d2f_rn(a[e]);
}

// y = s a (s = *scale, or 1 when scale is NULL): the identity "preconditioner"
template <typename TO, typename TI>
__global__ void k_scaled_copy(const TI *__restrict__ a, const double *__restrict__ scale, TO *__restrict__ y,
                              long long n) {
    const double sc = scale ? *scale : 1.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        y[e] = (TO)(sc * a[e]);
}

// m^{n+1} = (m + k v) / |m + k v|, and max_i | |m^{n+1}_i| - |m^n_i| |
__global__ void k_euler_update(const double *__restrict__ m, const double *__restrict__ v, double k, double *mn,
                               long long N, double *partials) {
    long long lo, hi;
    block_chunk(N, lo, hi);
    double drift = 0.0;
    for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const double a = m[j] + k * v[j], b = m[N + j] + k * v[N + j], c = m[2 * N + j] + k * v[2 * N + j];
        const double s = sqrt(a * a + b * b + c * c);
        mn[j] = a / s;
        mn[N + j] = b / s;
        mn[2 * N + j] = c / s;
        const double m0 = sqrt(m[j] * m[j] + m[N + j] * m[N + j] + m[2 * N + j] * m[2 * N + j]);
        drift = fmax(drift, fabs(1.0 - m0));
    }
    block_max_store(drift, partials + (long long)blockIdx.x * RB_STRIDE);
}

// out = m + c v (3 planes; v may be NULL)
__global__ void k_axpy3(const double *__restrict__ m, const double *__restrict__ v, double c, double *out, long long n3) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x)
        out[e] = m[e] + (v ? c * v[e] : 0.0);
}

// Picard advance: mhat' = m + hk v, and the exact residual of x for the new blocks,
// r0 = r_prev - [A(mhat') - A(mhat)] x = r_prev - (dm x v + dm r, -dm . v), dm = mhat' - mhat
// (only the nodal skew/constraint blocks depend on the midpoint field), written over r_prev,
// with per-block partial sums of |r0|^2
__global__ void __launch_bounds__(RB_THREADS) k_picard_advance(const double *__restrict__ m, const double *__restrict__ x,
                                                               double hk, double *mhat, double *r, long long N,
                                                               double *partials) {
    const double *rprev = r;
    double *r0 = r;
    f32x2 sq{0.0f, 0.0f};
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        const double v1 = x[j], v2 = x[N + j], v3 = x[2 * N + j], r = x[3 * N + j];
        const double a1 = m[j] + hk * v1, a2 = m[N + j] + hk * v2, a3 = m[2 * N + j] + hk * v3;
        const double d1 = a1 - mhat[j], d2 = a2 - mhat[N + j], d3 = a3 - mhat[2 * N + j];
        // the change of the nodal blocks and the squared norm in FP32-pair arithmetic (off the
        // FP64 unit): dm is small beside m, and its terms carry about 47 bits, far below the FP64
        // rounding of r0 itself; mhat and r0 stay FP64
        const fpair D1 = cvt<fpair>(d1), D2 = cvt<fpair>(d2), D3 = cvt<fpair>(d3);
        const fpair V1 = cvt<fpair>(v1), V2 = cvt<fpair>(v2), V3 = cvt<fpair>(v3), R = cvt<fpair>(r);
        const double q0 = rprev[j] - cvt<double>(fp_dot2(D2, V3, -D3, V2) + D1 * R);
        const double q1 = rprev[N + j] - cvt<double>(fp_dot2(D3, V1, -D1, V3) + D2 * R);
        const double q2 = rprev[2 * N + j] - cvt<double>(fp_dot2(D1, V2, -D2, V1) + D3 * R);
        const double q3 = rprev[3 * N + j] + cvt<double>(fp_dot2(D1, V1, D2, V2) + D3 * V3);
        r0[j] = q0;
        r0[N + j] = q1;
        r0[2 * N + j] = q2;
        r0[3 * N + j] = q3;
        mhat[j] = a1;
        mhat[N + j] = a2;
        mhat[2 * N + j] = a3;
        const f32x2 p0 = split_f64(q0), p1 = split_f64(q1), p2 = split_f64(q2), p3 = split_f64(q3);
        fma_acc(p0, p0, sq);
        fma_acc(p1, p1, sq);
        fma_acc(p2, p2, sq);
        fma_acc(p3, p3, sq);
    }
    double acc[1] = {pair_to_f64(sq)};
    block_reduce_store<1>(acc, 1, partials + (long long)blockIdx.x * RB_STRIDE);
}

// partial sums of |v - vold|^2 and |v|^2 for the Picard stopping test, then vold = v.  The
// difference is formed in FP64; the squares are summed in FP32 per thread (the test compares
// the two norms to a tolerance: six significant digits are plenty) and in FP64 across
// threads, off the FP64 unit that the three multiply-adds a value would otherwise load.
// (V2: two elements a thread per 16-byte access; both arrays 16-byte aligned)
template <bool V2>
__global__ void __launch_bounds__(RB_THREADS) k_picard_norms_advance(const double *__restrict__ v, double *__restrict__ vold,
                                                                     long long n3, double *partials) {
    long long lo, hi;
    block_chunk(n3, lo, hi);
    float s0 = 0.0f, s1 = 0.0f;
    auto one = [&](double ve, double vo) {
        const float d = d2f_rn(ve - vo), vf = d2f_rn(ve);
        s0 = __fmaf_rn(d, d, s0);
        s1 = __fmaf_rn(vf, vf, s1);
    };
    if constexpr (V2) {
        for (long long e = lo + 2 * threadIdx.x; e + 1 < hi; e += 2 * blockDim.x) {
            const double2 ve = *reinterpret_cast<const double2 *>(v + e), vo = *reinterpret_cast<const double2 *>(vold + e);
            one(ve.x, vo.x);
            one(ve.y, vo.y);
            *reinterpret_cast<double2 *>(vold + e) = ve;
        }
        if (((hi - lo) & 1) && threadIdx.x == 0) {
            one(v[hi - 1], vold[hi - 1]);
            vold[hi - 1] = v[hi - 1];
        }
    } else {
        for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
            one(v[e], vold[e]);
            vold[e] = v[e];
        }
    }
    double acc[2] = {(double)s0, (double)s1};
    block_reduce_store<2>(acc, 2, partials + (long long)blockIdx.x * RB_STRIDE);
}


// m^{n+1} = m^n + k v and max_i | |m^{n+1}_i| - |m^n_i| |
__global__ void k_mid_final(const double *__restrict__ m, const double *__restrict__ v, double k, double *mn,
                            long long N, double *partials) {
    long long lo, hi;
    block_chunk(N, lo, hi);
    double drift = 0.0;
    for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const double a0 = m[j], b0 = m[N + j], c0 = m[2 * N + j];
        const double a = a0 + k * v[j], b = b0 + k * v[N + j], c = c0 + k * v[2 * N + j];
        mn[j] = a;
        mn[N + j] = b;
        mn[2 * N + j] = c;
        drift = fmax(drift, fabs(sqrt(a * a + b * b + c * c) - sqrt(a0 * a0 + b0 * b0 + c0 * c0)));
    }
    block_max_store(drift, partials + (long long)blockIdx.x * RB_STRIDE);
}

// energy density sum: m . T - h . m, with T = (c_ex/2)(-Lap) m
// node sums of c_ex/2 m.(-Lap m) - (h + h_field).m + k_an (1 - (e.m)^2) - 1/2 m.h_dem
// (T = c_ex/2 (-Lap) m; hf, hd may be NULL)
__global__ void k_energy_partials(const double *__restrict__ m, const double *__restrict__ T, double h0, double h1,
                                  double h2, const double *__restrict__ hf, const double *__restrict__ hd, double kan,
                                  double e0, double e1, double e2, long long N, double *partials) {
    long long lo, hi;
    block_chunk(N, lo, hi);
    double acc[1] = {0.0};
    for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const double a = m[j], b = m[N + j], c = m[2 * N + j];
        double g0 = h0, g1 = h1, g2 = h2;
        if (hf) {
            g0 += hf[j];
            g1 += hf[N + j];
            g2 += hf[2 * N + j];
        }
        double ej = a * T[j] + b * T[N + j] + c * T[2 * N + j] - (g0 * a + g1 * b + g2 * c);
        if (kan != 0.0) {
            const double em = e0 * a + e1 * b + e2 * c;
            ej += kan * (1.0 - em * em);
        }
        if (hd) ej -= 0.5 * (a * hd[j] + b * hd[N + j] + c * hd[2 * N + j]);
        acc[0] += ej;
    }
    block_reduce_store<1>(acc, 1, partials + (long long)blockIdx.x * RB_STRIDE);
}

// adjoint preparation: mhat = m + (k/2) v; rhs = (k mbar, 0); u = alpha c_ex (k v + 2 m)
__global__ void k_adj_prep(const double *__restrict__ m, const double *__restrict__ v, const double *__restrict__ mbar,
                           double k, double ac, double *mhat, double *rhs, double *u, long long N) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        for (int q = 0; q < 3; ++q) {
            const long long e = q * N + j;
            mhat[e] = m[e] + 0.5 * k * v[e];
            rhs[e] = k * mbar[e];
            u[e] = ac * (k * v[e] + 2.0 * m[e]);
        }
        rhs[3 * N + j] = 0.0;
    }
}

// mbar_n = mbar_next - [Chat(-Lap) y_v + v x y_v + r y_v - v y_r];
// partial sums of -y_v . (v + (-Lap) u - 2 alpha h_j) and of y_v (per component), with
// h_j = h + hf_j the applied field at node j (hf may be NULL: zero)
__global__ void k_adj_final(const double *__restrict__ mbar_next, const double *__restrict__ y,
                            const double *__restrict__ lapy, const double *__restrict__ xf,
                            const double *__restrict__ lapu, double alpha, double h0, double h1, double h2,
                            const double *__restrict__ hf, double *mbar_n, long long N, double *partials) {
    long long lo, hi;
    block_chunk(N, lo, hi);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const double h[3] = {h0, h1, h2};
    for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const double y1 = y[j], y2 = y[N + j], y3 = y[2 * N + j], yr = y[3 * N + j];
        const double v1 = xf[j], v2 = xf[N + j], v3 = xf[2 * N + j], r = xf[3 * N + j];
        const double cx[3] = {v2 * y3 - v3 * y2, v3 * y1 - v1 * y3, v1 * y2 - v2 * y1};
        const double yv[3] = {y1, y2, y3}, vv[3] = {v1, v2, v3};
        for (int q = 0; q < 3; ++q) {
            const long long e = q * N + j;
            mbar_n[e] = mbar_next[e] - (lapy[e] + cx[q] + r * yv[q] - vv[q] * yr);
            const double hq = hf ? h[q] + hf[e] : h[q];
            acc[0] -= yv[q] * (vv[q] + lapu[e] - 2.0 * alpha * hq);
            acc[1 + q] += yv[q];
        }
    }
    block_reduce_store<4>(acc, 4, partials + (long long)blockIdx.x * RB_STRIDE);
}

}  // namespace llg

// ------------------------------------------------------------------ helpers

namespace {

bool is_pow2(int n) { return n >= 2 && n <= 1024 && (n & (n - 1)) == 0; }
int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
double chat(const llg_params *p) { return (1.0 + p->alpha * p->alpha) * p->c_ex; }

llg_status check_params(llg_ctx *c, const llg_params *p) {
    if (!p) return set_error(c, LLG_ERR_INVALID_ARG, "params is NULL");
    const double v[] = {p->alpha, p->c_ex, p->k, p->theta, p->lambda, p->h_ext[0], p->h_ext[1], p->h_ext[2]};
    for (double d : v)
        if (!std::isfinite(d)) return set_error(c, LLG_ERR_INVALID_ARG, "non-finite parameter");
    if (!(p->alpha > 0) || !(p->c_ex > 0) || !(p->lambda > 0) || p->k < 0 || !(p->theta > 0))
        return set_error(c, LLG_ERR_INVALID_ARG, "need alpha > 0, c_ex > 0, lambda > 0, k >= 0, theta > 0");
    if (p->exchange != LLG_EX_SPECTRAL && p->exchange != LLG_EX_FD2)
        return set_error(c, LLG_ERR_INVALID_ARG, "unknown exchange discretisation");
    if (!std::isfinite(p->k_an) || !std::isfinite(p->e_an[0]) || !std::isfinite(p->e_an[1]) || !std::isfinite(p->e_an[2]))
        return set_error(c, LLG_ERR_INVALID_ARG, "non-finite anisotropy parameter");
    if (p->demag != 0 && p->demag != 1) return set_error(c, LLG_ERR_INVALID_ARG, "demag must be 0 or 1");
    return LLG_OK;
}

// does h_low depend on m (demagnetising or anisotropy field)?
bool field_depends_on_m(const llg_params *p) { return p->demag != 0 || p->k_an != 0.0; }

llg_status check_opts(llg_ctx *c, const llg_opts *o) {
    if (!o) return set_error(c, LLG_ERR_INVALID_ARG, "opts is NULL");
    if (o->restart < 1 || o->restart > GmresDev::MAXM) return set_error(c, LLG_ERR_INVALID_ARG, "restart must be in [1, 64]");
    if (o->max_iters < 1 || !(o->rtol > 0) || !std::isfinite(o->rtol))
        return set_error(c, LLG_ERR_INVALID_ARG, "need max_iters >= 1 and rtol > 0");
    if (o->precision != LLG_PREC_FP64 && o->precision != LLG_PREC_FP32_FLEX)
        return set_error(c, LLG_ERR_INVALID_ARG, "unknown precision");
    if (o->picard_max < 1 || !(o->picard_tol > 0)) return set_error(c, LLG_ERR_INVALID_ARG, "need picard_max >= 1 and picard_tol > 0");
    if (o->preconditioner != LLG_PC_FFTHSS && o->preconditioner != LLG_PC_HERMITIAN && o->preconditioner != LLG_PC_NONE)
        return set_error(c, LLG_ERR_INVALID_ARG, "unknown preconditioner");
    if (o->gs_arith != LLG_GS_FP64 && o->gs_arith != LLG_GS_F32X2)
        return set_error(c, LLG_ERR_INVALID_ARG, "unknown Gram-Schmidt arithmetic");
    if (o->chain_arith != LLG_CHAIN_FP64 && o->chain_arith != LLG_CHAIN_F32X2)
        return set_error(c, LLG_ERR_INVALID_ARG, "unknown Fourier-chain arithmetic");
    return LLG_OK;
}

llg_status ensure_spec(llg_ctx *c, bool fp64, bool fp32) {
    const size_t elems = (size_t)c->geo.rows * c->geo.S;
    if (fp64 && !c->spec64) {
        cudaError_t e = cudaMalloc(&c->spec64, elems * sizeof(double2));
        if (e == cudaSuccess) e = cudaMemsetAsync(c->spec64, 0, elems * sizeof(double2), c->stream);
        if (e != cudaSuccess) { c->spec64 = nullptr; return cuda_check(c, e, "spectral buffer (FP64)"); }
    }
    if (fp32 && !c->spec32) {
        cudaError_t e = cudaMalloc(&c->spec32, elems * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemsetAsync(c->spec32, 0, elems * sizeof(float2), c->stream);
        if (e != cudaSuccess) { c->spec32 = nullptr; return cuda_check(c, e, "spectral buffer (FP32)"); }
    }
    return LLG_OK;
}

llg_status ensure_aux(llg_ctx *c) {
    if (c->aux) return LLG_OK;
    cudaError_t e = cudaMalloc(&c->aux, sizeof(double) * 24 * c->geo.N);
    if (e != cudaSuccess) { c->aux = nullptr; return cuda_check(c, e, "stepper scratch"); }
    return LLG_OK;
}

llg_status ensure_m32(llg_ctx *c) {
    if (c->m32) return LLG_OK;
    cudaError_t e = cudaMalloc(&c->m32, sizeof(float) * 3 * c->geo.N);
    if (e != cudaSuccess) { c->m32 = nullptr; return cuda_check(c, e, "FP32 field copy"); }
    return LLG_OK;
}

int grid_blocks(llg_ctx *c) { return 4 * c->sm_count; }

llg_status sync_scalars(llg_ctx *c, int count) {
    cudaError_t e = cudaMemcpyAsync(c->hsc, c->dsc, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "device->host scalars");
}

template <typename TIn, typename TOut, typename T>
NodalIO<TIn, TOut, T> make_io(const nodal_t<T> *m, const TIn *x, TOut *y, const double *scale, double lam) {
    NodalIO<TIn, TOut, T> io;
    std::memset(&io, 0, sizeof(io));
    io.m = m; io.x = x; io.y = y; io.scale = scale; io.lam = (T)lam;
    return io;
}

Symbol sym_shifted_inverse(llg_ctx *c, const llg_params *p, double theta) {
    return Symbol{p->alpha + p->lambda, theta * p->k * chat(p), 1.0 / (double)c->geo.N, 1, p->exchange};
}
Symbol sym_forward(llg_ctx *c, const llg_params *p, double theta) {
    return Symbol{p->alpha, theta * p->k * chat(p), 1.0 / (double)c->geo.N, 0, p->exchange};
}

// FP64 operators ------------------------------------------------------------

llg_status op_matvec64(llg_ctx *c, const llg_params *p, double theta, const double *m, const double *x,
                       const double *scale, double *y, int transpose, const int *skip = nullptr) {
    auto io = make_io<double, double, double>(m, x, y, scale, p->lambda);
    io.transpose = transpose;
    io.skip = skip;
    return spectral_chain<double, double, double>(c, IN_V, OUT_MATVEC, io, sym_forward(c, p, theta));
}

// the same matvec (unscaled, untransposed) with the Fourier chain in FP32-pair arithmetic
llg_status op_matvec_pair(llg_ctx *c, const llg_params *p, double theta, const double *m, const double *x, double *y,
                          int transpose = 0) {
    auto io = make_io<double, double, fpair>(m, x, y, nullptr, p->lambda);
    io.transpose = transpose;
    return spectral_chain<fpair, double, double>(c, IN_V, OUT_MATVEC, io, sym_forward(c, p, theta));
}

llg_status op_apply64(llg_ctx *c, const llg_params *p, double theta, const double *m, const double *x,
                      const double *scale, double *y, int transpose) {
    auto io = make_io<double, double, double>(m, x, y, scale, p->lambda);
    if (!transpose) return spectral_chain<double, double, double>(c, IN_V, OUT_APPLY, io, sym_shifted_inverse(c, p, theta));
    return spectral_chain<double, double, double>(c, IN_NODAL_T, OUT_PLAIN, io, sym_shifted_inverse(c, p, theta));
}

llg_status op_fused64(llg_ctx *c, const llg_params *p, double theta, const double *m, const double *x,
                      const double *scale, double *y, int plain_nodal = 0, const int *skip = nullptr) {
    auto io = make_io<double, double, double>(m, x, y, scale, p->lambda);
    io.plain_nodal = plain_nodal;
    io.skip = skip;
    return spectral_chain<double, double, double>(c, IN_FUSED, OUT_FUSED, io, sym_shifted_inverse(c, p, theta));
}

// the shifted symmetric part (lambda I + H)^{-1} alone (no nodal inverse)
llg_status op_hermitian64(llg_ctx *c, const llg_params *p, double theta, const double *m, const double *x,
                          const double *scale, double *y) {
    auto io = make_io<double, double, double>(m, x, y, scale, p->lambda);
    io.plain_nodal = 1;
    return spectral_chain<double, double, double>(c, IN_V, OUT_APPLY, io, sym_shifted_inverse(c, p, theta));
}

template <typename TO, typename TI = double>
llg_status op_scaled_copy(llg_ctx *c, const TI *x, const double *scale, TO *y) {
    k_scaled_copy<TO, TI><<<grid_blocks(c), RB_THREADS, 0, c->stream>>>(x, scale, y, 4 * c->geo.N);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "identity preconditioner");
}

llg_status check_nodes(llg_ctx *c, const double *m) {
    const int nb = reduction_blocks(c);
    k_min_norm2<<<nb, RB_THREADS, 0, c->stream>>>(m, c->geo.N, c->red);
    k_max_partials<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, c->dsc);
    c->launches += 2;
    llg_status st = cuda_check(c, cudaGetLastError(), "node check");
    if (st != LLG_OK) return st;
    if ((st = sync_scalars(c, 1)) != LLG_OK) return st;
    const double minn2 = -c->hsc[0];
    if (!(minn2 > 0.0) || !std::isfinite(minn2))
        return set_error(c, LLG_ERR_DEGENERATE_NODE, "some node has |m_i| = 0 (or non-finite): the saddle matrix is singular");
    return LLG_OK;
}

// solve A(m; theta) x = b with the chosen precision
// r0_ready: r0 is the workspace's own first-residual buffer with its squared norm already
// queued into device scalar 2 (the midpoint step's in-place Picard advance)
// bnorm_slot >= 0: ||b||^2 is already queued into that device scalar
llg_status solve(llg_ctx *c, const llg_params *p, double theta, const llg_opts *o, const double *m, const double *b,
                 double *x, llg_info *info, const double *r0 = nullptr, bool r0_ready = false, int bnorm_slot = -1) {
    const bool flex = o->precision == LLG_PREC_FP32_FLEX;
    llg_status st = LLG_OK;
    // FP64 solves check the nodes here; flexible solves in the pass that makes the FP32 copy
    // of m, read with the solve's first device scalars (no host round trip of its own)
    if (!flex && (st = check_nodes(c, m)) != LLG_OK) return st;
    if ((st = ensure_spec(c, true, flex)) != LLG_OK) return st;
    SolveOps ops;
    ops.r0_ready = r0_ready;
    ops.bnorm_slot = bnorm_slot;
    // the true residuals: FP64 chain, or the FP32-pair chain where every axis has one
    if (o->chain_arith == LLG_CHAIN_F32X2 && pair_chains_available(c))
        ops.matvec = [=](const double *xx, double *yy) { return op_matvec_pair(c, p, theta, m, xx, yy); };
    else
        ops.matvec = [=](const double *xx, double *yy) { return op_matvec64(c, p, theta, m, xx, nullptr, yy, 0); };
    const int pc = o->preconditioner;
    // operators issued inside a GMRES cycle return at once once the cycle's stopping flag
    // is set (the host may have queued one more step); v_0 and the true residual,
    // issued outside cycles, always run
    const int *cyc = &c->gdev->done;
    if (!flex) {
        if (pc == LLG_PC_NONE) {
            ops.prec = [=](const double *xx, const double *s, double *yy) { return op_scaled_copy<double>(c, xx, s, yy); };
            ops.pop = [=](const double *xx, const double *s, double *yy) { return op_matvec64(c, p, theta, m, xx, s, yy, 0, cyc); };
        } else if (pc == LLG_PC_HERMITIAN) {
            ops.prec = [=](const double *xx, const double *s, double *yy) { return op_hermitian64(c, p, theta, m, xx, s, yy); };
            ops.pop = [=](const double *xx, const double *s, double *yy) { return op_fused64(c, p, theta, m, xx, s, yy, 1, cyc); };
        } else {
            ops.prec = [=](const double *xx, const double *s, double *yy) { return op_apply64(c, p, theta, m, xx, s, yy, 0); };
            ops.pop = [=](const double *xx, const double *s, double *yy) { return op_fused64(c, p, theta, m, xx, s, yy, 0, cyc); };
        }
    } else {
        if ((st = ensure_m32(c)) != LLG_OK) return st;
        const int nb = reduction_blocks(c);
        k_to_f32_minnorm<<<nb, RB_THREADS, 0, c->stream>>>(m, c->m32, c->geo.N, c->red);
        k_max_partials<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, c->dsc + SolveOps::NODE_CHECK_SLOT);
        c->launches += 2;
        if ((st = cuda_check(c, cudaGetLastError(), "FP32 field copy")) != LLG_OK) return st;
        ops.node_check = true;
        const float *m32 = c->m32;
        ops.fprec = [=](const double *xx, const double *s, float *zz) {
            if (pc == LLG_PC_NONE) return op_scaled_copy<float>(c, xx, s, zz);
            auto io = make_io<double, float, float>(m32, xx, zz, s, p->lambda);
            io.plain_nodal = pc == LLG_PC_HERMITIAN;
            io.skip = cyc;
            return spectral_chain<float, double, float>(c, IN_V, OUT_APPLY, io, sym_shifted_inverse(c, p, theta));
        };
        ops.fmatvec = [=](const float *zz, double *ww) {
            auto io = make_io<float, double, float>(m32, zz, ww, nullptr, p->lambda);
            io.skip = cyc;
            return spectral_chain<float, float, double>(c, IN_V, OUT_MATVEC, io, sym_forward(c, p, theta));
        };
        // the same two operators on FP32 data (FP32-pair Gram-Schmidt: hi planes of the basis and of w)
        ops.fprec32 = [=](const float *xx, const double *s, float *zz) {
            if (pc == LLG_PC_NONE) return op_scaled_copy<float, float>(c, xx, s, zz);
            auto io = make_io<float, float, float>(m32, xx, zz, s, p->lambda);
            io.plain_nodal = pc == LLG_PC_HERMITIAN;
            io.skip = cyc;
            return spectral_chain<float, float, float>(c, IN_V, OUT_APPLY, io, sym_shifted_inverse(c, p, theta));
        };
        ops.fmatvec32 = [=](const float *zz, float *ww) {
            auto io = make_io<float, float, float>(m32, zz, ww, nullptr, p->lambda);
            io.skip = cyc;
            return spectral_chain<float, float, float>(c, IN_V, OUT_MATVEC, io, sym_forward(c, p, theta));
        };
        if (pc != LLG_PC_NONE && chain_pm_available(c)) {
            // preconditioner and matvec in one sequence: the x-pass inverse of the first fused
            // with the x-pass forward of the second
            ops.fpm = [=](const double *xx, const double *s, float *zz, float *ww) {
                auto io1 = make_io<double, float, float>(m32, xx, zz, s, p->lambda);
                io1.plain_nodal = pc == LLG_PC_HERMITIAN;
                io1.skip = cyc;
                auto io2 = make_io<float, float, float>(m32, zz, ww, nullptr, p->lambda);
                io2.skip = cyc;
                return spectral_chain_pm<double>(c, io1, sym_shifted_inverse(c, p, theta), io2, sym_forward(c, p, theta));
            };
            ops.fpm32 = [=](const float *xx, const double *s, float *zz, float *ww) {
                auto io1 = make_io<float, float, float>(m32, xx, zz, s, p->lambda);
                io1.plain_nodal = pc == LLG_PC_HERMITIAN;
                io1.skip = cyc;
                auto io2 = make_io<float, float, float>(m32, zz, ww, nullptr, p->lambda);
                io2.skip = cyc;
                return spectral_chain_pm<float>(c, io1, sym_shifted_inverse(c, p, theta), io2, sym_forward(c, p, theta));
            };
        }
    }
    return gmres_run(c, ops, flex, o, b, x, info, r0);
}

// the per-node part of h_low(m) (applied field array + demagnetising + anisotropy fields):
// *hf = NULL when there is none, p->h_field itself when that is all, else `out` (3N)
llg_status lowfield_nodal(llg_ctx *c, const llg_params *p, const double *m, double *out, const double **hf) {
    *hf = nullptr;
    if (!field_depends_on_m(p)) {
        *hf = p->h_field;
        return LLG_OK;
    }
    const long long N = c->geo.N;
    llg_status st = LLG_OK;
    if (p->demag) {
        if ((st = demag_field(c, m, out)) != LLG_OK) return st;
    } else {
        cudaMemsetAsync(out, 0, sizeof(double) * 3 * N, c->stream);
    }
    if (p->h_field) {
        k_axpy3<<<grid_blocks(c), RB_THREADS, 0, c->stream>>>(out, p->h_field, 1.0, out, 3 * N);
        c->launches++;
    }
    if (p->k_an != 0.0 && (st = anisotropy_add(c, m, p->k_an, p->e_an, out)) != LLG_OK) return st;
    *hf = out;
    return cuda_check(c, cudaGetLastError(), "lower-order field");
}

template <typename T>
llg_status rhs_velocity_t(llg_ctx *c, const llg_params *p, const double *m, const double *hf, double *b) {
    // f = Chat Lap_N m + (1 + alpha^2) (h_ext + per-node part of h_low) ; multiplier row 0
    auto io = make_io<double, double, T>(m, m, b, nullptr, p->lambda);
    const double s = 1.0 + p->alpha * p->alpha;
    for (int q = 0; q < 3; ++q) io.fld[q] = (T)(s * p->h_ext[q]);
    io.hf = hf;
    io.hs = s;
    Symbol sym{0.0, -chat(p), 1.0 / (double)c->geo.N, 0, p->exchange};
    return spectral_chain<T, double, double>(c, IN_M, OUT_FIELD, io, sym);
}

// the right-hand side in the arithmetic opts->chain_arith asks for (FP64 where the grid has
// no FP32-pair chain)
llg_status rhs_velocity(llg_ctx *c, const llg_params *p, const llg_opts *o, const double *m, const double *hf, double *b) {
    if (o->chain_arith == LLG_CHAIN_F32X2 && pair_chains_available(c)) return rhs_velocity_t<fpair>(c, p, m, hf, b);
    return rhs_velocity_t<double>(c, p, m, hf, b);
}

llg_status energy_async(llg_ctx *c, const llg_params *p, const double *m, double *tmp, double *dst_dev) {
    auto io = make_io<double, double, double>(m, m, tmp, nullptr, p->lambda);
    Symbol sym{0.0, 0.5 * p->c_ex, 1.0 / (double)c->geo.N, 0, p->exchange};
    llg_status st = spectral_chain<double, double, double>(c, IN_M, OUT_PLAIN, io, sym);
    if (st != LLG_OK) return st;
    const double *hd = nullptr;
    if (p->demag) {
        double *hbuf = c->aux + 21 * c->geo.N;   // 3N scratch no caller of energy_async uses
        if ((st = demag_field(c, m, hbuf)) != LLG_OK) return st;
        hd = hbuf;
    }
    const int nb = reduction_blocks(c);
    k_energy_partials<<<nb, RB_THREADS, 0, c->stream>>>(m, tmp, p->h_ext[0], p->h_ext[1], p->h_ext[2], p->h_field, hd,
                                                        p->k_an, p->e_an[0], p->e_an[1], p->e_an[2], c->geo.N, c->red);
    k_sum_partials_n<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, 1, dst_dev);
    c->launches += 2;
    return cuda_check(c, cudaGetLastError(), "energy");
}

#define LLG_GUARD(ctx)                                                                       \
    if (!(ctx)) return LLG_ERR_INVALID_ARG;                                                  \
    (ctx)->err.clear();

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

llg_status llg_create(const llg_grid *grid, void *cuda_stream, llg_ctx **out) {
    if (!out || !grid) return LLG_ERR_INVALID_ARG;
    *out = nullptr;
    if (grid->dim != 2 && grid->dim != 3) return LLG_ERR_INVALID_ARG;
    for (int l = 0; l < grid->dim; ++l) {
        if (!is_pow2(grid->n[l])) return LLG_ERR_UNSUPPORTED_SIZE;
        if (!(grid->L[l] > 0) || !std::isfinite(grid->L[l])) return LLG_ERR_INVALID_ARG;
    }
    llg_ctx *c = new (std::nothrow) llg_ctx();
    if (!c) return LLG_ERR_OOM;
    c->grid = *grid;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    SpecGeom &g = c->geo;
    g.dim = grid->dim;
    for (int l = 0; l < 3; ++l) {
        g.n[l] = l < grid->dim ? grid->n[l] : 1;
        g.logn[l] = ilog2(g.n[l]);
    }
    g.N = (long long)g.n[0] * g.n[1] * g.n[2];
    g.rows = (long long)g.n[1] * g.n[2];
    g.S = ((g.n[0] + g.n[0] / 2 + 1) + 15) / 16 * 16;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    auto fail = [&](cudaError_t err, const char *what) {
        llg_status s = cuda_check(c, err, what);
        llg_destroy(c);
        return s;
    };
    if (e != cudaSuccess) return fail(e, "device query");
    // twiddle and symbol tables
    for (int l = 0; l < 3; ++l) {
        const int n = g.n[l];
        std::vector<double2> t64(n);
        std::vector<float2> t32(n);
        std::vector<double> s64[2];
        std::vector<float> s32[2];
        for (int ex = 0; ex < 2; ++ex) { s64[ex].resize(n); s32[ex].resize(n); }
        const long double twopi = 6.283185307179586476925286766559L;
        for (int i = 0; i < n; ++i) {
            const long double ang = twopi * (long double)i / (long double)n;
            t64[i] = make_double2((double)cosl(ang), (double)-sinl(ang));
            t32[i] = make_float2((float)cosl(ang), (float)-sinl(ang));
            const int kw = i < n / 2 ? i : i - n;
            double sp = 0.0, fd = 0.0;
            if (l < grid->dim && n > 1) {
                const long double xi = twopi * (long double)kw / (long double)grid->L[l];
                sp = (double)(xi * xi);
                const long double h = (long double)grid->L[l] / (long double)n;
                const long double sn = sinl(3.14159265358979323846264338327950L * (long double)kw / (long double)n);
                fd = (double)(4.0L / (h * h) * sn * sn);
            }
            s64[0][i] = sp; s64[1][i] = fd;
            s32[0][i] = (float)sp; s32[1][i] = (float)fd;
        }
        // FP32 pairs: hi = the value rounded to FP32, lo = the rest rounded to FP32
        std::vector<cfpair> tp(n);
        std::vector<fpair> sp2[2];
        for (int i = 0; i < n; ++i) {
            const long double ang = twopi * (long double)i / (long double)n;
            const long double cr = cosl(ang), ci = -sinl(ang);
            tp[i].x = fpair((float)cr, (float)(cr - (long double)(float)cr));
            tp[i].y = fpair((float)ci, (float)(ci - (long double)(float)ci));
        }
        for (int ex = 0; ex < 2; ++ex) {
            sp2[ex].resize(n);
            for (int i = 0; i < n; ++i) sp2[ex][i] = fpair(s64[ex][i]);
        }
        if ((e = cudaMalloc(&c->twp[l], sizeof(cfpair) * n)) != cudaSuccess) return fail(e, "tables");
        cudaMemcpy(c->twp[l], tp.data(), sizeof(cfpair) * n, cudaMemcpyHostToDevice);
        for (int ex = 0; ex < 2; ++ex) {
            if ((e = cudaMalloc(&c->sigp[ex][l], sizeof(fpair) * n)) != cudaSuccess) return fail(e, "tables");
            cudaMemcpy(c->sigp[ex][l], sp2[ex].data(), sizeof(fpair) * n, cudaMemcpyHostToDevice);
        }
        if ((e = cudaMalloc(&c->tw64[l], sizeof(double2) * n)) != cudaSuccess) return fail(e, "tables");
        if ((e = cudaMalloc(&c->tw32[l], sizeof(float2) * n)) != cudaSuccess) return fail(e, "tables");
        cudaMemcpy(c->tw64[l], t64.data(), sizeof(double2) * n, cudaMemcpyHostToDevice);
        cudaMemcpy(c->tw32[l], t32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
        for (int ex = 0; ex < 2; ++ex) {
            if ((e = cudaMalloc(&c->sig64[ex][l], sizeof(double) * n)) != cudaSuccess) return fail(e, "tables");
            if ((e = cudaMalloc(&c->sig32[ex][l], sizeof(float) * n)) != cudaSuccess) return fail(e, "tables");
            cudaMemcpy(c->sig64[ex][l], s64[ex].data(), sizeof(double) * n, cudaMemcpyHostToDevice);
            cudaMemcpy(c->sig32[ex][l], s32[ex].data(), sizeof(float) * n, cudaMemcpyHostToDevice);
        }
    }
    if ((e = cudaMalloc(&c->red, sizeof(double) * RB_STRIDE * partial_capacity(c))) != cudaSuccess) return fail(e, "scratch");
    if ((e = cudaMalloc(&c->dsc, sizeof(double) * 64)) != cudaSuccess) return fail(e, "scratch");
    if ((e = cudaMallocHost(&c->hsc, sizeof(double) * 64)) != cudaSuccess) return fail(e, "pinned scratch");
    if ((e = cudaMalloc(&c->gdev, sizeof(GmresDev))) != cudaSuccess) return fail(e, "GMRES state");
    if ((e = cudaMemset(c->gdev, 0, sizeof(GmresDev))) != cudaSuccess) return fail(e, "GMRES state");
    if ((e = cudaMallocHost(&c->ghost, sizeof(GmresDev))) != cudaSuccess) return fail(e, "pinned GMRES state");
    {
        // progress words the Arnoldi kernels write straight into host memory, so the host can
        // follow a cycle without synchronising the stream; without mapped memory it polls
        void *hp = nullptr;
        int *dp = nullptr;
        const char *poll = getenv("LLG_HOST_POLL");
        const bool want = !(poll && strcmp(poll, "1") == 0);
        if (want && cudaHostAlloc(&hp, 64, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer((void **)&dp, hp, 0) == cudaSuccess) {
            memset(hp, 0, 64);
            c->hprog = static_cast<volatile int *>(hp);
            c->dprog = dp;
            volatile int *dpv = dp;
            if ((e = cudaMemcpy(&c->gdev->prog, &dpv, sizeof(dpv), cudaMemcpyHostToDevice)) != cudaSuccess)
                return fail(e, "GMRES progress words");
        } else {
            if (hp) cudaFreeHost(hp);
            cudaGetLastError();
        }
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "create");
    *out = c;
    return LLG_OK;
}

llg_status llg_destroy(llg_ctx *c) {
    if (!c) return LLG_ERR_INVALID_ARG;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (int l = 0; l < 3; ++l) {
        cudaFree(c->tw64[l]);
        cudaFree(c->tw32[l]);
        cudaFree(c->twp[l]);
        for (int ex = 0; ex < 2; ++ex) { cudaFree(c->sig64[ex][l]); cudaFree(c->sig32[ex][l]); cudaFree(c->sigp[ex][l]); }
    }
    cudaFree(c->spec64); cudaFree(c->spec32); cudaFree(c->red); cudaFree(c->dsc);
    cudaFree(c->gdev); cudaFree(c->m32); cudaFree(c->aux); cudaFree(c->dem_tab);
    for (auto &e : c->prof) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    if (c->hsc) cudaFreeHost(c->hsc);
    if (c->ghost) cudaFreeHost(c->ghost);
    if (c->hprog) cudaFreeHost((void *)c->hprog);
    Workspace &w = c->ws;
    cudaFree(w.V); cudaFree(w.Z); cudaFree(w.W); cudaFree(w.T); cudaFree(w.R);
    cudaGetLastError();
    delete c;
    return LLG_OK;
}

const char *llg_last_error(const llg_ctx *c) { return c ? c->err.c_str() : "null context"; }

llg_status llg_autotune(llg_ctx *c, int precision_mask, char *report, int report_len) {
    LLG_GUARD(c);
    if (precision_mask < 1 || precision_mask > 3) return set_error(c, LLG_ERR_INVALID_ARG, "precision_mask must be 1, 2 or 3");
    llg_status st = ensure_spec(c, (precision_mask & 1) != 0, (precision_mask & 2) != 0);
    if (st != LLG_OK) return st;
    std::string rep;
    st = llg::autotune(c, precision_mask, &rep);
    if (report && report_len > 0) {
        std::strncpy(report, rep.c_str(), (size_t)report_len - 1);
        report[report_len - 1] = 0;
    }
    return st;
}

llg_status llg_set_axis_shape(llg_ctx *c, int fp32, int slot, int kind, int E, int TW, int CB) {
    LLG_GUARD(c);
    return llg::set_axis_shape(c, fp32, slot, ColCfg{kind, E, TW, CB});
}

llg_status llg_profile_begin(llg_ctx *c, int kernel_class) {
    LLG_GUARD(c);
    if (kernel_class < LLG_KCLASS_NONE || kernel_class > LLG_KCLASS_ARNOLDI)
        return set_error(c, LLG_ERR_INVALID_ARG, "unknown kernel class");
    c->prof_class = kernel_class;
    c->prof_used = 0;
    c->prof_open = -1;
    return LLG_OK;
}

llg_status llg_profile_end(llg_ctx *c, double *total_ms, long long *launches, double *bytes, double *flops) {
    LLG_GUARD(c);
    llg_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "profile sync");
    if (st != LLG_OK) return st;
    double ms = 0.0, by = 0.0, fl = 0.0;
    long long n = 0;
    for (size_t i = 0; i < c->prof_used; ++i) {
        const llg_ctx::ProfEntry &e = c->prof[i];
        if (!e.valid) continue;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, e.a, e.b) != cudaSuccess) { cudaGetLastError(); continue; }
        ms += t;
        by += e.bytes;
        fl += e.flops;
        n += e.count;
    }
    c->prof_class = 0;
    c->prof_used = 0;
    if (total_ms) *total_ms = ms;
    if (launches) *launches = n;
    if (bytes) *bytes = by;
    if (flops) *flops = fl;
    return LLG_OK;
}

llg_status llg_set_pass_plan(llg_ctx *c, int plan) {
    LLG_GUARD(c);
    if (plan != LLG_PLAN_FIVE && plan != LLG_PLAN_CLUSTER) return set_error(c, LLG_ERR_INVALID_ARG, "unknown pass plan");
    c->pass_plan = plan;
    return LLG_OK;
}

llg_status llg_krylov_orthogonality(llg_ctx *c, double *max_dev, int *nvec) {
    LLG_GUARD(c);
    if (!max_dev || !nvec) return set_error(c, LLG_ERR_INVALID_ARG, "null pointer");
    return krylov_orthogonality(c, max_dev, nvec);
}

llg_status llg_probe_fma_rate(llg_ctx *c, int fp64, double *tflops) {
    LLG_GUARD(c);
    if (!tflops) return set_error(c, LLG_ERR_INVALID_ARG, "null pointer");
    const int blocks = c->sm_count * 8, threads = 256, iters = fp64 ? 4000 : 40000;
    void *out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * 8);
    if (e != cudaSuccess) return cuda_check(c, e, "probe buffer");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
        cudaEventRecord(e0, c->stream);
        if (fp64) k_fma_probe<double><<<blocks, threads, 0, c->stream>>>((double *)out, iters);
        else k_fma_probe<float><<<blocks, threads, 0, c->stream>>>((float *)out, iters);
        cudaEventRecord(e1, c->stream);
    }
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    c->launches += 2;
    if (e != cudaSuccess) return cuda_check(c, e, "probe");
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    return LLG_OK;
}

llg_status llg_check_conversions(llg_ctx *c, long long n_doubles, long long *f2d_mismatches,
                                 long long *d2f_mismatches) {
    LLG_GUARD(c);
    if (!f2d_mismatches || !d2f_mismatches || n_doubles < 0) return set_error(c, LLG_ERR_INVALID_ARG, "bad argument");
    unsigned long long *bad = nullptr;
    cudaError_t e = cudaMalloc(&bad, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_check(c, e, "conversion check buffer");
    e = cudaMemsetAsync(bad, 0, 2 * sizeof(unsigned long long), c->stream);
    const int blocks = c->sm_count * 16, threads = 256;
    const unsigned long long slice = 1ull << 30;   // all 2^32 float patterns in four launches
    for (unsigned long long first = 0; e == cudaSuccess && first < (1ull << 32); first += slice) {
        k_conv_check_f2d<<<blocks, threads, 0, c->stream>>>(first, slice, bad);
        e = cudaGetLastError();
        c->launches++;
    }
    if (e == cudaSuccess && n_doubles > 0) {
        k_conv_check_d2f<<<blocks, threads, 0, c->stream>>>(0x5EEDull, (unsigned long long)n_doubles, bad);
        e = cudaGetLastError();
        c->launches++;
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, bad, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(bad);
    if (e != cudaSuccess) return cuda_check(c, e, "conversion check");
    *f2d_mismatches = (long long)h[0];
    *d2f_mismatches = (long long)h[1];
    return LLG_OK;
}

llg_status llg_set_stream(llg_ctx *c, void *stream) {
    LLG_GUARD(c);
    c->stream = static_cast<cudaStream_t>(stream);
    return LLG_OK;
}

long long llg_launch_count(const llg_ctx *c) { return c ? c->launches : 0; }
long long llg_nodes(const llg_ctx *c) { return c ? c->geo.N : 0; }

llg_status llg_saddle_apply(llg_ctx *c, const llg_params *p, const double *m, const double *x, double *y, int transpose) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st != LLG_OK) return st;
    if (!m || !x || !y) return set_error(c, LLG_ERR_INVALID_ARG, "null array");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    return op_matvec64(c, p, p->theta, m, x, nullptr, y, transpose);
}

llg_status llg_saddle_apply_f32x2(llg_ctx *c, const llg_params *p, const double *m, const double *x, double *y,
                                  int transpose) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st != LLG_OK) return st;
    if (!m || !x || !y) return set_error(c, LLG_ERR_INVALID_ARG, "null array");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    if (!pair_chains_available(c)) return set_error(c, LLG_ERR_UNSUPPORTED_SIZE, "FP32-pair chain: axis length outside 64..1024");
    return op_matvec_pair(c, p, p->theta, m, x, y, transpose);
}

llg_status llg_ffthss_apply(llg_ctx *c, const llg_params *p, const double *m, const double *pin, double *z, int transpose) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st != LLG_OK) return st;
    if (!m || !pin || !z) return set_error(c, LLG_ERR_INVALID_ARG, "null array");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    return op_apply64(c, p, p->theta, m, pin, nullptr, z, transpose);
}

llg_status llg_ffthss_apply_f32(llg_ctx *c, const llg_params *p, const float *m, const float *pin, float *z, int transpose) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st != LLG_OK) return st;
    if (!m || !pin || !z) return set_error(c, LLG_ERR_INVALID_ARG, "null array");
    if ((st = ensure_spec(c, false, true)) != LLG_OK) return st;
    auto io = make_io<float, float, float>(m, pin, z, nullptr, p->lambda);
    Symbol sym = sym_shifted_inverse(c, p, p->theta);
    if (!transpose) return spectral_chain<float, float, float>(c, IN_V, OUT_APPLY, io, sym);
    return spectral_chain<float, float, float>(c, IN_NODAL_T, OUT_PLAIN, io, sym);
}

llg_status llg_precond_saddle_apply(llg_ctx *c, const llg_params *p, const double *m, const double *x, double *z) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st != LLG_OK) return st;
    if (!m || !x || !z) return set_error(c, LLG_ERR_INVALID_ARG, "null array");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    return op_fused64(c, p, p->theta, m, x, nullptr, z);
}

llg_status llg_gmres_solve(llg_ctx *c, const llg_params *p, const llg_opts *o, const double *m, const double *b,
                           double *x, llg_info *info) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st == LLG_OK) st = check_opts(c, o);
    if (st != LLG_OK) return st;
    if (!m || !b || !x) return set_error(c, LLG_ERR_INVALID_ARG, "null array");
    llg_info inf = llg_info();
    st = solve(c, p, p->theta, o, m, b, x, &inf);
    inf.status = st;
    if (info) *info = inf;
    return st;
}

llg_status llg_energy(llg_ctx *c, const llg_params *p, const double *m, double *out) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st != LLG_OK) return st;
    if (!m || !out) return set_error(c, LLG_ERR_INVALID_ARG, "null pointer");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    if ((st = ensure_aux(c)) != LLG_OK) return st;
    if ((st = energy_async(c, p, m, c->aux, c->dsc)) != LLG_OK) return st;
    if ((st = sync_scalars(c, 1)) != LLG_OK) return st;
    *out = c->hsc[0] / (double)c->geo.N;
    return LLG_OK;
}

// h = h_ext + per-node part of h_low(m)
__global__ void k_add_uniform3(const double *__restrict__ hf, double h0, double h1, double h2, double *h, long long N) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        h[j] = h0 + (hf ? hf[j] : 0.0);
        h[N + j] = h1 + (hf ? hf[N + j] : 0.0);
        h[2 * N + j] = h2 + (hf ? hf[2 * N + j] : 0.0);
    }
}

llg_status llg_lower_order_field(llg_ctx *c, const llg_params *p, const double *m, double *h) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st != LLG_OK) return st;
    if (!m || !h) return set_error(c, LLG_ERR_INVALID_ARG, "null pointer");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    if ((st = ensure_aux(c)) != LLG_OK) return st;
    const double *hf = nullptr;
    if ((st = lowfield_nodal(c, p, m, c->aux + 18 * c->geo.N, &hf)) != LLG_OK) return st;
    k_add_uniform3<<<grid_blocks(c), RB_THREADS, 0, c->stream>>>(hf, p->h_ext[0], p->h_ext[1], p->h_ext[2], h, c->geo.N);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "lower-order field");
}

llg_status llg_step_euler(llg_ctx *c, const llg_params *p, const llg_opts *o, const double *m_n, double *m_next,
                          double *x_out, llg_info *info) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st == LLG_OK) st = check_opts(c, o);
    if (st != LLG_OK) return st;
    if (!m_n || !m_next || !x_out) return set_error(c, LLG_ERR_INVALID_ARG, "null array");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    if ((st = ensure_aux(c)) != LLG_OK) return st;
    const long long N = c->geo.N;
    double *b = c->aux;            // 4N
    double *tmp = c->aux + 4 * N;  // 4N
    llg_info inf = llg_info();
    if (o->diagnostics) {
        if ((st = energy_async(c, p, m_n, tmp, c->dsc + 8)) != LLG_OK) return st;
    }
    const double *hf = nullptr;
    if ((st = lowfield_nodal(c, p, m_n, c->aux + 18 * N, &hf)) != LLG_OK) return st;
    if ((st = rhs_velocity(c, p, o, m_n, hf, b)) != LLG_OK) return st;
    cudaMemsetAsync(x_out, 0, sizeof(double) * 4 * N, c->stream);
    st = solve(c, p, 1.0, o, m_n, b, x_out, &inf);
    if (st != LLG_OK && st != LLG_ERR_NOT_CONVERGED) { inf.status = st; if (info) *info = inf; return st; }
    llg_status solve_st = st;
    const int nb = reduction_blocks(c);
    k_euler_update<<<nb, RB_THREADS, 0, c->stream>>>(m_n, x_out, p->k, m_next, N, c->red);
    k_max_partials<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, c->dsc + 9);
    c->launches += 2;
    if ((st = cuda_check(c, cudaGetLastError(), "euler update")) != LLG_OK) return st;
    if (o->diagnostics) {
        if ((st = energy_async(c, p, m_next, tmp, c->dsc + 10)) != LLG_OK) return st;
    }
    if ((st = sync_scalars(c, 11)) != LLG_OK) return st;
    inf.max_len_drift = c->hsc[9];
    if (o->diagnostics) {
        inf.energy_before = c->hsc[8] / (double)N;
        inf.energy_after = c->hsc[10] / (double)N;
    }
    inf.picard_iters = 1;
    inf.status = solve_st;
    if (info) *info = inf;
    return solve_st;
}

// device scalar that holds ||b||^2 across the solves of a midpoint step
constexpr int kBnormSlot = 4;

llg_status llg_step_midpoint(llg_ctx *c, const llg_params *p, const llg_opts *o, const double *m_n, const double *v_prev,
                             double *m_next, double *x_out, llg_info *info) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st == LLG_OK) st = check_opts(c, o);
    if (st != LLG_OK) return st;
    if (!m_n || !m_next || !x_out) return set_error(c, LLG_ERR_INVALID_ARG, "null array");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    if ((st = ensure_aux(c)) != LLG_OK) return st;
    const long long N = c->geo.N;
    double *b = c->aux;                // 4N
    double *vold = c->aux + 4 * N;     // 3N
    double *mhat = c->aux + 7 * N;     // 3N
    double *tmp = c->aux + 10 * N;     // 4N
    double *r0 = c->aux + 14 * N;      // 4N
    const int nb = reduction_blocks(c), gb = grid_blocks(c);
    llg_info inf = llg_info();
    if (o->diagnostics) {
        if ((st = energy_async(c, p, m_n, tmp, c->dsc + 8)) != LLG_OK) return st;
    }
    // exchange at m^n, lower-order field at the midpoint field mhat (eq. (hatm))
    const bool mdep = field_depends_on_m(p);
    double *hfbuf = c->aux + 18 * N;   // 3N
    const double *hf = nullptr;
    k_axpy3<<<gb, RB_THREADS, 0, c->stream>>>(m_n, v_prev, 0.5 * p->k, mhat, 3 * N);
    if ((st = lowfield_nodal(c, p, mhat, hfbuf, &hf)) != LLG_OK) return st;
    if ((st = rhs_velocity(c, p, o, m_n, hf, b)) != LLG_OK) return st;
    // ||b||^2 once for the step's solves (device scalar kBnormSlot)
    if ((st = dot_async(c, b, b, 4 * N, c->dsc + kBnormSlot)) != LLG_OK) return st;
    // warm start (v_prev | 0), or zero
    if (v_prev) cudaMemcpyAsync(x_out, v_prev, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, c->stream);
    else cudaMemsetAsync(x_out, 0, sizeof(double) * 3 * N, c->stream);
    cudaMemsetAsync(x_out + 3 * N, 0, sizeof(double) * N, c->stream);
    c->launches++;
    llg_status lin_st = LLG_OK;
    bool conv = false;
    bool have_r0 = false;
    for (int it = 0; it < o->picard_max; ++it) {
        llg_info si = llg_info();
        st = solve(c, p, 0.5, o, mhat, b, x_out, &si, have_r0 ? r0 : nullptr, have_r0, kBnormSlot);
        inf.iters += si.iters;
        inf.restarts += si.restarts;
        inf.applies += si.applies;
        inf.rel_res_true = std::max(inf.rel_res_true, si.rel_res_true);
        inf.picard_iters = it + 1;
        if (st == LLG_ERR_NOT_CONVERGED) lin_st = st;
        else if (st != LLG_OK) { inf.status = st; if (info) *info = inf; return st; }
        if (it >= 1) {
            // the stopping test's norms, and vold = v in the same pass
            if ((((uintptr_t)x_out | (uintptr_t)vold) & 15u) == 0)
                k_picard_norms_advance<true><<<nb, RB_THREADS, 0, c->stream>>>(x_out, vold, 3 * N, c->red);
            else
                k_picard_norms_advance<false><<<nb, RB_THREADS, 0, c->stream>>>(x_out, vold, 3 * N, c->red);
            k_sum_partials_n<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, 2, c->dsc);
            c->launches += 2;
            if ((st = sync_scalars(c, 2)) != LLG_OK) return st;
            if (std::sqrt(c->hsc[0]) <= o->picard_tol * std::sqrt(c->hsc[1])) { conv = true; break; }
        } else {
            cudaMemcpyAsync(vold, x_out, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, c->stream);
        }
        if (mdep) {
            // the right-hand side moves with mhat: rebuild it, solve from the true residual
            k_axpy3<<<gb, RB_THREADS, 0, c->stream>>>(m_n, x_out, 0.5 * p->k, mhat, 3 * N);
            c->launches++;
            if ((st = lowfield_nodal(c, p, mhat, hfbuf, &hf)) != LLG_OK) return st;
            if ((st = rhs_velocity(c, p, o, m_n, hf, b)) != LLG_OK) return st;
            if ((st = dot_async(c, b, b, 4 * N, c->dsc + kBnormSlot)) != LLG_OK) return st;
            have_r0 = false;
            continue;
        }
        if (c->ws.last_res) {
            // the last solve's final true residual, advanced in place (it is the next solve's
            // first residual and first basis vector), its squared norm into device scalar 2
            double *res = const_cast<double *>(c->ws.last_res);
            k_picard_advance<<<nb, RB_THREADS, 0, c->stream>>>(m_n, x_out, 0.5 * p->k, mhat, res, N, c->red);
            k_sum_partials_n<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, 1, c->dsc + 2);
            c->launches++;
            r0 = res;
            have_r0 = true;
        } else {
            k_axpy3<<<gb, RB_THREADS, 0, c->stream>>>(m_n, x_out, 0.5 * p->k, mhat, 3 * N);
            have_r0 = false;
        }
        c->launches++;
    }
    k_mid_final<<<nb, RB_THREADS, 0, c->stream>>>(m_n, x_out, p->k, m_next, N, c->red);
    k_max_partials<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, c->dsc + 9);
    c->launches += 2;
    if ((st = cuda_check(c, cudaGetLastError(), "midpoint update")) != LLG_OK) return st;
    if (o->diagnostics) {
        if ((st = energy_async(c, p, m_next, tmp, c->dsc + 10)) != LLG_OK) return st;
        if ((st = dot_async(c, x_out, x_out, 3 * N, c->dsc + 11)) != LLG_OK) return st;
    }
    if ((st = sync_scalars(c, 12)) != LLG_OK) return st;
    inf.max_len_drift = c->hsc[9];
    if (o->diagnostics) {
        inf.energy_before = c->hsc[8] / (double)N;
        inf.energy_after = c->hsc[10] / (double)N;
        const double v2 = c->hsc[11] / (double)N;
        inf.dissipation_residual = inf.energy_after - inf.energy_before + p->alpha * p->k / (1.0 + p->alpha * p->alpha) * v2;
    }
    llg_status res = lin_st != LLG_OK ? lin_st : (conv ? LLG_OK : LLG_ERR_NOT_CONVERGED);
    if (res == LLG_ERR_NOT_CONVERGED && c->err.empty()) set_error(c, res, "Picard iteration reached picard_max");
    inf.status = res;
    if (info) *info = inf;
    return res;
}

llg_status llg_adjoint_step(llg_ctx *c, const llg_params *p, const llg_opts *o, const double *m_n, const double *x,
                            const double *mbar_next, double *mbar_n, double *dalpha, double dh[3], llg_info *info) {
    LLG_GUARD(c);
    llg_status st = check_params(c, p);
    if (st == LLG_OK) st = check_opts(c, o);
    if (st != LLG_OK) return st;
    if (!m_n || !x || !mbar_next || !mbar_n || !dalpha || !dh) return set_error(c, LLG_ERR_INVALID_ARG, "null pointer");
    if (field_depends_on_m(p))
        return set_error(c, LLG_ERR_INVALID_ARG, "the adjoint covers exchange and applied fields (no demag or anisotropy)");
    if ((st = ensure_spec(c, true, false)) != LLG_OK) return st;
    if ((st = ensure_aux(c)) != LLG_OK) return st;
    const long long N = c->geo.N;
    double *y = c->aux;               // 4N
    double *mhat = c->aux + 4 * N;    // 3N
    double *rhs = c->aux + 7 * N;     // 4N
    double *lapy = c->aux + 11 * N;   // 4N (3 used)
    double *u = c->aux + 15 * N;      // 3N
    double *lapu = c->aux + 18 * N;   // 4N (3 used)
    const int nb = reduction_blocks(c), gb = grid_blocks(c);
    const double hk = 0.5 * p->k;
    k_adj_prep<<<gb, RB_THREADS, 0, c->stream>>>(m_n, x, mbar_next, p->k, p->alpha * p->c_ex, mhat, rhs, u, N);
    cudaMemsetAsync(y, 0, sizeof(double) * 4 * N, c->stream);
    c->launches++;
    if ((st = check_nodes(c, mhat)) != LLG_OK) return st;
    // J^T and the transposed preconditioner M(mhat)^{-T}
    Symbol fwd = sym_forward(c, p, 0.5);
    Symbol inv = sym_shifted_inverse(c, p, 0.5);
    auto jt = [=](const double *xx, const double *s, double *yy) {
        auto io = make_io<double, double, double>(mhat, xx, yy, s, p->lambda);
        io.mn = m_n; io.vf = x; io.half_k = hk;
        return spectral_chain<double, double, double>(c, IN_V, OUT_JT, io, fwd);
    };
    auto pt = [=](const double *xx, const double *s, double *yy) {
        auto io = make_io<double, double, double>(mhat, xx, yy, s, p->lambda);
        return spectral_chain<double, double, double>(c, IN_NODAL_T, OUT_PLAIN, io, inv);
    };
    SolveOps ops;
    ops.matvec = [=](const double *xx, double *yy) { return jt(xx, nullptr, yy); };
    ops.prec = pt;
    ops.pop = [=](const double *xx, const double *s, double *yy) {
        llg_status s2 = jt(xx, s, c->ws.R);
        if (s2 != LLG_OK) return s2;
        return pt(c->ws.R, nullptr, yy);
    };
    llg_opts o64 = *o;
    o64.precision = LLG_PREC_FP64;
    llg_info inf = llg_info();
    llg_status solve_st = gmres_run(c, ops, false, &o64, rhs, y, &inf);
    if (solve_st != LLG_OK && solve_st != LLG_ERR_NOT_CONVERGED) { inf.status = solve_st; if (info) *info = inf; return solve_st; }
    inf.applies *= 2;
    // Chat (-Lap) y_v and (-Lap) u
    {
        auto io = make_io<double, double, double>(mhat, y, lapy, nullptr, p->lambda);
        Symbol s{0.0, chat(p), 1.0 / (double)N, 0, p->exchange};
        if ((st = spectral_chain<double, double, double>(c, IN_V, OUT_PLAIN, io, s)) != LLG_OK) return st;
        auto io2 = make_io<double, double, double>(mhat, u, lapu, nullptr, p->lambda);
        Symbol s2{0.0, 1.0, 1.0 / (double)N, 0, p->exchange};
        if ((st = spectral_chain<double, double, double>(c, IN_V, OUT_PLAIN, io2, s2)) != LLG_OK) return st;
    }
    k_adj_final<<<nb, RB_THREADS, 0, c->stream>>>(mbar_next, y, lapy, x, lapu, p->alpha, p->h_ext[0], p->h_ext[1],
                                                  p->h_ext[2], p->h_field, mbar_n, N, c->red);
    k_sum_partials_n<<<1, RB_THREADS, 0, c->stream>>>(c->red, nb, 4, c->dsc);
    c->launches += 2;
    if ((st = cuda_check(c, cudaGetLastError(), "adjoint")) != LLG_OK) return st;
    if ((st = sync_scalars(c, 4)) != LLG_OK) return st;
    const double s = 1.0 + p->alpha * p->alpha;
    *dalpha += c->hsc[0];
    for (int q = 0; q < 3; ++q) dh[q] += s * c->hsc[1 + q];
    inf.status = solve_st;
    if (info) *info = inf;
    return solve_st;
}

}  // extern "C"
