// spectral.cu -- the Fourier round trip at the heart of every operator of the
// library, as three (2D) or five (3D) bandwidth-bound passes over HBM:
//
//   x-pass forward : nodal prologue (what to transform: v, m x v + m r - lambda v,
//                    m, or the transposed nodal solve) -> FFT along x of the packed
//                    pair (c1 + i c2) per row and of c3 for two rows at a time,
//                    split into two half spectra (real-input symmetry)
//   y-pass [3D]    : FFT along y
//   last axis      : FFT, pointwise real even multiplier (the shifted exchange symbol
//                    of Algorithm 1, or its non-inverted form for the matvec), inverse FFT
//   y-pass [3D]    : inverse FFT along y
//   x-pass inverse : inverse FFT along x -> nodal epilogue (closed-form 4x4 inverse of
//                    eq. (inverse S), saddle matvec, ...), written as SoA planes.
//
// Because the multiplier is real and even, the operator maps real fields to real
// fields and is complex-linear, so c1 and c2 share one complex transform; c3 is
// transformed two rows at a time and stored as a half spectrum.
#include "spectral_kernels.cuh"

namespace llg {

// ------------------------------------------------------------------ launch plumbing

template <typename T> static const cplx<T> *tw_of(llg_ctx *c, int axis);
template <> const double2 *tw_of<double>(llg_ctx *c, int axis) { return c->tw64[axis]; }
template <> const float2 *tw_of<float>(llg_ctx *c, int axis) { return c->tw32[axis]; }
template <typename T> static const T *sig_of(llg_ctx *c, int ex, int axis);
template <> const double *sig_of<double>(llg_ctx *c, int ex, int axis) { return c->sig64[ex][axis]; }
template <> const float *sig_of<float>(llg_ctx *c, int ex, int axis) { return c->sig32[ex][axis]; }
template <typename T> static cplx<T> *spec_of(llg_ctx *c);
template <> double2 *spec_of<double>(llg_ctx *c) { return c->spec64; }
template <> float2 *spec_of<float>(llg_ctx *c) { return c->spec32; }

template <typename T, typename TIn, typename TOut, int E>
static cudaError_t launch_row_fwd_E(llg_ctx *c, int in_mode, RowArgs<T, TIn, TOut> a, int blocks, int threads, size_t sm) {
#define LLG_RF(MODE)                                                                          \
    case MODE: {                                                                              \
        auto k = row_fwd_kernel<T, TIn, TOut, E, MODE>;                                       \
        cudaError_t e = set_smem(k, sm);                                                      \
        if (e != cudaSuccess) return e;                                                       \
        k<<<blocks, threads, sm, c->stream>>>(a);                                             \
        return cudaGetLastError();                                                            \
    }
    switch (in_mode) {
        LLG_RF(IN_V) LLG_RF(IN_FUSED) LLG_RF(IN_M) LLG_RF(IN_NODAL_T)
    }
#undef LLG_RF
    return cudaErrorInvalidValue;
}

template <typename T, typename TIn, typename TOut, int E>
static cudaError_t launch_row_inv_E(llg_ctx *c, int out_mode, RowArgs<T, TIn, TOut> a, int blocks, int threads, size_t sm) {
#define LLG_RI(MODE)                                                                          \
    case MODE: {                                                                              \
        auto k = row_inv_kernel<T, TIn, TOut, E, MODE>;                                       \
        cudaError_t e = set_smem(k, sm);                                                      \
        if (e != cudaSuccess) return e;                                                       \
        k<<<blocks, threads, sm, c->stream>>>(a);                                             \
        return cudaGetLastError();                                                            \
    }
    switch (out_mode) {
        LLG_RI(OUT_APPLY) LLG_RI(OUT_FUSED) LLG_RI(OUT_MATVEC) LLG_RI(OUT_FIELD) LLG_RI(OUT_PLAIN) LLG_RI(OUT_JT)
    }
#undef LLG_RI
    return cudaErrorInvalidValue;
}

template <typename T, int E, int TW>
static cudaError_t launch_col_ETW(llg_ctx *c, int mode, const ColArgs<T> &a, dim3 grid) {
    size_t sm = (size_t)a.nl * TW * sizeof(cplx<T>);
    int threads = TW * (a.nl / E);
#define LLG_CK(MODE)                                                                          \
    case MODE: {                                                                              \
        auto k = col_kernel<T, E, TW, MODE>;                                                  \
        cudaError_t e = set_smem(k, sm);                                                      \
        if (e != cudaSuccess) return e;                                                       \
        k<<<grid, threads, sm, c->stream>>>(a);                                               \
        return cudaGetLastError();                                                            \
    }
    switch (mode) {
        LLG_CK(1) LLG_CK(2) LLG_CK(7)
    }
#undef LLG_CK
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_col(llg_ctx *c, int mode, const ColArgs<T> &a, dim3 grid) {
    ColPlan p = col_plan<T>(a.nl);
#define LLG_CE(EE, TT) if (p.E == EE && p.TW == TT) return launch_col_ETW<T, EE, TT>(c, mode, a, grid);
    LLG_CE(2, 8) LLG_CE(4, 8) LLG_CE(8, 8) LLG_CE(16, 8)
    LLG_CE(2, 16) LLG_CE(4, 16) LLG_CE(8, 16) LLG_CE(16, 16)
#undef LLG_CE
    return cudaErrorInvalidValue;
}

template <typename T, typename TIn, typename TOut>
llg_status spectral_chain(llg_ctx *c, int in_mode, int out_mode, const NodalIO<TIn, TOut, T> &io,
                          const Symbol &sym) {
    const SpecGeom &g = c->geo;
    const int n0 = g.n[0];
    const int E = row_E(n0), P = n0 / E;
    const long long pairs = g.rows / 2;
    int G = 256 / (3 * P);
    if (G < 1) G = 1;
    long long want = pairs / (2LL * c->sm_count);
    if (want < G) G = (int)(want < 1 ? 1 : want);
    const int blocks = (int)((pairs + G - 1) / G);
    const int threads = 3 * G * P;
    const size_t smr = (size_t)3 * G * RowLayout::size(n0) * sizeof(cplx<T>);

    RowArgs<T, TIn, TOut> ra;
    ra.spec = spec_of<T>(c);
    ra.tw0 = tw_of<T>(c, 0);
    ra.n0 = n0; ra.logn0 = g.logn[0]; ra.S = g.S; ra.G = G;
    ra.rows = g.rows; ra.N = g.N; ra.io = io;

    // algorithmic bytes / flops of each pass (live spectrum only; inputs read and outputs written once)
    const double W = sizeof(T), CB = 2.0 * sizeof(T), Ti = sizeof(TIn), To = sizeof(TOut);
    const double Nd = (double)g.N, live = (double)g.rows * (n0 + n0 / 2 + 1);
    auto fftf = [](double lines, int n, int logn) { return lines * 5.0 * n * logn; };
    double in_b = 3 * Nd * Ti;
    if (in_mode == IN_FUSED) in_b = 3 * Nd * W + 4 * Nd * Ti;
    if (in_mode == IN_NODAL_T) in_b = 3 * Nd * W + 4 * Nd * Ti + Nd * To;
    double out_b = 0;
    switch (out_mode) {
        case OUT_APPLY: out_b = Nd * (3 * W + Ti + 4 * To); break;
        case OUT_FUSED: out_b = Nd * (3 * W + 3 * Ti + 4 * To); break;
        case OUT_MATVEC: out_b = Nd * (3 * W + 4 * Ti + 4 * To); break;
        case OUT_FIELD: out_b = Nd * 4 * To; break;
        case OUT_PLAIN: out_b = Nd * 3 * To; break;
        default: out_b = Nd * (4 * Ti + 7 * W + 4 * To); break;
    }
    const double xf = fftf(1.5 * g.rows, n0, g.logn[0]);

    cudaError_t e;
#define LLG_DISPATCH_E(FN, MODE)                                                              \
    switch (E) {                                                                              \
        case 2: e = FN<T, TIn, TOut, 2>(c, MODE, ra, blocks, threads, smr); break;            \
        case 4: e = FN<T, TIn, TOut, 4>(c, MODE, ra, blocks, threads, smr); break;            \
        case 8: e = FN<T, TIn, TOut, 8>(c, MODE, ra, blocks, threads, smr); break;            \
        default: e = FN<T, TIn, TOut, 16>(c, MODE, ra, blocks, threads, smr); break;          \
    }
    prof_begin(c, K_XFWD, in_b + live * CB, xf);
    LLG_DISPATCH_E(launch_row_fwd_E, in_mode)
    prof_end(c);
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass forward");
    c->launches++;

    ColArgs<T> ca;
    ca.spec = spec_of<T>(c);
    ca.n0 = n0; ca.S = g.S;
    ca.tx = sig_of<T>(c, sym.exchange, 0);
    ca.sa = (T)sym.a; ca.sb = (T)sym.b; ca.sscale = (T)sym.scale; ca.sinv = sym.invert;
    auto tiles = [&](int nl) { return g.S / col_plan<T>(nl).TW; };
    if (g.dim == 2) {
        ca.tw = tw_of<T>(c, 1); ca.nl = g.n[1]; ca.logn = g.logn[1];
        ca.ls = g.S; ca.bs = 0; ca.tl = sig_of<T>(c, sym.exchange, 1); ca.tb = nullptr;
        prof_begin(c, K_AXIS, 2 * live * CB, 2 * fftf((double)(n0 + n0 / 2 + 1), g.n[1], g.logn[1]));
        e = launch_col<T>(c, 7, ca, dim3(tiles(g.n[1]), 1));
        prof_end(c);
        if (e != cudaSuccess) return cuda_check(c, e, "y-pass");
        c->launches++;
    } else {
        ColArgs<T> cy = ca;
        cy.tw = tw_of<T>(c, 1); cy.nl = g.n[1]; cy.logn = g.logn[1];
        cy.ls = g.S; cy.bs = (long long)g.n[1] * g.S; cy.tl = nullptr; cy.tb = nullptr;
        const double ylines = (double)(n0 + n0 / 2 + 1) * g.n[2], zlines = (double)(n0 + n0 / 2 + 1) * g.n[1];
        prof_begin(c, K_AXIS, 2 * live * CB, fftf(ylines, g.n[1], g.logn[1]));
        e = launch_col<T>(c, 1, cy, dim3(tiles(g.n[1]), g.n[2]));
        prof_end(c);
        if (e != cudaSuccess) return cuda_check(c, e, "y-pass forward");
        ColArgs<T> cz = ca;
        cz.tw = tw_of<T>(c, 2); cz.nl = g.n[2]; cz.logn = g.logn[2];
        cz.ls = (long long)g.n[1] * g.S; cz.bs = g.S;
        cz.tl = sig_of<T>(c, sym.exchange, 2); cz.tb = sig_of<T>(c, sym.exchange, 1);
        prof_begin(c, K_AXIS, 2 * live * CB, 2 * fftf(zlines, g.n[2], g.logn[2]));
        e = launch_col<T>(c, 7, cz, dim3(tiles(g.n[2]), g.n[1]));
        prof_end(c);
        if (e != cudaSuccess) return cuda_check(c, e, "z-pass");
        prof_begin(c, K_AXIS, 2 * live * CB, fftf(ylines, g.n[1], g.logn[1]));
        e = launch_col<T>(c, 2, cy, dim3(tiles(g.n[1]), g.n[2]));
        prof_end(c);
        if (e != cudaSuccess) return cuda_check(c, e, "y-pass inverse");
        c->launches += 3;
    }
    prof_begin(c, K_XINV, live * CB + out_b, xf);
    LLG_DISPATCH_E(launch_row_inv_E, out_mode)
    prof_end(c);
#undef LLG_DISPATCH_E
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass inverse");
    c->launches++;
    return LLG_OK;
}

template llg_status spectral_chain<double, double, double>(llg_ctx *, int, int, const NodalIO<double, double, double> &, const Symbol &);
template llg_status spectral_chain<float, double, float>(llg_ctx *, int, int, const NodalIO<double, float, float> &, const Symbol &);
template llg_status spectral_chain<float, float, double>(llg_ctx *, int, int, const NodalIO<float, double, float> &, const Symbol &);
template llg_status spectral_chain<float, float, float>(llg_ctx *, int, int, const NodalIO<float, float, float> &, const Symbol &);

}  // namespace llg
