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
#include <vector>
#include <string>
#include <cstdio>
#include <algorithm>
#include "spectral_kernels.cuh"
#include "spectral_ct_launch.h"
#include "spectral_xy.h"
#include "col_tma.h"

namespace llg {

// ------------------------------------------------------------------ launch plumbing

template <typename T> static const cplx<T> *tw_of(llg_ctx *c, int axis);
template <> const double2 *tw_of<double>(llg_ctx *c, int axis) { return c->tw64[axis]; }
template <> const float2 *tw_of<float>(llg_ctx *c, int axis) { return c->tw32[axis]; }
template <> const cfpair *tw_of<fpair>(llg_ctx *c, int axis) { return c->twp[axis]; }
template <typename T> static const T *sig_of(llg_ctx *c, int ex, int axis);
template <> const double *sig_of<double>(llg_ctx *c, int ex, int axis) { return c->sig64[ex][axis]; }
template <> const float *sig_of<float>(llg_ctx *c, int ex, int axis) { return c->sig32[ex][axis]; }
template <> const fpair *sig_of<fpair>(llg_ctx *c, int ex, int axis) { return c->sigp[ex][axis]; }
template <typename T> static cplx<T> *spec_of(llg_ctx *c);
template <> double2 *spec_of<double>(llg_ctx *c) { return c->spec64; }
template <> float2 *spec_of<float>(llg_ctx *c) { return c->spec32; }
// FP32-pair chains use the FP64 buffer (a complex pair is 16 bytes, as a complex double)
template <> cfpair *spec_of<fpair>(llg_ctx *c) { return reinterpret_cast<cfpair *>(c->spec64); }

bool pair_chains_available(const llg_ctx *c) {
    const SpecGeom &g = c->geo;
    return c->twp[0] != nullptr && c->spec64 != nullptr && ct::covers(g.logn[0]) && ct::covers(g.logn[1]) &&
           (g.dim == 2 || ct::covers(g.logn[2]));
}

template <typename T, typename TIn, typename TOut, int E>
static cudaError_t launch_row_fwd_E(llg_ctx *c, int in_mode, RowArgs<T, TIn, TOut> a, int blocks, int threads, size_t sm) {
#define LLG_RF(MODE)                                                                          \
    case MODE: {                                                                              \
        auto k = row_fwd_kernel<T, TIn, TOut, E, MODE>;                                       \
        cudaError_t e = set_smem(k, sm);                                                      \
        if (e != cudaSuccess) return e;                                                       \
        return launch_pdl(k, dim3(blocks), dim3(threads), sm, c->stream, a);                  \
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
        return launch_pdl(k, dim3(blocks), dim3(threads), sm, c->stream, a);                  \
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
        return launch_pdl(k, dim3(grid), dim3(threads), sm, c->stream, a);                    \
    }
    switch (mode) {
        LLG_CK(1) LLG_CK(2) LLG_CK(7)
    }
#undef LLG_CK
    return cudaErrorInvalidValue;
}

template <int TWL, int CB>
static cudaError_t launch_staged_TW(llg_ctx *c, int mode, const ColArgs<float> &a, int live, int batches) {
    constexpr int SROW = StagedRow<TWL>::value;
    const size_t sm = (size_t)a.nl * SROW * sizeof(float2);
    const int threads = CB * (a.nl / 8);
    const dim3 grid((live + TWL - 1) / TWL, batches);
#define LLG_CS(MODE)                                                                          \
    case MODE: {                                                                              \
        auto k = col_staged_kernel<8, TWL, CB, MODE>;                                         \
        cudaError_t e = set_smem(k, sm);                                                      \
        if (e != cudaSuccess) return e;                                                       \
        return launch_pdl(k, dim3(grid), dim3(threads), sm, c->stream, a, live);              \
    }
    switch (mode) {
        LLG_CS(1) LLG_CS(2) LLG_CS(7)
    }
#undef LLG_CS
    return cudaErrorInvalidValue;
}

// the staged shapes that are compiled: (tile columns, columns per sub-batch)
static const int kStaged[][2] = {{64, 64}, {64, 32}, {64, 16}, {32, 32}, {32, 16}, {32, 8},
                                 {16, 16}, {16, 8},  {16, 4},  {8, 8},   {8, 4}};

static cudaError_t launch_staged(llg_ctx *c, int mode, const ColArgs<float> &a, int live, int batches, int TWL, int CB) {
#define LLG_ST(X, Y) if (TWL == X && CB == Y) return launch_staged_TW<X, Y>(c, mode, a, live, batches);
    LLG_ST(64, 64) LLG_ST(64, 32) LLG_ST(64, 16) LLG_ST(32, 32) LLG_ST(32, 16) LLG_ST(32, 8)
    LLG_ST(16, 16) LLG_ST(16, 8) LLG_ST(16, 4) LLG_ST(8, 8) LLG_ST(8, 4)
#undef LLG_ST
    return cudaErrorInvalidValue;
}

static int ilog2_int(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
template <typename T> static int col_E(int nl) { return (sizeof(T) == 4 && nl >= 1024) ? 16 : (nl >= 8 ? 8 : nl); }

// every launch shape the tuner may pick for a line length
template <typename T> static std::vector<ColCfg> col_candidates(const llg_ctx *c, int nl) {
    std::vector<ColCfg> v;
    const int E = col_E<T>(nl);
    const int tws[] = {4, 8, 16};
    for (int TW : tws) {
        if (sizeof(T) == 4 && TW == 4) continue;
        if (sizeof(T) == 8 && TW == 16) continue;
        if (TW * (nl / E) > 512) continue;
        if ((size_t)nl * TW * sizeof(cplx<T>) > 200 * 1024) continue;
        v.push_back({0, E, TW, 0});
    }
    if (sizeof(T) == 4 && ct::covers(ilog2_int(nl))) {
        // two adjacent columns per thread (16-byte accesses)
        for (int TW : {8, 16})
            if ((TW / 2) * (nl / E) <= 512) v.push_back({3, E, TW, 0});
    }
    if (sizeof(T) == 4 && tma::available(c, nl)) {
        // persistent kernels fed by the tensor memory accelerator
        for (int TW : {8, 16})
            for (int E : {8, 16}) v.push_back({4, E, TW, 0});
    }
    if (sizeof(T) == 4 && nl >= 64) {
        for (auto &sc : kStaged) {
            const int TWL = sc[0], CB = sc[1];
            const int srow = TWL + ((8 - (TWL & 15)) & 15);
            if (CB * (nl / 8) > 512 || CB * (nl / 8) < 64) continue;
            if ((size_t)nl * srow * sizeof(float2) > 160 * 1024) continue;
            v.push_back({1, 8, TWL, CB});
        }
    }
    return v;
}

// untuned default: the register kernel with the widest tile that fits 512 threads
template <typename T> static ColCfg col_default(int nl) {
    const ColPlan p = col_plan<T>(nl);
    return {0, p.E, p.TW, 0};
}

template <typename T>
static cudaError_t launch_col_cfg(llg_ctx *c, int mode, const ColArgs<T> &a, int batches, const ColCfg &cfg) {
    if (cfg.kind == 4) {
        if constexpr (sizeof(T) == 4) return tma::col_launch(c, mode, a, batches, cfg.TW, cfg.E);
        return cudaErrorInvalidValue;
    }
    if (cfg.kind == 1) {
        if constexpr (sizeof(T) == 4) {
            if (ct::covers(a.logn)) return ct::staged(c, a.logn, mode, a, a.n0 + a.n0 / 2 + 1, batches, cfg.TW, cfg.CB);
            return launch_staged(c, mode, a, a.n0 + a.n0 / 2 + 1, batches, cfg.TW, cfg.CB);
        }
        return cudaErrorInvalidValue;
    }
    const dim3 grid(a.S / cfg.TW, batches);
    if (cfg.kind == 3) {
        if constexpr (sizeof(T) == 4) {
            if (ct::covers(a.logn)) return ct::col_v2(c, a.logn, mode, a, grid, cfg.TW);
        }
        return cudaErrorInvalidValue;
    }
    if (ct::covers(a.logn) && cfg.E == col_E<T>(a.nl)) return ct::col<T>(c, a.logn, mode, a, grid, cfg.TW);
#define LLG_CE(EE, TT) if (cfg.E == EE && cfg.TW == TT) return launch_col_ETW<T, EE, TT>(c, mode, a, grid);
    if constexpr (is_fpair<T>::value) {
        return cudaErrorInvalidValue;   // compile-time lengths only
    } else if constexpr (sizeof(T) == 8) {
        LLG_CE(2, 8) LLG_CE(4, 8) LLG_CE(8, 8) LLG_CE(2, 4) LLG_CE(4, 4) LLG_CE(8, 4)
    } else {
        LLG_CE(2, 16) LLG_CE(4, 16) LLG_CE(8, 16) LLG_CE(16, 16) LLG_CE(2, 8) LLG_CE(4, 8) LLG_CE(8, 8) LLG_CE(16, 8)
    }
#undef LLG_CE
    return cudaErrorInvalidValue;
}

template <typename T> static ColCfg slot_cfg(llg_ctx *c, int slot, int nl) {
    // FP32-pair chains: the widest register tile (six blocks of 128 threads per SM)
    if constexpr (is_fpair<T>::value) return col_default<T>(nl);
    const int pi = sizeof(T) == 4 ? 0 : 1;
    return c->tuned[pi] ? c->colcfg[pi][slot] : col_default<T>(nl);
}

// column arguments of one axis-pass slot, with a given multiplier
template <typename T>
static void slot_args(llg_ctx *c, int slot, const Symbol &sym, ColArgs<T> &ca, int &batches, int &mode) {
    const SpecGeom &g = c->geo;
    ca.spec = spec_of<T>(c);
    ca.n0 = g.n[0]; ca.S = g.S;
    ca.tx = sig_of<T>(c, sym.exchange, 0);
    ca.sa = (T)sym.a; ca.sb = (T)sym.b; ca.sscale = (T)sym.scale; ca.sinv = sym.invert;
    ca.tl = nullptr; ca.tb = nullptr;
    if (slot == SLOT_2D) {
        ca.tw = tw_of<T>(c, 1); ca.nl = g.n[1]; ca.logn = g.logn[1]; ca.ls = g.S; ca.bs = 0;
        ca.tl = sig_of<T>(c, sym.exchange, 1);
        batches = 1; mode = 7;
    } else if (slot == SLOT_Z) {
        ca.tw = tw_of<T>(c, 2); ca.nl = g.n[2]; ca.logn = g.logn[2];
        ca.ls = (long long)g.n[1] * g.S; ca.bs = g.S;
        ca.tl = sig_of<T>(c, sym.exchange, 2); ca.tb = sig_of<T>(c, sym.exchange, 1);
        batches = g.n[1]; mode = 7;
    } else {
        ca.tw = tw_of<T>(c, 1); ca.nl = g.n[1]; ca.logn = g.logn[1];
        ca.ls = g.S; ca.bs = (long long)g.n[1] * g.S;
        batches = g.n[2]; mode = slot == SLOT_Y_FWD ? 1 : 2;
    }
}

// spectral columns that carry data (full spectrum of the packed pair + half spectrum)
static double livec3(const SpecGeom &g) { return (double)(g.n[0] + g.n[0] / 2 + 1); }

template <typename T, typename TIn, typename TOut>
llg_status spectral_chain(llg_ctx *c, int in_mode, int out_mode, const NodalIO<TIn, TOut, T> &io,
                          const Symbol &sym) {
    const SpecGeom &g = c->geo;
    const int n0 = g.n[0];
    const int E = row_E<T>(n0), P = n0 / E;
    const long long pairs = g.rows / 2;
    int G = 256 / (3 * P);
    if (G < 1) G = 1;
    long long want = pairs / (2LL * c->sm_count);
    if (want < G) G = (int)(want < 1 ? 1 : want);
    const int blocks = (int)((pairs + G - 1) / G);
    const int threads = 3 * G * P;
    const bool rct = ct::covers(g.logn[0]);
    const size_t smr = rct ? ct::row_smem<T>(n0, G) : (size_t)3 * G * RowLayout::size(n0) * sizeof(cplx<T>);

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
    if constexpr (sizeof(T) == 4) {
        if (c->pass_plan == LLG_PLAN_CLUSTER && xy::available(c, in_mode, out_mode)) {
            // three passes: xy forward (cluster per plane), z, xy inverse
            const double ylines = livec3(g) * g.n[2], zlines = livec3(g) * g.n[1];
            prof_begin(c, K_XFWD, in_b + live * CB, xf + fftf(ylines, g.n[1], g.logn[1]));
            e = xy::forward<TIn, TOut>(c, in_mode, ra);
            prof_end(c);
            if (e != cudaSuccess) return cuda_check(c, e, "xy-pass forward");
            c->launches++;
            ColArgs<T> ca{};
            int batches = 1, mode = 7;
            slot_args<T>(c, SLOT_Z, sym, ca, batches, mode);
            ca.skip = io.skip;
            prof_begin(c, K_AXIS, 2 * live * CB, 2 * fftf(zlines, g.n[2], g.logn[2]));
            e = launch_col_cfg<T>(c, mode, ca, batches, slot_cfg<T>(c, SLOT_Z, ca.nl));
            prof_end(c);
            c->launches++;
            if (e != cudaSuccess) return cuda_check(c, e, "z-pass");
            prof_begin(c, K_XINV, live * CB + out_b, xf + fftf(ylines, g.n[1], g.logn[1]));
            e = xy::inverse<TIn, TOut>(c, out_mode, ra);
            prof_end(c);
            if (e != cudaSuccess) return cuda_check(c, e, "xy-pass inverse");
            c->launches++;
            return LLG_OK;
        }
    }
#define LLG_DISPATCH_E(FN, MODE)                                                              \
    switch (E) {                                                                              \
        case 2: e = FN<T, TIn, TOut, 2>(c, MODE, ra, blocks, threads, smr); break;            \
        case 4: e = FN<T, TIn, TOut, 4>(c, MODE, ra, blocks, threads, smr); break;            \
        case 8: e = FN<T, TIn, TOut, 8>(c, MODE, ra, blocks, threads, smr); break;            \
        default:                                                                              \
            if constexpr (sizeof(T) == 4) e = FN<T, TIn, TOut, 16>(c, MODE, ra, blocks, threads, smr); \
            else e = cudaErrorInvalidValue;                                                   \
            break;                                                                            \
    }
    if constexpr (is_fpair<T>::value) {
        if (!pair_chains_available(c)) return set_error(c, LLG_ERR_UNSUPPORTED_SIZE, "FP32-pair chain: axis length outside 64..1024");
    }
    prof_begin(c, K_XFWD, in_b + live * CB, xf);
    if (rct) e = ct::row_fwd<T, TIn, TOut>(c, g.logn[0], in_mode, ra, blocks, threads, smr);
    else if constexpr (is_fpair<T>::value) e = cudaErrorInvalidValue;
    else { LLG_DISPATCH_E(launch_row_fwd_E, in_mode) }
    prof_end(c);
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass forward");
    c->launches++;

    const double livec = (double)(n0 + n0 / 2 + 1);
    auto run_slot = [&](int slot, double flops) -> cudaError_t {
        ColArgs<T> ca{};
        int batches = 1, mode = 7;
        slot_args<T>(c, slot, sym, ca, batches, mode);
        ca.skip = io.skip;
        prof_begin(c, K_AXIS, 2 * live * CB, flops);
        cudaError_t err = launch_col_cfg<T>(c, mode, ca, batches, slot_cfg<T>(c, slot, ca.nl));
        prof_end(c);
        c->launches++;
        return err;
    };
    if (g.dim == 2) {
        e = run_slot(SLOT_2D, 2 * fftf(livec, g.n[1], g.logn[1]));
        if (e != cudaSuccess) return cuda_check(c, e, "y-pass");
    } else {
        const double ylines = livec * g.n[2], zlines = livec * g.n[1];
        if ((e = run_slot(SLOT_Y_FWD, fftf(ylines, g.n[1], g.logn[1]))) != cudaSuccess) return cuda_check(c, e, "y-pass forward");
        if ((e = run_slot(SLOT_Z, 2 * fftf(zlines, g.n[2], g.logn[2]))) != cudaSuccess) return cuda_check(c, e, "z-pass");
        if ((e = run_slot(SLOT_Y_INV, fftf(ylines, g.n[1], g.logn[1]))) != cudaSuccess) return cuda_check(c, e, "y-pass inverse");
    }
    prof_begin(c, K_XINV, live * CB + out_b, xf);
    if (rct) e = ct::row_inv<T, TIn, TOut>(c, g.logn[0], out_mode, ra, blocks, threads, smr);
    else if constexpr (is_fpair<T>::value) e = cudaErrorInvalidValue;
    else { LLG_DISPATCH_E(launch_row_inv_E, out_mode) }
    prof_end(c);
#undef LLG_DISPATCH_E
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass inverse");
    c->launches++;
    return LLG_OK;
}

// the axis passes between the x passes of a five-pass (3D) or three-pass (2D) FP32 round trip
static llg_status axis_passes32(llg_ctx *c, const Symbol &sym, const int *skip) {
    const SpecGeom &g = c->geo;
    const int n0 = g.n[0];
    const double CB = 2.0 * sizeof(float), livec = (double)(n0 + n0 / 2 + 1), live = (double)g.rows * livec;
    auto fftf = [](double lines, int n, int logn) { return lines * 5.0 * n * logn; };
    auto run_slot = [&](int slot, double flops) -> cudaError_t {
        ColArgs<float> ca{};
        int batches = 1, mode = 7;
        slot_args<float>(c, slot, sym, ca, batches, mode);
        ca.skip = skip;
        prof_begin(c, K_AXIS, 2 * live * CB, flops);
        cudaError_t err = launch_col_cfg<float>(c, mode, ca, batches, slot_cfg<float>(c, slot, ca.nl));
        prof_end(c);
        c->launches++;
        return err;
    };
    cudaError_t e;
    if (g.dim == 2) {
        if ((e = run_slot(SLOT_2D, 2 * fftf(livec, g.n[1], g.logn[1]))) != cudaSuccess) return cuda_check(c, e, "y-pass");
        return LLG_OK;
    }
    const double ylines = livec * g.n[2], zlines = livec * g.n[1];
    if ((e = run_slot(SLOT_Y_FWD, fftf(ylines, g.n[1], g.logn[1]))) != cudaSuccess) return cuda_check(c, e, "y-pass forward");
    if ((e = run_slot(SLOT_Z, 2 * fftf(zlines, g.n[2], g.logn[2]))) != cudaSuccess) return cuda_check(c, e, "z-pass");
    if ((e = run_slot(SLOT_Y_INV, fftf(ylines, g.n[1], g.logn[1]))) != cudaSuccess) return cuda_check(c, e, "y-pass inverse");
    return LLG_OK;
}

bool chain_pm_available(const llg_ctx *c) {
    return c->pass_plan == LLG_PLAN_FIVE && ct::covers(c->geo.logn[0]) && c->spec32 != nullptr;
}

template <typename TIn1>
llg_status spectral_chain_pm(llg_ctx *c, const NodalIO<TIn1, float, float> &io1, const Symbol &sym1,
                             const NodalIO<float, float, float> &io2, const Symbol &sym2) {
    const SpecGeom &g = c->geo;
    const int n0 = g.n[0];
    if (!chain_pm_available(c) || io2.scale != nullptr || io1.skip != io2.skip)
        return set_error(c, LLG_ERR_INVALID_ARG, "fused preconditioner-matvec chain: unsupported arguments");
    const int E = row_E<float>(n0), P = n0 / E;
    const long long pairs = g.rows / 2;
    int G = 256 / (3 * P);
    if (G < 1) G = 1;
    long long want = pairs / (2LL * c->sm_count);
    if (want < G) G = (int)(want < 1 ? 1 : want);
    const int blocks = (int)((pairs + G - 1) / G);
    const int threads = 3 * G * P;
    const size_t smr = ct::row_smem<float>(n0, G);
    RowArgs<float, TIn1, float> ra1;
    ra1.spec = spec_of<float>(c);
    ra1.tw0 = tw_of<float>(c, 0);
    ra1.n0 = n0; ra1.logn0 = g.logn[0]; ra1.S = g.S; ra1.G = G;
    ra1.rows = g.rows; ra1.N = g.N; ra1.io = io1;
    RowArgs<float, float, float> ra2;
    ra2.spec = ra1.spec; ra2.tw0 = ra1.tw0;
    ra2.n0 = n0; ra2.logn0 = g.logn[0]; ra2.S = g.S; ra2.G = G;
    ra2.rows = g.rows; ra2.N = g.N; ra2.io = io2;
    const double W = 4.0, CB = 8.0, Nd = (double)g.N, live = (double)g.rows * (n0 + n0 / 2 + 1);
    const double xf = (double)g.rows * 1.5 * 5.0 * n0 * g.logn[0];
    cudaError_t e;
    llg_status st;
    prof_begin(c, K_XFWD, 3 * Nd * sizeof(TIn1) + live * CB, xf);
    e = ct::row_fwd<float, TIn1, float>(c, g.logn[0], IN_V, ra1, blocks, threads, smr);
    prof_end(c);
    c->launches++;
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass forward");
    if ((st = axis_passes32(c, sym1, io1.skip)) != LLG_OK) return st;
    // x-pass inverse of the preconditioner (reads the spectrum, m, r; writes z) and x-pass
    // forward of the matvec from z in shared memory (writes the spectrum)
    prof_begin(c, K_XINV, 2 * live * CB + Nd * (3 * W + sizeof(TIn1) + 4 * W), 2 * xf);
    e = ct::row_inv_fwd<TIn1>(c, g.logn[0], ra1, ra2, blocks, threads, smr);
    prof_end(c);
    c->launches++;
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass inverse + forward");
    if ((st = axis_passes32(c, sym2, io2.skip)) != LLG_OK) return st;
    prof_begin(c, K_XINV, live * CB + Nd * (3 * W + 4 * W + 4 * W), xf);
    e = ct::row_inv<float, float, float>(c, g.logn[0], OUT_MATVEC, ra2, blocks, threads, smr);
    prof_end(c);
    c->launches++;
    if (e != cudaSuccess) return cuda_check(c, e, "x-pass inverse");
    return LLG_OK;
}

template llg_status spectral_chain_pm<double>(llg_ctx *, const NodalIO<double, float, float> &, const Symbol &,
                                              const NodalIO<float, float, float> &, const Symbol &);
template llg_status spectral_chain_pm<float>(llg_ctx *, const NodalIO<float, float, float> &, const Symbol &,
                                             const NodalIO<float, float, float> &, const Symbol &);

llg_status plain_axis_pass64(llg_ctx *c, int axis, bool forward) {
    if (axis != 1 || c->geo.dim != 3) return set_error(c, LLG_ERR_INVALID_ARG, "plain axis pass: 3D y axis only");
    ColArgs<double> ca{};
    int batches = 1, mode = 1;
    Symbol sym{1.0, 0.0, 1.0, 0, 0};
    slot_args<double>(c, forward ? SLOT_Y_FWD : SLOT_Y_INV, sym, ca, batches, mode);
    // the register kernel covers every column slot (the staged one only the live ones of
    // the packed layout)
    const cudaError_t e = launch_col_cfg<double>(c, mode, ca, batches, col_default<double>(ca.nl));
    c->launches++;
    return cuda_check(c, e, "axis pass");
}

// ------------------------------------------------------------------ autotuner

// deterministic pseudo-random fill in [-1, 1) (hash of the index)
template <typename C>
__global__ void k_fill_pattern(C *p, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull;
        h ^= h >> 29; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 32;
        const double a = (double)(h & 0xFFFFFF) / 8388608.0 - 1.0, b = (double)((h >> 24) & 0xFFFFFF) / 8388608.0 - 1.0;
        p[i].x = (decltype(p[i].x))a;
        p[i].y = (decltype(p[i].y))b;
    }
}

// per-block max |a - b| and max |b| over the live columns of every spectral row
template <typename C>
__global__ void k_live_maxdiff(const C *a, const C *b, long long rows, int S, int live, double *partials) {
    double d = 0.0, m = 0.0;
    const long long n = rows * live;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / live, col = i % live, k = r * S + col;
        d = fmax(d, fmax(fabs((double)a[k].x - (double)b[k].x), fabs((double)a[k].y - (double)b[k].y)));
        m = fmax(m, fmax(fabs((double)b[k].x), fabs((double)b[k].y)));
    }
    __shared__ double sd[256], sm2[256];
    sd[threadIdx.x] = d;
    sm2[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < (int)blockDim.x; ++t) { d = fmax(d, sd[t]); m = fmax(m, sm2[t]); }
        partials[2 * blockIdx.x] = d;
        partials[2 * blockIdx.x + 1] = m;
    }
}

static std::string cfg_name(const ColCfg &f) {
    char b[64];
    if (f.kind == 0) snprintf(b, sizeof b, "register(E%d,TW%d)", f.E, f.TW);
    else if (f.kind == 3) snprintf(b, sizeof b, "paired(E%d,TW%d)", f.E, f.TW);
    else if (f.kind == 4 && f.E == 8) snprintf(b, sizeof b, "tma(TW%d)", f.TW);
    else if (f.kind == 4) snprintf(b, sizeof b, "tma(E%d,TW%d)", f.E, f.TW);
    else snprintf(b, sizeof b, "staged(TW%d,CB%d)", f.TW, f.CB);
    return b;
}

template <typename T>
static llg_status tune_prec(llg_ctx *c, std::string *report) {
    using C = cplx<T>;
    const SpecGeom &g = c->geo;
    const int pi = sizeof(T) == 4 ? 0 : 1;
    const long long elems = g.rows * (long long)g.S;
    const int live = g.n[0] + g.n[0] / 2 + 1;
    C *pristine = nullptr, *ref = nullptr;
    double *part = nullptr, hp[2 * 512];
    cudaError_t e = cudaMalloc(&pristine, sizeof(C) * elems);
    if (e == cudaSuccess) e = cudaMalloc(&ref, sizeof(C) * elems);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * 2 * 512);
    auto cleanup = [&]() { cudaFree(pristine); cudaFree(ref); cudaFree(part); };
    if (e != cudaSuccess) { cleanup(); return cuda_check(c, e, "autotune buffers"); }
    k_fill_pattern<<<512, 256, 0, c->stream>>>(pristine, elems);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<int> slots = g.dim == 2 ? std::vector<int>{SLOT_2D} : std::vector<int>{SLOT_Y_FWD, SLOT_Z, SLOT_Y_INV};
    static const char *slot_names[] = {"y(2D)", "y-forward", "z", "y-inverse"};
    llg_status st = LLG_OK;
    for (int slot : slots) {
        ColArgs<T> ca{};
        int batches = 1, mode = 7;
        Symbol sym{1.0, 1e-3, 1.0, 1, 0};
        slot_args<T>(c, slot, sym, ca, batches, mode);
        ca.sscale = (T)(1.0 / ca.nl);
        const ColCfg def = col_default<T>(ca.nl);
        auto run_once = [&](const ColCfg &f, float *ms) -> cudaError_t {
            cudaMemcpyAsync(ca.spec, pristine, sizeof(C) * elems, cudaMemcpyDeviceToDevice, c->stream);
            cudaEventRecord(e0, c->stream);
            cudaError_t err = launch_col_cfg<T>(c, mode, ca, batches, f);
            cudaEventRecord(e1, c->stream);
            if (err != cudaSuccess) return err;
            err = cudaEventSynchronize(e1);
            if (err == cudaSuccess && ms) err = cudaEventElapsedTime(ms, e0, e1);
            return err;
        };
        if ((e = run_once(def, nullptr)) != cudaSuccess) { st = cuda_check(c, e, "autotune reference"); break; }
        cudaMemcpyAsync(ref, ca.spec, sizeof(C) * elems, cudaMemcpyDeviceToDevice, c->stream);
        ColCfg best = def;
        float best_ms = 1e30f;
        char line[256];
        snprintf(line, sizeof line, "%s slot %s (n=%d):", sizeof(T) == 4 ? "fp32" : "fp64", slot_names[slot], ca.nl);
        std::string rep = line;
        for (const ColCfg &f : col_candidates<T>(c, ca.nl)) {
            if ((e = run_once(f, nullptr)) != cudaSuccess) { cudaGetLastError(); rep += " " + cfg_name(f) + "=launch-fail"; continue; }
            k_live_maxdiff<C><<<512, 256, 0, c->stream>>>(ca.spec, ref, g.rows, g.S, live, part);
            cudaMemcpy(hp, part, sizeof(double) * 2 * 512, cudaMemcpyDeviceToHost);
            double d = 0, m = 0;
            for (int b = 0; b < 512; ++b) { d = std::max(d, hp[2 * b]); m = std::max(m, hp[2 * b + 1]); }
            const double tol = sizeof(T) == 4 ? 1e-4 : 1e-11;
            if (!(d <= tol * m)) { rep += " " + cfg_name(f) + "=rejected"; continue; }
            // median of seven timed runs; a later candidate replaces the best so far only when
            // it is at least 3% faster, so that near-ties keep the earlier (register, paired,
            // TMA-fed) shapes instead of following timing noise
            constexpr int REPS = 7;
            float t[REPS], ms = 0.f;
            int got = 0;
            for (; got < REPS; ++got) {
                if ((e = run_once(f, &ms)) != cudaSuccess) break;
                t[got] = ms;
            }
            if (e != cudaSuccess) { cudaGetLastError(); continue; }
            std::sort(t, t + REPS);
            const float tot = t[REPS / 2];
            snprintf(line, sizeof line, " %s=%.1fus", cfg_name(f).c_str(), tot * 1e3f);
            rep += line;
            if (tot < 0.97f * best_ms) { best_ms = tot; best = f; }
        }
        c->colcfg[pi][slot] = best;
        *report += rep + " -> " + cfg_name(best) + "\n";
    }
    // slots the grid does not use keep the default
    if (g.dim == 2) {
        for (int sl = 1; sl < NSLOT; ++sl) c->colcfg[pi][sl] = col_default<T>(sl == SLOT_Z ? g.n[2] : g.n[1]);
    } else {
        c->colcfg[pi][SLOT_2D] = col_default<T>(g.n[1]);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    if (st == LLG_OK) c->tuned[pi] = true;
    return st;
}

template <typename T> static void fill_defaults(llg_ctx *c) {
    const int pi = sizeof(T) == 4 ? 0 : 1;
    const SpecGeom &g = c->geo;
    for (int sl = 0; sl < NSLOT; ++sl) c->colcfg[pi][sl] = col_default<T>(sl == SLOT_Z ? g.n[2] : g.n[1]);
    c->tuned[pi] = true;
}

// one slot's shape, set by hand (kept only if the tuner would consider it for this grid)
llg_status set_axis_shape(llg_ctx *c, int fp32, int slot, const ColCfg &f) {
    const SpecGeom &g = c->geo;
    if (slot < 0 || slot >= NSLOT || (g.dim == 2) != (slot == SLOT_2D))
        return set_error(c, LLG_ERR_INVALID_ARG, "axis shape: no such pass on this grid");
    const int nl = slot == SLOT_Z ? g.n[2] : g.n[1];
    const std::vector<ColCfg> cand = fp32 ? col_candidates<float>(c, nl) : col_candidates<double>(c, nl);
    bool ok = false;
    for (const ColCfg &q : cand) ok = ok || (q.kind == f.kind && q.E == f.E && q.TW == f.TW && q.CB == f.CB);
    if (!ok) return set_error(c, LLG_ERR_INVALID_ARG, "axis shape: not a compiled shape for this line length");
    const int pi = fp32 ? 0 : 1;
    if (!c->tuned[pi]) {
        if (fp32) fill_defaults<float>(c);
        else fill_defaults<double>(c);
    }
    c->colcfg[pi][slot] = f;
    return LLG_OK;
}

llg_status autotune(llg_ctx *c, int prec_mask, std::string *report) {
    llg_status st = LLG_OK;
    if ((prec_mask & 2) && c->spec32) st = tune_prec<float>(c, report);
    if (st == LLG_OK && (prec_mask & 1) && c->spec64) st = tune_prec<double>(c, report);
    return st;
}

template llg_status spectral_chain<double, double, double>(llg_ctx *, int, int, const NodalIO<double, double, double> &, const Symbol &);
template llg_status spectral_chain<float, double, float>(llg_ctx *, int, int, const NodalIO<double, float, float> &, const Symbol &);
template llg_status spectral_chain<float, float, double>(llg_ctx *, int, int, const NodalIO<float, double, float> &, const Symbol &);
template llg_status spectral_chain<float, float, float>(llg_ctx *, int, int, const NodalIO<float, float, float> &, const Symbol &);
template llg_status spectral_chain<fpair, double, double>(llg_ctx *, int, int, const NodalIO<double, double, fpair> &, const Symbol &);

}  // namespace llg
