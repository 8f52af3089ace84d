// spectral_ct_inst.cuh -- definitions and explicit instantiations of the
// compile-time-length launchers for one LOGN (set by the including file).
#pragma once
#include <algorithm>
#include "spectral_ct.cuh"
#include "spectral_ct_launch.h"

#ifndef LLG_CT_LOGN
#error "define LLG_CT_LOGN before including spectral_ct_inst.cuh"
#endif

namespace llg {
namespace ct {

template <typename K> static inline cudaError_t prep(K kern) {
    static thread_local const void *done[64];
    static thread_local int ndone = 0;
    for (int i = 0; i < ndone; ++i)
        if (done[i] == (const void *)kern) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess && ndone < 64) done[ndone++] = (const void *)kern;
    return e;
}

template <typename T, typename TIn, typename TOut, int LOGN>
cudaError_t row_fwd_launch(llg_ctx *c, int in_mode, const RowArgs<T, TIn, TOut> &a, int blocks, int threads, size_t sm) {
#define LLG_RF(MODE)                                                   \
    case MODE: {                                                       \
        auto k = row_fwd_ct<T, TIn, TOut, LOGN, MODE>;                 \
        cudaError_t e = prep(k);                                       \
        if (e != cudaSuccess) return e;                                \
        return launch_pdl(k, dim3(blocks), dim3(threads), sm, c->stream, a); \
    }
    if constexpr (is_fpair<T>::value) {
        // FP32-pair chains: the true residual and the right-hand side only
        switch (in_mode) {
            LLG_RF(IN_V) LLG_RF(IN_M)
        }
    } else {
        switch (in_mode) {
            LLG_RF(IN_V) LLG_RF(IN_FUSED) LLG_RF(IN_M) LLG_RF(IN_NODAL_T)
        }
    }
#undef LLG_RF
    return cudaErrorInvalidValue;
}

template <typename T, typename TIn, typename TOut, int LOGN>
cudaError_t row_inv_launch(llg_ctx *c, int out_mode, const RowArgs<T, TIn, TOut> &a, int blocks, int threads, size_t sm) {
#define LLG_RI(MODE)                                                   \
    case MODE: {                                                       \
        auto k = row_inv_ct<T, TIn, TOut, LOGN, MODE>;                 \
        cudaError_t e = prep(k);                                       \
        if (e != cudaSuccess) return e;                                \
        return launch_pdl(k, dim3(blocks), dim3(threads), sm, c->stream, a); \
    }
    if constexpr (is_fpair<T>::value) {
        switch (out_mode) {
            LLG_RI(OUT_MATVEC) LLG_RI(OUT_FIELD)
        }
    } else {
        switch (out_mode) {
            LLG_RI(OUT_APPLY) LLG_RI(OUT_FUSED) LLG_RI(OUT_MATVEC) LLG_RI(OUT_FIELD) LLG_RI(OUT_PLAIN) LLG_RI(OUT_JT)
        }
    }
#undef LLG_RI
    return cudaErrorInvalidValue;
}

template <typename TIn1, int LOGN>
cudaError_t row_inv_fwd_launch(llg_ctx *c, const RowArgs<float, TIn1, float> &a1, const RowArgs<float, float, float> &a2,
                               int blocks, int threads, size_t sm) {
    auto k = row_inv_fwd_ct<TIn1, LOGN>;
    cudaError_t e = prep(k);
    if (e != cudaSuccess) return e;
    return launch_pdl(k, dim3(blocks), dim3(threads), sm, c->stream, a1, a2);
}

template <typename T, int LOGN, int TW>
static cudaError_t col_launch_tw(llg_ctx *c, int mode, const ColArgs<T> &a, dim3 grid) {
    constexpr int N = 1 << LOGN, E = LineE<T, LOGN>::value, threads = TW * (N / E);
    if constexpr (threads > 512 || threads < 32) {
        return cudaErrorInvalidValue;
    } else {
        constexpr bool DB = 2 * N * TW * sizeof(cplx<T>) <= 96 * 1024;
        constexpr size_t sm = (DB ? 2 : 1) * (size_t)N * TW * sizeof(cplx<T>);
        if constexpr (sm > 200 * 1024) {
            return cudaErrorInvalidValue;
        } else {
#define LLG_CK(MODE)                                                   \
    case MODE: {                                                       \
        auto k = col_ct<T, LOGN, E, TW, MODE, DB>;                     \
        cudaError_t e = prep(k);                                       \
        if (e != cudaSuccess) return e;                                \
        return launch_pdl(k, dim3(grid), dim3(threads), sm, c->stream, a); \
    }
            switch (mode) {
                LLG_CK(1) LLG_CK(2) LLG_CK(7)
            }
#undef LLG_CK
            return cudaErrorInvalidValue;
        }
    }
}

template <typename T, int LOGN>
cudaError_t col_launch(llg_ctx *c, int mode, const ColArgs<T> &a, dim3 grid, int TW) {
    if constexpr (sizeof(T) == 4) {
        if (TW == 16) return col_launch_tw<T, LOGN, 16>(c, mode, a, grid);
        if (TW == 8) return col_launch_tw<T, LOGN, 8>(c, mode, a, grid);
    } else {
        if (TW == 8) return col_launch_tw<T, LOGN, 8>(c, mode, a, grid);
        if (TW == 4) return col_launch_tw<T, LOGN, 4>(c, mode, a, grid);
    }
    return cudaErrorInvalidValue;
}

template <int LOGN, int TW>
static cudaError_t col_v2_launch_tw(llg_ctx *c, int mode, const ColArgs<float> &a, dim3 grid) {
    constexpr int N = 1 << LOGN, E = LineE<float, LOGN>::value, threads = (TW / 2) * (N / E);
    if constexpr (threads > 512 || threads < 32) {
        return cudaErrorInvalidValue;
    } else {
        constexpr bool DB = 2 * N * TW * sizeof(float2) <= 96 * 1024;
        constexpr size_t sm = (DB ? 2 : 1) * (size_t)N * TW * sizeof(float2);
#define LLG_C2(MODE)                                                   \
    case MODE: {                                                       \
        auto k = col_ct_v2<LOGN, TW, MODE, DB>;                        \
        cudaError_t e = prep(k);                                       \
        if (e != cudaSuccess) return e;                                \
        return launch_pdl(k, dim3(grid), dim3(threads), sm, c->stream, a); \
    }
        switch (mode) {
            LLG_C2(1) LLG_C2(2) LLG_C2(7)
        }
#undef LLG_C2
        return cudaErrorInvalidValue;
    }
}

template <int LOGN>
cudaError_t col_v2_launch(llg_ctx *c, int mode, const ColArgs<float> &a, dim3 grid, int TW) {
    if (TW == 16) return col_v2_launch_tw<LOGN, 16>(c, mode, a, grid);
    if (TW == 8) return col_v2_launch_tw<LOGN, 8>(c, mode, a, grid);
    return cudaErrorInvalidValue;
}

template <int LOGN, int TWL, int CB>
static cudaError_t staged_launch_tw(llg_ctx *c, int mode, const ColArgs<float> &a, int live, int batches) {
    constexpr int N = 1 << LOGN, threads = CB * (N / 8);
    constexpr int SROW = StagedRow<TWL>::value;
    constexpr size_t sm = (size_t)N * SROW * sizeof(float2);
    if constexpr (threads > 512 || threads < 64 || sm > 160 * 1024) {
        return cudaErrorInvalidValue;
    } else {
        const dim3 grid((live + TWL - 1) / TWL, batches);
#define LLG_CS(MODE)                                                   \
    case MODE: {                                                       \
        auto k = col_staged_ct<LOGN, TWL, CB, MODE>;                   \
        cudaError_t e = prep(k);                                       \
        if (e != cudaSuccess) return e;                                \
        return launch_pdl(k, dim3(grid), dim3(threads), sm, c->stream, a, live); \
    }
        switch (mode) {
            LLG_CS(1) LLG_CS(2) LLG_CS(7)
        }
#undef LLG_CS
        return cudaErrorInvalidValue;
    }
}

template <int LOGN>
cudaError_t staged_launch(llg_ctx *c, int mode, const ColArgs<float> &a, int live, int batches, int TWL, int CB) {
#define LLG_ST(X, Y) if (TWL == X && CB == Y) return staged_launch_tw<LOGN, X, Y>(c, mode, a, live, batches);
    LLG_ST(64, 64) LLG_ST(64, 32) LLG_ST(64, 16) LLG_ST(32, 32) LLG_ST(32, 16) LLG_ST(32, 8)
    LLG_ST(16, 16) LLG_ST(16, 8) LLG_ST(16, 4) LLG_ST(8, 8) LLG_ST(8, 4)
#undef LLG_ST
    return cudaErrorInvalidValue;
}

#define LLG_CT_ROWS(T, TI, TO)                                                                                   \
    template cudaError_t row_fwd_launch<T, TI, TO, LLG_CT_LOGN>(llg_ctx *, int, const RowArgs<T, TI, TO> &, int, int, size_t); \
    template cudaError_t row_inv_launch<T, TI, TO, LLG_CT_LOGN>(llg_ctx *, int, const RowArgs<T, TI, TO> &, int, int, size_t);
LLG_CT_ROWS(double, double, double)
LLG_CT_ROWS(float, double, float)
LLG_CT_ROWS(float, float, double)
LLG_CT_ROWS(float, float, float)
LLG_CT_ROWS(fpair, double, double)
#undef LLG_CT_ROWS
template cudaError_t row_inv_fwd_launch<double, LLG_CT_LOGN>(llg_ctx *, const RowArgs<float, double, float> &,
                                                             const RowArgs<float, float, float> &, int, int, size_t);
template cudaError_t row_inv_fwd_launch<float, LLG_CT_LOGN>(llg_ctx *, const RowArgs<float, float, float> &,
                                                            const RowArgs<float, float, float> &, int, int, size_t);
template cudaError_t col_launch<double, LLG_CT_LOGN>(llg_ctx *, int, const ColArgs<double> &, dim3, int);
template cudaError_t col_launch<fpair, LLG_CT_LOGN>(llg_ctx *, int, const ColArgs<fpair> &, dim3, int);
template cudaError_t col_launch<float, LLG_CT_LOGN>(llg_ctx *, int, const ColArgs<float> &, dim3, int);
template cudaError_t staged_launch<LLG_CT_LOGN>(llg_ctx *, int, const ColArgs<float> &, int, int, int, int);
template cudaError_t col_v2_launch<LLG_CT_LOGN>(llg_ctx *, int, const ColArgs<float> &, dim3, int);

}  // namespace ct
}  // namespace llg
