// spectral_ct_launch.h -- launchers of the compile-time-length pass kernels
// (spectral_ct.cuh).  Each line length 2^LOGN, 6 <= LOGN <= 10, is compiled in a
// translation unit of its own (spectral_ct<LOGN>.cu).
#pragma once
#include "spectral_kernels.cuh"

namespace llg {
namespace ct {

constexpr int kMinLog = 6, kMaxLog = 10;
inline bool covers(int logn) { return logn >= kMinLog && logn <= kMaxLog; }

template <typename T, typename TIn, typename TOut, int LOGN>
cudaError_t row_fwd_launch(llg_ctx *c, int in_mode, const RowArgs<T, TIn, TOut> &a, int blocks, int threads, size_t sm);
template <typename T, typename TIn, typename TOut, int LOGN>
cudaError_t row_inv_launch(llg_ctx *c, int out_mode, const RowArgs<T, TIn, TOut> &a, int blocks, int threads, size_t sm);
template <typename T, int LOGN>
cudaError_t col_launch(llg_ctx *c, int mode, const ColArgs<T> &a, dim3 grid, int TW);
template <typename TIn1, int LOGN>
cudaError_t row_inv_fwd_launch(llg_ctx *c, const RowArgs<float, TIn1, float> &a1, const RowArgs<float, float, float> &a2,
                               int blocks, int threads, size_t sm);
template <int LOGN>
cudaError_t staged_launch(llg_ctx *c, int mode, const ColArgs<float> &a, int live, int batches, int TWL, int CB);
template <int LOGN>
cudaError_t col_v2_launch(llg_ctx *c, int mode, const ColArgs<float> &a, dim3 grid, int TW);

// shared memory of a row block of G pairs: two exchange buffers of 3G padded lines
template <typename T> inline size_t row_smem(int n0, int G) { return (size_t)2 * 3 * G * (n0 + n0 / 8) * sizeof(cplx<T>); }
// shared memory of a column tile: two exchange buffers when they fit in 96 KB, else one
template <typename T> inline bool col_db(int nl, int TW) { return (size_t)2 * nl * TW * sizeof(cplx<T>) <= 96 * 1024; }
template <typename T> inline size_t col_smem(int nl, int TW) { return (size_t)(col_db<T>(nl, TW) ? 2 : 1) * nl * TW * sizeof(cplx<T>); }

// runtime dispatch over the compiled lengths (not seen by the per-length units, so
// that each of them instantiates its own length only)
#ifndef LLG_CT_LOGN
#define LLG_CT_SWITCH(LOGN_VAR, CALL)                     \
    switch (LOGN_VAR) {                                   \
        case 6: { constexpr int LG = 6; return CALL; }    \
        case 7: { constexpr int LG = 7; return CALL; }    \
        case 8: { constexpr int LG = 8; return CALL; }    \
        case 9: { constexpr int LG = 9; return CALL; }    \
        case 10: { constexpr int LG = 10; return CALL; }  \
        default: return cudaErrorInvalidValue;            \
    }

template <typename T, typename TIn, typename TOut>
inline cudaError_t row_fwd(llg_ctx *c, int logn, int in_mode, const RowArgs<T, TIn, TOut> &a, int blocks, int threads, size_t sm) {
    LLG_CT_SWITCH(logn, (row_fwd_launch<T, TIn, TOut, LG>(c, in_mode, a, blocks, threads, sm)))
}
template <typename T, typename TIn, typename TOut>
inline cudaError_t row_inv(llg_ctx *c, int logn, int out_mode, const RowArgs<T, TIn, TOut> &a, int blocks, int threads, size_t sm) {
    LLG_CT_SWITCH(logn, (row_inv_launch<T, TIn, TOut, LG>(c, out_mode, a, blocks, threads, sm)))
}
template <typename TIn1>
inline cudaError_t row_inv_fwd(llg_ctx *c, int logn, const RowArgs<float, TIn1, float> &a1,
                               const RowArgs<float, float, float> &a2, int blocks, int threads, size_t sm) {
    LLG_CT_SWITCH(logn, (row_inv_fwd_launch<TIn1, LG>(c, a1, a2, blocks, threads, sm)))
}
template <typename T>
inline cudaError_t col(llg_ctx *c, int logn, int mode, const ColArgs<T> &a, dim3 grid, int TW) {
    LLG_CT_SWITCH(logn, (col_launch<T, LG>(c, mode, a, grid, TW)))
}
inline cudaError_t staged(llg_ctx *c, int logn, int mode, const ColArgs<float> &a, int live, int batches, int TWL, int CB) {
    LLG_CT_SWITCH(logn, (staged_launch<LG>(c, mode, a, live, batches, TWL, CB)))
}
inline cudaError_t col_v2(llg_ctx *c, int logn, int mode, const ColArgs<float> &a, dim3 grid, int TW) {
    LLG_CT_SWITCH(logn, (col_v2_launch<LG>(c, mode, a, grid, TW)))
}
#undef LLG_CT_SWITCH
#endif

}  // namespace ct
}  // namespace llg
