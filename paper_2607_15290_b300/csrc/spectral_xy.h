// spectral_xy.h -- the cluster plan of a 3D FP32 Fourier round trip (spectral_xy.cu):
// x and y transforms of each z-plane in one thread-block cluster, three HBM passes
// per round trip instead of five.
#pragma once
#include "spectral_kernels.cuh"

namespace llg {
namespace xy {

// a compiled cluster plan covers this grid's x/y lengths and these prologue/epilogue modes
bool available(const llg_ctx *c, int in_mode, int out_mode);
// the xy forward pass (nodal prologue, x and y transforms) and the xy inverse pass (y and
// x inverse transforms, nodal epilogue), launched on the context's stream
template <typename TIn, typename TOut>
cudaError_t forward(llg_ctx *c, int in_mode, const RowArgs<float, TIn, TOut> &a);
template <typename TIn, typename TOut>
cudaError_t inverse(llg_ctx *c, int out_mode, const RowArgs<float, TIn, TOut> &a);

}  // namespace xy
}  // namespace llg
