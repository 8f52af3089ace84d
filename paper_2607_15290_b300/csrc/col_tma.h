// col_tma.h -- FP32 axis passes fed by the tensor memory accelerator (col_tma.cu).
#pragma once
#include "spectral_kernels.cuh"

namespace llg {
namespace tma {

// the TMA-fed kernels cover lines of this length (and the context has the host-mapped
// error word their bounded waits report through)
bool available(const llg_ctx *c, int nl);
// one axis pass (mode 1: forward, 2: inverse, 7: forward, multiplier, inverse) over
// `batches` batches of spectral column tiles of TW columns (8 or 16), E points of a line per
// thread (8: radix-8 stages; 16: radix-16 stages)
cudaError_t col_launch(llg_ctx *c, int mode, const ColArgs<float> &a, int batches, int TW, int E);

}  // namespace tma
}  // namespace llg
