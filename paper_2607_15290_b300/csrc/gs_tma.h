// gs_tma.h -- Gram-Schmidt passes of flexible solves in FP32-pair arithmetic with their
// operands staged in shared memory by bulk copies (gs_tma.cu).
#pragma once
#include "llg_internal.h"

namespace llg {
namespace gst {

// usable for vectors of n values (n a multiple of 4) on a context with the host-mapped
// error word the bounded waits report through
bool available(const llg_ctx *c, long long n);
// one pass (PASS_DOT, PASS_UPD_DOT, PASS_UPD_NRM) over nv <= 32 basis vectors, arguments as
// for the register form (w's hi plane wh, its lo plane wl in pass C, outputs oh / ol)
cudaError_t pass(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const float *wh, const float *wl,
                 float *oh, float *ol, long long n);

}  // namespace gst
}  // namespace llg
