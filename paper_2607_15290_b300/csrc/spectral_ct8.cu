// spectral_ct8.cu -- compile-time-length pass kernels for 256-point lines.
#define LLG_CT_LOGN 8
#include "spectral_ct_inst.cuh"
