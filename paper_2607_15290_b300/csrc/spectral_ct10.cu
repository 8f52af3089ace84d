// spectral_ct10.cu -- compile-time-length pass kernels for 1024-point lines.
#define LLG_CT_LOGN 10
#include "spectral_ct_inst.cuh"
