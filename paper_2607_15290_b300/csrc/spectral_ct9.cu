// spectral_ct9.cu -- compile-time-length pass kernels for 512-point lines.
#define LLG_CT_LOGN 9
#include "spectral_ct_inst.cuh"
