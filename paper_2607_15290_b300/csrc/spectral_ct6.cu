// spectral_ct6.cu -- compile-time-length pass kernels for 64-point lines.
#define LLG_CT_LOGN 6
#include "spectral_ct_inst.cuh"
