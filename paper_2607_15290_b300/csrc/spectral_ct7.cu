// spectral_ct7.cu -- compile-time-length pass kernels for 128-point lines.
#define LLG_CT_LOGN 7
#include "spectral_ct_inst.cuh"
