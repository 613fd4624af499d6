// ssp_fp32_clamp.cu -- FP32C kernels with windows clamped inside the data
// (Listing 1 iper = 1).
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_PGRAM(float, false, false, false, fp32_clamp, false)
