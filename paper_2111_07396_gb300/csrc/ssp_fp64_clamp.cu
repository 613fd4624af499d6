// ssp_fp64_clamp.cu -- FP64 kernels with windows clamped inside the data
// (Listing 1 iper = 1).
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_PGRAM(double, false, false, false, fp64_clamp, false)
