// ssp_fp32.cu -- FP32C instantiation, periodic windows: exact fixed-point fold,
// FP32 smoothing about local origins from double-float window prefixes,
// compensated chi2.
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_PREP(float, fp32)
SSP_INSTANTIATE_SIZES(float, false, fp32)
SSP_INSTANTIATE_PGRAM(float, false, true, false, fp32_per, true)
