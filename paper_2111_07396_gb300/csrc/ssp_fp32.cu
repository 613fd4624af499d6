// ssp_fp32.cu -- FP32C instantiation: exact fixed-point fold, FP32 smoothing
// about local origins, compensated chi2.
#include "ssp_kernels.cuh"
SSP_INSTANTIATE(float, fp32)
