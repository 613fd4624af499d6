// ssp_fp32_shared.cu -- FP32C kernels (periodic windows) whose work items may
// cover several objects with identical times: one fold and sort per frequency
// for all of them.
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_PGRAM(float, false, true, true, fp32_shared, true)
