// ssp_fp64_shared.cu -- FP64 kernels (periodic windows) whose work items may
// cover several objects with identical times.
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_PGRAM(double, false, true, true, fp64_shared, false)
