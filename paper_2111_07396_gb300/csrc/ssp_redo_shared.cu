// ssp_redo_shared.cu -- the FP64 recompute kernels (periodic windows) for work
// items that cover several objects with identical times.
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_PGRAM(double, true, true, true, redo_shared, false)
