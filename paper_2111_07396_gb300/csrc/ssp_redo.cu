// ssp_redo.cu -- the FP64 kernel that recomputes the frequencies an FP32C
// launch flagged: binary64 smoothing with plain binary64 window prefixes,
// accurate to about 1e-8, far inside the FP32C tolerance its results serve.
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_SIZES(double, true, redo)
SSP_INSTANTIATE_PGRAM(double, true, true, false, redo_per, false)
