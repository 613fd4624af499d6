// ssp_redo_clamp.cu -- the FP64 recompute kernels with windows clamped inside
// the data (Listing 1 iper = 1).
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_PGRAM(double, true, false, false, redo_clamp, false)
