// ssp_fp64.cu -- FP64 instantiation, periodic windows: binary64 throughout
// (double-double window prefixes), phase fold bit-identical to Alg. 1's
// rounded product.
#include "ssp_kernels.cuh"
SSP_INSTANTIATE_PREP(double, fp64)
SSP_INSTANTIATE_SIZES(double, false, fp64)
SSP_INSTANTIATE_PGRAM(double, false, true, false, fp64_per, false)
