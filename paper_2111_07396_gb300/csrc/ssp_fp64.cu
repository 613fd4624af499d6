// ssp_fp64.cu -- FP64 instantiation: binary64 throughout, phase fold
// bit-identical to Alg. 1's rounded product.
#include "ssp_kernels.cuh"
SSP_INSTANTIATE(double, fp64)
