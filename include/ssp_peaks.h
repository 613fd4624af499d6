/*
 * ssp_peaks.h -- ALU peaks of the current GPU, measured with FMA-chain
 * microbenchmarks (no counterpart in the paper: the periodogram kernels are
 * bound by FP32 issue, not by HBM or tensor cores, so their roofline needs
 * these rates).
 */
#ifndef SSP_PEAKS_H
#define SSP_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Times a grid of 8 blocks per SM x 256 threads, each thread running eight
 * independent chains of fused multiply-adds (2 flops each), in float and in
 * double; best of five runs after one warm-up.  Writes TFLOP/s (1e12
 * flops/s) to *fp32_tflops and *fp64_tflops.  Takes about a second.
 * Returns 0, -1 (NULL argument) or -3 (a CUDA call failed).
 */
int ssp_measure_alu_peaks(double *fp32_tflops, double *fp64_tflops);

#ifdef __cplusplus
}
#endif
#endif /* SSP_PEAKS_H */
