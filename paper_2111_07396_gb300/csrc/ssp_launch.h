// ssp_launch.h -- host-side launch wrappers shared by the kernel translation
// units (one per precision) and the C ABI in ssp_api.cu.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ssp_device.cuh"

namespace ssp {

struct PrepArgs {
    const double *t, *y, *dy;  // [N] caller's device arrays
    const int64_t *off;        // [n_obj + 1]
    double *tt;                // [N] t - min t, binary64 (both paths)
    void *yc, *wv;             // [N] R: centred magnitudes, weights
    double *yc64, *wv64;       // [N] FP64 copies for the FP32C recompute (or null)
    float2 *ydf, *wdf;         // [N] FP32C: the same as double-float pairs, for the SP settle
    double *chi0;              // [n_obj]
    double *ymax;              // [n_obj] largest |y - ybar_w|
    int *bad;                  // [n_obj]
};

struct ArgmaxArgs {
    const void *power;         // [n_obj][n_freq] R
    const double *freq;
    const int64_t *fbase;      // null: one grid; else object o's grid starts at freq[fbase[o]]
    int64_t n_freq;
    const int *bad;
    double *best_period;       // [n_obj]
    double *best_power;        // [n_obj] or null
};

// search-and-refine: per object, the top k local maxima of its coarse power
// row and a grid of n_fine frequencies across each (see peaks_kernel)
struct PeaksArgs {
    const void *power;         // [n_obj][n_coarse] R
    const double *coarse;      // [n_coarse], increasing
    int64_t n_coarse;
    int k, n_fine;
    double *fine;              // [n_obj][k * n_fine]
};

// precision: 0 = FP64, 1 = FP32C, kPrecRedo = the FP64 recompute of flagged
// FP32C frequencies (plain binary64 window prefixes)
constexpr int kPrecRedo = 2;
cudaError_t prep_launch(int precision, const PrepArgs &a, int n_obj, cudaStream_t s);
cudaError_t argmax_launch(int precision, const ArgmaxArgs &a, int n_obj, cudaStream_t s);
cudaError_t peaks_launch(int precision, const PeaksArgs &a, int n_obj, cudaStream_t s);
// variant: VAR_SS, VAR_SP or VAR_FIXED; per: periodic windows, else clamped.
// Sets the dynamic shared-memory limit and returns resident CTAs per SM.
// shared: work items may cover several objects with identical times
// (periodic windows only).
// lng: the SS kernel that initialises its windows out of line (FP32C).
cudaError_t pgram_occupancy(int precision, int variant, bool gmem, bool lng, bool per, bool shared,
                            int G, size_t smem, int *blocks_per_sm);
cudaError_t pgram_launch(int precision, int variant, bool gmem, bool lng, bool per, bool shared,
                         int grid, int G, size_t smem, const PgramArgs &a, cudaStream_t s);

size_t pgram_small_bytes(int precision, int G, int variant);
size_t pgram_frame_bytes(int precision, int n, int variant, bool keep_perm, bool smo_out = false);

}  // namespace ssp
