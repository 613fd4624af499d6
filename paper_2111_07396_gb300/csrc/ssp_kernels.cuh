// ssp_kernels.cuh -- per-object preparation and per-object argmax kernels,
// and the launch wrappers instantiated once per precision (ssp_fp32.cu,
// ssp_fp64.cu define SSP_R and SSP_PREC before including this file).
#pragma once
#include <cfloat>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "ssp_launch.h"

namespace ssp {

__device__ inline double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Alg. 1 compute_chi0_tt_weights, one CTA per object: tt = t - min t,
// w = dy^-2, ybar = sum w y / sum w, chi0 = sum w (y - ybar)^2; the smoother's
// inputs are stored in R (magnitudes centred on ybar, which leaves chi2
// unchanged because every running line reproduces constants) and, for the
// FP32C path, also in binary64 for the recompute of flagged frequencies.
template <typename R>
__global__ void __launch_bounds__(256) prep_kernel(PrepArgs a)
{
    __shared__ double s_red[4][8];
    __shared__ int s_bad[8];
    const int o = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = a.off[o];
    const int n = (int)(a.off[o + 1] - base);
    double tmin = INFINITY, sw = 0.0, swy = 0.0;
    int bad = 0;
    for (int i = tid; i < n; i += blockDim.x) {
        const double t = a.t[base + i], y = a.y[base + i], dy = a.dy[base + i];
        if (!isfinite(t) || !isfinite(y) || !isfinite(dy) || !(dy > 0.0)) bad = 1;
        const double w = __ddiv_rn(1.0, __dmul_rn(dy, dy));
        if (!(w > 0.0) || !isfinite(w)) bad = 1;
        if (sizeof(R) == 4 && !(w >= (double)FLT_MIN && w <= (double)FLT_MAX)) bad = 1;
        tmin = fmin(tmin, t);
        sw += w;
        swy += w * y;
    }
    for (int off = 16; off > 0; off >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, off));
    sw = warp_sum(sw);
    swy = warp_sum(swy);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        s_red[0][warp] = tmin;
        s_red[2][warp] = sw;
        s_red[3][warp] = swy;
        s_bad[warp] = bad;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    tmin = s_red[0][0];
    sw = 0.0;
    swy = 0.0;
    bad = 0;
    for (int k = 0; k < nw; ++k) {
        tmin = fmin(tmin, s_red[0][k]);
        sw += s_red[2][k];
        swy += s_red[3][k];
        bad |= s_bad[k];
    }
    __syncthreads();
    const double ybar = swy / sw;
    double c0 = 0.0, ym = 0.0;
    R *yc = (R *)a.yc + base;
    R *wv = (R *)a.wv + base;
    for (int i = tid; i < n; i += blockDim.x) {
        const double t = a.t[base + i], y = a.y[base + i], dy = a.dy[base + i];
        const double w = __ddiv_rn(1.0, __dmul_rn(dy, dy));
        const double tt = __dsub_rn(t, tmin);
        const double d = y - ybar;
        c0 += w * d * d;
        ym = fmax(ym, fabs(d));
        a.tt[base + i] = tt;
        yc[i] = (R)d;
        wv[i] = (R)w;
        if (a.yc64) {
            a.yc64[base + i] = d;
            a.wv64[base + i] = w;
        }
        if (a.ydf) {
            const float dh = (float)d, wh = (float)w;
            a.ydf[base + i] = make_float2(dh, (float)(d - (double)dh));
            a.wdf[base + i] = make_float2(wh, (float)(w - (double)wh));
        }
    }
    c0 = warp_sum(c0);
    for (int off = 16; off > 0; off >>= 1) ym = fmax(ym, __shfl_xor_sync(0xffffffffu, ym, off));
    if (lane == 0) {
        s_red[0][warp] = c0;
        s_red[1][warp] = ym;
    }
    __syncthreads();
    if (tid == 0) {
        double c = 0.0, m = 0.0;
        for (int k = 0; k < nw; ++k) {
            c += s_red[0][k];
            m = fmax(m, s_red[1][k]);
        }
        a.chi0[o] = c;
        a.ymax[o] = m;
        a.bad[o] = bad;
    }
}

// findPeriod (Alg. 1): first index of the largest power, period = 1/f.
template <typename R>
__global__ void __launch_bounds__(256) argmax_kernel(ArgmaxArgs a)
{
    __shared__ double s_v[8];
    __shared__ long long s_i[8];
    const int o = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const R *row = (const R *)a.power + (int64_t)o * a.n_freq;
    double bv = -INFINITY;
    long long bi = -1;
    for (int64_t q = tid; q < a.n_freq; q += blockDim.x) {
        const double v = (double)row[q];
        if (v > bv) { bv = v; bi = q; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_v[warp] = bv; s_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            const double ov = s_v[k];
            const long long oi = s_i[k];
            if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) { bv = ov; bi = oi; }
        }
        const double *fq = a.freq + (a.fbase ? a.fbase[o] : 0);
        const bool nan = a.bad[o] || bi < 0;
        a.best_period[o] = nan ? __longlong_as_double(0x7ff8000000000000LL) : 1.0 / fq[bi];
        if (a.best_power) a.best_power[o] = nan ? __longlong_as_double(0x7ff8000000000000LL) : bv;
    }
}

// Search-and-refine (the outlook of Sec. 6), one CTA per object: k rounds
// pick the largest local maximum of the coarse power row (p[q] >= p[q-1]
// and p[q] > p[q+1], a missing neighbour counting as lower; ties to the
// lower index) that is not next to one already taken; fewer than k maxima
// repeat the first.  Each peak q gets n_fine frequencies evenly from
// f[q-1] to f[q+1] (one coarse step beyond q at either end of the grid; a
// start at or below 0 moves to f[q]/2).
template <typename R>
__global__ void __launch_bounds__(256) peaks_kernel(PeaksArgs a)
{
    __shared__ double s_v[8];
    __shared__ long long s_i[8];
    __shared__ long long s_taken[64];
    __shared__ int s_count;
    const int o = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    const R *p = (const R *)a.power + (int64_t)o * a.n_coarse;
    const int64_t n = a.n_coarse;
    if (tid == 0) s_count = 0;
    __syncthreads();
    for (int round = 0; round < a.k; ++round) {
        const int taken = s_count;
        double bv = -INFINITY;
        long long bi = -1;
        for (int64_t q = tid; q < n; q += blockDim.x) {
            const R v = p[q];
            if (!((q == 0 || v >= p[q - 1]) && (q == n - 1 || v > p[q + 1]))) continue;
            bool skip = false;
            for (int i = 0; i < taken; ++i)
                if (s_taken[i] >= q - 1 && s_taken[i] <= q + 1) skip = true;
            if (skip) continue;
            if (bi < 0 || (double)v > bv) { bv = (double)v; bi = q; }   // q ascends: ties keep the lower
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
            const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
        }
        if (lane == 0) { s_v[warp] = bv; s_i[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nw; ++w) {
                const double ov = s_v[w];
                const long long oi = s_i[w];
                if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
            }
            if (bi >= 0) s_taken[s_count++] = bi;
        }
        __syncthreads();
        if (s_count == taken) break;   // no maximum left
    }
    const int got = s_count;
    double *out = a.fine + (int64_t)o * a.k * a.n_fine;
    for (int i = tid; i < a.k * a.n_fine; i += blockDim.x) {
        const int pk = i / a.n_fine, j = i - pk * a.n_fine;
        const long long q = got > 0 ? s_taken[pk < got ? pk : 0] : 0;
        const double *f = a.coarse;
        const double step_lo = q > 0 ? f[q] - f[q - 1] : (n > 1 ? f[1] - f[0] : 0.0);
        const double step_hi = q < n - 1 ? f[q + 1] - f[q] : (n > 1 ? f[n - 1] - f[n - 2] : 0.0);
        double lo = f[q] - step_lo;
        const double hi = f[q] + step_hi;
        if (!(lo > 0.0)) lo = 0.5 * f[q];
        out[i] = a.n_fine > 1 ? lo + (hi - lo) * (double)j / (double)(a.n_fine - 1) : f[q];
    }
}

}  // namespace ssp

// prep and argmax kernels of one precision
#define SSP_INSTANTIATE_PREP(R, PREC)                                                         \
    namespace ssp {                                                                           \
    cudaError_t prep_launch_##PREC(const PrepArgs &a, int n_obj, cudaStream_t s)              \
    {                                                                                         \
        prep_kernel<R><<<n_obj, 256, 0, s>>>(a);                                              \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    cudaError_t argmax_launch_##PREC(const ArgmaxArgs &a, int n_obj, cudaStream_t s)          \
    {                                                                                         \
        argmax_kernel<R><<<n_obj, 256, 0, s>>>(a);                                            \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    cudaError_t peaks_launch_##PREC(const PeaksArgs &a, int n_obj, cudaStream_t s)            \
    {                                                                                         \
        peaks_kernel<R><<<n_obj, 256, 0, s>>>(a);                                             \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    }

// A kernel's dynamic shared-memory limit is one setting per function and
// device for the whole process, read when a launch is enqueued.  Plans are
// built and launched by several host threads (the serving loop's launcher
// beside direct calls), so the limit is only ever raised: lowering it for a
// small plan could fail another thread's launch that was planned with more
// ("invalid argument").
namespace ssp {
inline cudaError_t raise_smem_limit(void (*kernel)(PgramArgs), int smem)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> cur;   // (device, kernel) -> limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    int &c = cur[std::make_pair(dev, (const void *)kernel)];
    if (c >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) c = smem;
    return e;
}
}  // namespace ssp

// periodogram kernels of one precision, accumulator and window mode (PER:
// periodic windows, else clamped inside the data); SHARED: work items may
// cover several objects with identical times; WL: also the SS kernels that
// initialise windows out of line, for long objects; SUF names the functions
#define SSP_INSTANTIATE_PGRAM(R, PLAIN, PER, SHARED, SUF, WL)                                  \
    namespace ssp {                                                                           \
    template <int V, bool GM, bool L>                                                         \
    static cudaError_t occ_##SUF(int G, size_t smem, int *bps)                                \
    {                                                                                         \
        cudaError_t e = raise_smem_limit(pgram_kernel<R, V, GM, PLAIN, PER, SHARED, L>,       \
                                         (int)smem);                                          \
        if (e != cudaSuccess) return e;                                                       \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                 \
            bps, pgram_kernel<R, V, GM, PLAIN, PER, SHARED, L>, G, smem);                     \
    }                                                                                         \
    template <int V, bool L>                                                                  \
    static cudaError_t occ2_##SUF(bool gmem, int G, size_t smem, int *bps)                    \
    {                                                                                         \
        return gmem ? occ_##SUF<V, true, L>(G, smem, bps) : occ_##SUF<V, false, L>(G, smem, bps); \
    }                                                                                         \
    cudaError_t pgram_occupancy_##SUF(int variant, bool gmem, bool lng, int G, size_t smem,   \
                                      int *bps)                                               \
    {                                                                                         \
        switch (variant) {                                                                    \
        case VAR_SS:                                                                          \
            if constexpr (WL) {                                                               \
                if (lng) return occ2_##SUF<VAR_SS, true>(gmem, G, smem, bps);                 \
            }                                                                                 \
            return occ2_##SUF<VAR_SS, false>(gmem, G, smem, bps);                             \
        case VAR_SP: return occ2_##SUF<VAR_SP, false>(gmem, G, smem, bps);                    \
        case VAR_SPG: return occ2_##SUF<VAR_SPG, false>(gmem, G, smem, bps);                  \
        default: return occ2_##SUF<VAR_FIXED, false>(gmem, G, smem, bps);                     \
        }                                                                                     \
    }                                                                                         \
    template <int V, bool L>                                                                  \
    static void launch2_##SUF(bool gmem, int grid, int G, size_t smem, const PgramArgs &a,    \
                              cudaStream_t s)                                                 \
    {                                                                                         \
        if (gmem) pgram_kernel<R, V, true, PLAIN, PER, SHARED, L><<<grid, G, smem, s>>>(a);   \
        else pgram_kernel<R, V, false, PLAIN, PER, SHARED, L><<<grid, G, smem, s>>>(a);       \
    }                                                                                         \
    cudaError_t pgram_launch_##SUF(int variant, bool gmem, bool lng, int grid, int G,         \
                                   size_t smem, const PgramArgs &a, cudaStream_t s)           \
    {                                                                                         \
        switch (variant) {                                                                    \
        case VAR_SS:                                                                          \
            if constexpr (WL) {                                                               \
                if (lng) {                                                                    \
                    launch2_##SUF<VAR_SS, true>(gmem, grid, G, smem, a, s);                   \
                    break;                                                                    \
                }                                                                             \
            }                                                                                 \
            launch2_##SUF<VAR_SS, false>(gmem, grid, G, smem, a, s);                          \
            break;                                                                            \
        case VAR_SP: launch2_##SUF<VAR_SP, false>(gmem, grid, G, smem, a, s); break;          \
        case VAR_SPG: launch2_##SUF<VAR_SPG, false>(gmem, grid, G, smem, a, s); break;        \
        default: launch2_##SUF<VAR_FIXED, false>(gmem, grid, G, smem, a, s);                  \
        }                                                                                     \
        return cudaGetLastError();                                                            \
    }                                                                                         \
    }

// shared-memory sizes of one precision and accumulator
#define SSP_INSTANTIATE_SIZES(R, PLAIN, PREC)                                                 \
    namespace ssp {                                                                           \
    size_t pgram_small_bytes_##PREC(int G, int variant)                                       \
    {                                                                                         \
        return small_bytes<typename AccSel<R, PLAIN>::T>(G, variant);                         \
    }                                                                                         \
    size_t pgram_frame_bytes_##PREC(int n, int variant, bool keep_perm, bool smo_out)         \
    {                                                                                         \
        return frame_bytes<R>(n, variant, keep_perm, smo_out);                                \
    }                                                                                         \
    }
