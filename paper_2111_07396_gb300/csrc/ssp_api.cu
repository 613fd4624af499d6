// ssp_api.cu -- the C ABI of libssp (include/ssp.h): argument checks, the
// launch planner (length buckets, work items, device-memory batches) and the
// host/device entry points.  All arithmetic of the method runs in the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ssp.h"
#include "ssp_fold.h"
#include "ssp_internal.h"
#include "ssp_launch.h"

namespace ssp {
cudaError_t prep_launch_fp32(const PrepArgs &, int, cudaStream_t);
cudaError_t prep_launch_fp64(const PrepArgs &, int, cudaStream_t);
cudaError_t argmax_launch_fp32(const ArgmaxArgs &, int, cudaStream_t);
cudaError_t argmax_launch_fp64(const ArgmaxArgs &, int, cudaStream_t);
cudaError_t peaks_launch_fp32(const PeaksArgs &, int, cudaStream_t);
cudaError_t peaks_launch_fp64(const PeaksArgs &, int, cudaStream_t);
cudaError_t pgram_occupancy_fp32_per(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_fp32_per(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
cudaError_t pgram_occupancy_fp32_clamp(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_fp32_clamp(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
cudaError_t pgram_occupancy_fp64_per(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_fp64_per(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
cudaError_t pgram_occupancy_fp64_clamp(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_fp64_clamp(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
cudaError_t pgram_occupancy_redo_per(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_redo_per(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
cudaError_t pgram_occupancy_redo_clamp(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_redo_clamp(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
cudaError_t pgram_occupancy_fp32_shared(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_fp32_shared(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
cudaError_t pgram_occupancy_fp64_shared(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_fp64_shared(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
cudaError_t pgram_occupancy_redo_shared(int, bool, bool, int, size_t, int *);
cudaError_t pgram_launch_redo_shared(int, bool, bool, int, int, size_t, const PgramArgs &, cudaStream_t);
size_t pgram_small_bytes_fp32(int, int);
size_t pgram_frame_bytes_fp32(int, int, bool, bool);
size_t pgram_small_bytes_fp64(int, int);
size_t pgram_frame_bytes_fp64(int, int, bool, bool);
size_t pgram_small_bytes_redo(int, int);
size_t pgram_frame_bytes_redo(int, int, bool, bool);

cudaError_t prep_launch(int p, const PrepArgs &a, int n, cudaStream_t s)
{
    return p == SSP_FP64 ? prep_launch_fp64(a, n, s) : prep_launch_fp32(a, n, s);
}
cudaError_t argmax_launch(int p, const ArgmaxArgs &a, int n, cudaStream_t s)
{
    return p == SSP_FP64 ? argmax_launch_fp64(a, n, s) : argmax_launch_fp32(a, n, s);
}
cudaError_t peaks_launch(int p, const PeaksArgs &a, int n, cudaStream_t s)
{
    return p == SSP_FP64 ? peaks_launch_fp64(a, n, s) : peaks_launch_fp32(a, n, s);
}
cudaError_t pgram_occupancy(int p, int v, bool g, bool lng, bool per, bool shared, int G,
                            size_t smem, int *bps)
{
    if (shared)   // periodic windows only
        return p == SSP_FP64 ? pgram_occupancy_fp64_shared(v, g, lng, G, smem, bps)
             : p == kPrecRedo ? pgram_occupancy_redo_shared(v, g, lng, G, smem, bps)
                              : pgram_occupancy_fp32_shared(v, g, lng, G, smem, bps);
    if (per)
        return p == SSP_FP64 ? pgram_occupancy_fp64_per(v, g, lng, G, smem, bps)
             : p == kPrecRedo ? pgram_occupancy_redo_per(v, g, lng, G, smem, bps)
                              : pgram_occupancy_fp32_per(v, g, lng, G, smem, bps);
    return p == SSP_FP64 ? pgram_occupancy_fp64_clamp(v, g, lng, G, smem, bps)
         : p == kPrecRedo ? pgram_occupancy_redo_clamp(v, g, lng, G, smem, bps)
                          : pgram_occupancy_fp32_clamp(v, g, lng, G, smem, bps);
}
cudaError_t pgram_launch(int p, int v, bool g, bool lng, bool per, bool shared, int grid, int G,
                         size_t smem, const PgramArgs &a, cudaStream_t s)
{
    if (shared)   // periodic windows only
        return p == SSP_FP64 ? pgram_launch_fp64_shared(v, g, lng, grid, G, smem, a, s)
             : p == kPrecRedo ? pgram_launch_redo_shared(v, g, lng, grid, G, smem, a, s)
                              : pgram_launch_fp32_shared(v, g, lng, grid, G, smem, a, s);
    if (per)
        return p == SSP_FP64 ? pgram_launch_fp64_per(v, g, lng, grid, G, smem, a, s)
             : p == kPrecRedo ? pgram_launch_redo_per(v, g, lng, grid, G, smem, a, s)
                              : pgram_launch_fp32_per(v, g, lng, grid, G, smem, a, s);
    return p == SSP_FP64 ? pgram_launch_fp64_clamp(v, g, lng, grid, G, smem, a, s)
         : p == kPrecRedo ? pgram_launch_redo_clamp(v, g, lng, grid, G, smem, a, s)
                          : pgram_launch_fp32_clamp(v, g, lng, grid, G, smem, a, s);
}
size_t pgram_small_bytes(int p, int G, int variant)
{
    return p == SSP_FP64 ? pgram_small_bytes_fp64(G, variant)
         : p == kPrecRedo ? pgram_small_bytes_redo(G, variant)
                          : pgram_small_bytes_fp32(G, variant);
}
size_t pgram_frame_bytes(int p, int n, int variant, bool keep_perm, bool smo_out)
{
    return p == SSP_FP64 ? pgram_frame_bytes_fp64(n, variant, keep_perm, smo_out)
         : p == kPrecRedo ? pgram_frame_bytes_redo(n, variant, keep_perm, smo_out)
                          : pgram_frame_bytes_fp32(n, variant, keep_perm, smo_out);
}
}  // namespace ssp

using namespace ssp;

namespace ssp_internal {
std::atomic<int> g_fault_alloc{0}, g_fault_stall{0}, g_fault_upload{0};

bool testing()
{
    const char *e = std::getenv("SSP_TESTING");
    return e && std::strcmp(e, "1") == 0;
}

// one countdown step of an injected fault: true while the count lasts
static bool take_fault(std::atomic<int> &c)
{
    int v = c.load();
    while (v > 0)
        if (c.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s)
{
    if (take_fault(g_fault_alloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;   // as the allocator reports it; nothing was allocated
    }
    return cudaMallocAsync(p, bytes, s);
}

bool stall_injected() { return take_fault(g_fault_stall); }
bool upload_fault_injected() { return take_fault(g_fault_upload); }
}  // namespace ssp_internal

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(SSP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SSP_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr int kMaxN = 65535;
// device bytes set aside per batch for the per-CTA frames of large objects
constexpr double kSlabReserve = 2.0e9;

int check_params(const ssp_params *p)
{
    if (!(p->spans[0] > 0.0 && p->spans[0] < p->spans[1] && p->spans[1] < p->spans[2] &&
          p->spans[2] <= 1.0))
        return fail(SSP_ERR_ARG, "spans must satisfy 0 < s0 < s1 < s2 <= 1");
    if (!(p->alpha >= 0.0 && p->alpha <= 10.0)) return fail(SSP_ERR_ARG, "alpha must be in [0, 10]");
    if (p->precision != SSP_FP64 && p->precision != SSP_FP32C)
        return fail(SSP_ERR_ARG, "unknown precision %d", (int)p->precision);
    if (!(p->hbm_fraction > 0.0 && p->hbm_fraction <= 1.0))
        return fail(SSP_ERR_ARG, "hbm_fraction must be in (0, 1]");
    if (p->periodic != 0 && p->periodic != 1) return fail(SSP_ERR_ARG, "periodic must be 0 or 1");
    if (!(p->span >= 0.0 && p->span <= 1.0)) return fail(SSP_ERR_ARG, "span must be in [0, 1]");
    return SSP_OK;
}

int check_shape(const int64_t *n_per_object, int64_t n_objects, int64_t n_freq, ssp_variant v)
{
    if (n_objects < 1) return fail(SSP_ERR_ARG, "n_objects must be >= 1");
    if (n_objects > (int64_t)1 << 30) return fail(SSP_ERR_ARG, "n_objects too large");
    if (n_freq < 1) return fail(SSP_ERR_ARG, "n_freq must be >= 1");
    // work items carry frequency bounds as int
    if (n_freq > (int64_t)INT32_MAX) return fail(SSP_ERR_ARG, "n_freq too large (at most 2^31 - 1)");
    if (v != SSP_SS && v != SSP_SP && v != SSP_SPG)
        return fail(SSP_ERR_ARG, "unknown variant %d", (int)v);
    if (!n_per_object) return fail(SSP_ERR_ARG, "n_per_object is NULL");
    for (int64_t o = 0; o < n_objects; ++o) {
        if (n_per_object[o] < 4)
            return fail(SSP_ERR_ARG, "object %lld has %lld points; at least 4 are needed",
                        (long long)o, (long long)n_per_object[o]);
        if (n_per_object[o] > kMaxN)
            return fail(SSP_ERR_ARG, "object %lld has %lld points; at most %d are supported",
                        (long long)o, (long long)n_per_object[o], kMaxN);
    }
    return SSP_OK;
}

// Objects are planned in length ranges; the objects of one range share a
// launch.  Threads per CTA by default: about a dozen centres per thread
// (SSP_GROUP_SCALE, a power of two, scales the rule for calibration under
// SSP_TESTING=1; read once per process).  FP32C
// SS objects above 2048 points take 256 threads when pass A's smooths live
// in the global slab (their frame then leaves room for two CTAs per SM), and
// 512 otherwise (one CTA per SM: 16 warps hide more latency than 8; the FP64
// kernel, bound by its FP64 pipe, runs slower that way).  ssp_autotune
// replaces the rule per (precision, variant, range) with measured choices.
constexpr int kRanges = 5;
constexpr int kRangeMax[kRanges] = {384, 768, 1536, 2048, 65535};
std::atomic<int> g_tuned[2][4][kRanges];   // [precision][kernel variant][range]; 0 = rule

int range_of(int n)
{
    for (int r = 0; r < kRanges; ++r)
        if (n <= kRangeMax[r]) return r;
    return kRanges - 1;
}

int group_size_rule(int n, int variant, int precision, bool smo_ok = true)
{
    static const int scale = [] {
        const char *e = ssp_internal::testing() ? std::getenv("SSP_GROUP_SCALE") : nullptr;
        const int v = e ? std::atoi(e) : 0;
        return (v == 2 || v == 4 || v == -2 || v == -4) ? v : 1;
    }();
    int g;
    if (n <= 384) g = 32;
    else if (n <= 768) g = 64;
    else if (n <= 2048) g = 128;   // 12-16 centres per thread
    else if (variant == SSP_SS && precision == SSP_FP32C) g = smo_ok ? 256 : 512;
    else g = 256;
    if (scale > 1) g = std::min(512, g * scale);
    if (scale < 0) g = std::max(32, g / -scale);
    return g;
}

// the kernel a request runs: SS, SP, or (a fixed span, either variant) the
// single smooth
int kernel_variant(ssp_variant v, const ssp_params &P)
{
    if (P.span > 0.0) return VAR_FIXED;
    return v == SSP_SS ? VAR_SS : v == SSP_SP ? VAR_SP : VAR_SPG;
}

int group_size(int n, int variant, int precision, bool smo_ok = true)
{
    const int t = g_tuned[precision == SSP_FP64 ? 0 : 1][variant][range_of(n)].load();
    return t ? t : group_size_rule(n, variant, precision, smo_ok);
}

struct LaunchCfg {
    bool gmem = false;
    bool cnt_smem = false;   // gmem: the sort's bucket counts in shared memory
    bool lng = false;        // SS kernel that initialises windows out of line
    bool smo_out = false;    // SS: pass A's smooths in the global slab
    bool redo_inline = false; // SS: flagged frequencies recomputed in binary64 in the kernel
    size_t smem = 0, slab_bytes = 0, smo_stride = 0, redo_slab_bytes = 0;
    int grid = 0;
};

struct Bucket {
    int G = 32, n_max = 0;
    int G_redo = 32;        // threads per CTA of the FP64 recompute launch
    bool shared = false;    // some item covers several objects with identical times
    LaunchCfg main, redo;   // redo: FP64 recompute of flagged FP32C frequencies
    std::vector<int> objects;
    std::vector<int4> items;
};

struct Plan {
    std::vector<Bucket> buckets;
    size_t items_total = 0, slab_total = 0, smo_total = 0, redo_total = 0;
    bool redo = false;
};

int device_limits(int *num_sms, size_t *max_smem)
{
    int dev = 0, sms = 0, optin = 0;
    SSP_CUDA(cudaGetDevice(&dev));
    SSP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    *num_sms = sms;
    *max_smem = (size_t)optin;
    return SSP_OK;
}

// frame placement and persistent grid of one kernel for one bucket
int configure(int precision, int variant, bool per, bool shared, int G, int n_max, int sms,
              size_t max_smem, LaunchCfg &c, bool smo_ok = true)
{
    // FP32C SS objects of many points keep pass A's smooths in the global slab
    // (coalesced), which shrinks their frame by 12 bytes a point.  Only the
    // kernels built for long objects (LONG: periodic windows, shared or not)
    // address the slab; the frame layout here and in the kernel must agree.
    const bool long_kernel = variant == VAR_SS && precision == SSP_FP32C && n_max > kLongN &&
                             (per || shared);
    c.smo_out = smo_ok && long_kernel;
    c.smo_stride = c.smo_out ? align16(smo_bytes(n_max, G, 4)) +
                                   (shared ? kept_perm_bytes(n_max) : 0)
                             : 0;
    // the same kernels recompute their flagged frequencies in binary64 at once,
    // in per-CTA binary64 frames in global memory
    c.redo_inline = c.smo_out;
    c.redo_slab_bytes = c.redo_inline ? align16(pgram_frame_bytes(kPrecRedo, n_max, variant, false)) : 0;
    const size_t small = align16(pgram_small_bytes(precision, G, variant));
    const size_t frame = align16(pgram_frame_bytes(precision, n_max, variant, shared, c.smo_out));
    c.gmem = small + frame + 1024 > max_smem;
    // a single-sweep frame in global memory keeps its sort's bucket counts in
    // shared memory where they fit (C4 SP: 9% faster).  SS does not: its
    // streaming passes need the L1 that the counts would take (19% slower).
    const size_t cnt = align16(4 * (size_t)bucket_count(n_max));
    c.cnt_smem = c.gmem && variant != VAR_SS && small + cnt + 1024 <= max_smem;
    c.smem = c.gmem ? small + (c.cnt_smem ? cnt : 0) : small + frame;
    c.slab_bytes = c.gmem ? frame : 0;
    int bps = 0;
    // objects of many points (long windows, few centres per thread) take the SS
    // kernel whose window initialisation is out of line (FP32C: the only
    // precision it is built for)
    c.lng = variant == VAR_SS && precision == SSP_FP32C && n_max > kLongN;
    cudaError_t e = pgram_occupancy(precision, variant, c.gmem, c.lng, per, shared, G, c.smem,
                                    &bps);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (bps < 1) return fail(SSP_ERR_NOMEM, "a CTA frame for n = %d does not fit", n_max);
    c.grid = bps * sms;
    return SSP_OK;
}

// Length buckets (one launch each, sized for the bucket's largest object),
// work items (object, frequency range) ordered longest first.
// group (host, or null): group[o] = number of objects o, o+1, ... that share
// object o's times when o leads such a run, 0 for the run's other objects
int build_plan(const int64_t *npo, int64_t n_obj, int64_t n_freq, int precision, int variant,
               bool per, Plan &plan, const int *group = nullptr, bool smo_ok = true)
{
    int sms = 0;
    size_t max_smem = 0;
    int rc = device_limits(&sms, &max_smem);
    if (rc) return rc;
    plan.buckets.clear();
    plan.redo = precision == SSP_FP32C;
    for (int r = 0; r < kRanges; ++r) {
        Bucket b;
        for (int64_t o = 0; o < n_obj; ++o)
            if (range_of((int)npo[o]) == r && (!group || group[o] > 0)) {
                b.objects.push_back((int)o);
                b.n_max = std::max(b.n_max, (int)npo[o]);
                if (group && group[o] > 1) b.shared = true;
            }
        if (b.objects.empty()) continue;
        // (the smooth slab exists only for periodic windows: see configure)
        const bool slab_ok = smo_ok && (per || b.shared);
        b.G = group_size(b.n_max, variant, precision, slab_ok);
        if (b.G == 256 && slab_ok && variant == VAR_SS && precision == SSP_FP32C && b.n_max > 2048 &&
            !g_tuned[1][variant][range_of(b.n_max)].load()) {
            // 256 threads only where two CTAs of them fit an SM's shared memory
            // with the smooths in the global slab; otherwise 512 (one CTA)
            const size_t need = align16(pgram_small_bytes(precision, 256, variant)) +
                                align16(pgram_frame_bytes(precision, b.n_max, variant, b.shared, true)) +
                                1024;
            if (2 * need > max_smem + 1024) b.G = 512;
        }
        // the kernels split chunks and scans by shifts: a power of two, 32..512
        if (b.G < 32 || b.G > 512 || (b.G & (b.G - 1)) != 0)
            return fail(SSP_ERR_ARG, "threads per CTA must be a power of two in 32..512, not %d", b.G);
        plan.buckets.push_back(std::move(b));
    }
    plan.items_total = 0;
    plan.slab_total = 0;
    plan.smo_total = 0;
    plan.redo_total = 0;
    for (Bucket &b : plan.buckets) {
        rc = configure(precision, variant, per, b.shared, b.G, b.n_max, sms, max_smem, b.main, smo_ok);
        if (rc) return rc;
        if (plan.redo) {
            b.G_redo = b.G;
            rc = configure(kPrecRedo, variant, per, b.shared, b.G_redo, b.n_max, sms, max_smem, b.redo);
            if (rc) return rc;
        }
        const int resident = b.main.grid;
        // enough items for dynamic balance: ~8 per resident CTA
        const int64_t want = std::max<int64_t>(8LL * resident, (int64_t)b.objects.size());
        int64_t per_obj = (want + (int64_t)b.objects.size() - 1) / (int64_t)b.objects.size();
        per_obj = std::max<int64_t>(1, std::min<int64_t>(per_obj, n_freq));
        const int64_t chunk = (n_freq + per_obj - 1) / per_obj;
        std::vector<std::pair<int64_t, int4>> keyed;
        for (int o : b.objects) {
            const int m = group ? group[o] : 1;
            for (int64_t q0 = 0; q0 < n_freq; q0 += chunk) {
                const int q1 = (int)std::min<int64_t>(n_freq, q0 + chunk);
                keyed.push_back({-(int64_t)npo[o] * m * (q1 - q0), make_int4(o, (int)q0, q1, m)});
            }
        }
        std::stable_sort(keyed.begin(), keyed.end(),
                         [](const auto &x, const auto &y) { return x.first < y.first; });
        b.items.resize(keyed.size());
        for (size_t k = 0; k < keyed.size(); ++k) b.items[k] = keyed[k].second;
        b.main.grid = (int)std::min<int64_t>((int64_t)b.items.size(), b.main.grid);
        b.redo.grid = (int)std::min<int64_t>((int64_t)b.items.size(), b.redo.grid);
        plan.items_total += b.items.size();
        plan.slab_total += b.main.gmem ? b.main.slab_bytes * (size_t)b.main.grid : 0;
        plan.smo_total += b.main.smo_stride * (size_t)b.main.grid;
        plan.redo_total += b.main.redo_slab_bytes * (size_t)b.main.grid;
        if (plan.redo && b.redo.gmem && !b.main.redo_inline)
            plan.slab_total += b.redo.slab_bytes * (size_t)b.redo.grid;
    }
    return SSP_OK;
}

size_t rsize(int precision) { return precision == SSP_FP64 ? 8 : 4; }

// FP32C margins, overridable for testing and tuning by SSP_NEAR_SS,
// SSP_NEAR_SP, SSP_SENS_TAU, SSP_SENS_ULPS and SSP_REFIT_FRAC (a value of 1e6
// or more keeps the default; a negative margin disables its test), honoured
// only while SSP_TESTING=1: a stray variable cannot change the numerics
float near_margin(const char *env, float dflt)
{
    if (!ssp_internal::testing()) return dflt;
    const char *e = std::getenv(env);
    if (e && *e) {
        const double v = std::atof(e);
        if (v < 1e6) return (float)v;
    }
    return dflt;
}

// device bytes of one batch apart from the caller's arrays
size_t workspace_bytes(const Plan &plan, int64_t n_obj, int64_t n_points, int64_t n_freq,
                       int precision)
{
    size_t b = 0;
    b += align16(8 * (size_t)(n_obj + 1));                  // off
    b += align16(8 * (size_t)n_points);                     // tt
    b += align16(4 * (size_t)n_obj);                        // bad
    b += align16(rsize(precision) * (size_t)n_points) * 2;  // yc, wv
    if (plan.redo) b += align16(8 * (size_t)n_points) * 4;  // FP64 copies, double-float pairs
    b += align16(8 * (size_t)n_obj);                        // chi0
    b += align16(8 * (size_t)n_obj);                        // ymax
    b += align16(sizeof(int4) * plan.items_total);
    b += align16(8 * plan.buckets.size() + 8);              // two counters per bucket
    if (plan.redo) b += align16((size_t)n_obj * (size_t)n_freq);  // near flags
    b += plan.slab_total;
    b += plan.smo_total;
    b += plan.redo_total;
    return b;
}

// ---- per-phase event timers ----
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
struct Mark {
    int phase;
    cudaEvent_t a, b;
};
std::vector<Mark> g_marks;

bool prof_begin(int phase, cudaStream_t s, Mark &m)
{
    if (!g_prof_on) return false;
    m.phase = phase;
    if (cudaEventCreate(&m.a) != cudaSuccess) return false;
    if (cudaEventCreate(&m.b) != cudaSuccess) {
        cudaEventDestroy(m.a);
        return false;
    }
    cudaEventRecord(m.a, s);
    return true;
}

// a launch failed after prof_begin: its two events are never recorded
void prof_drop(bool on, Mark &m)
{
    if (!on) return;
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
}

void prof_end(bool on, Mark &m, cudaStream_t s)
{
    if (!on) return;
    cudaEventRecord(m.b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_marks.push_back(m);
}

void keep_pool_memory()
{
    // keep freed stream-ordered memory cached in the pool between calls
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}


// The whole device path of one batch, enqueued on stream s.
// value rules for host inputs: finite t and y, finite dy > 0 whose weight is
// finite (and within float range for SSP_FP32C)
int check_values(const double *t, const double *y, const double *dy, int64_t N, int precision)
{
    for (int64_t i = 0; i < N; ++i) {
        if (!std::isfinite(t[i]) || !std::isfinite(y[i]))
            return fail(SSP_ERR_ARG, "t or y at point %lld is not finite", (long long)i);
        if (!std::isfinite(dy[i]) || !(dy[i] > 0.0))
            return fail(SSP_ERR_ARG, "dy at point %lld must be finite and > 0", (long long)i);
        const double w = 1.0 / (dy[i] * dy[i]);
        if (!(w > 0.0) || !std::isfinite(w))
            return fail(SSP_ERR_ARG, "dy at point %lld gives a weight outside binary64", (long long)i);
        if (precision == SSP_FP32C && !(w >= 1.1754943508222875e-38 && w <= 3.4028234663852886e38))
            return fail(SSP_ERR_UNSUPPORTED,
                        "dy at point %lld gives a weight outside float range; use SSP_FP64",
                        (long long)i);
    }
    return SSP_OK;
}

// Objects of one batch whose time arrays are bitwise equal (same survey
// cadence) share each frequency's fold and sort.  order lists the batch's
// objects (indices from o0) with every such run adjacent, its leader first;
// group holds the run length at each leader and 0 at the others.
struct Grouping {
    std::vector<int64_t> order, npo;
    std::vector<int> group;
    bool any = false;
};

Grouping group_by_times(const double *t, const int64_t *npo, int64_t o0, int64_t o1, int64_t p0)
{
    const int64_t nb = o1 - o0;
    std::vector<int64_t> off((size_t)nb + 1, p0);
    for (int64_t k = 0; k < nb; ++k) off[k + 1] = off[k] + npo[o0 + k];
    std::vector<std::pair<uint64_t, int64_t>> hk((size_t)nb);
    for (int64_t k = 0; k < nb; ++k) {
        uint64_t h = 1469598103934665603ull ^ (uint64_t)npo[o0 + k];   // FNV-1a
        const unsigned char *b = (const unsigned char *)(t + off[k]);
        for (size_t i = 0; i < 8 * (size_t)npo[o0 + k]; ++i) h = (h ^ b[i]) * 1099511628211ull;
        hk[(size_t)k] = {h, k};
    }
    std::sort(hk.begin(), hk.end());
    std::vector<int64_t> lead((size_t)nb, -1);   // each object's group leader
    for (size_t a = 0; a < hk.size();) {
        size_t b = a;
        while (b < hk.size() && hk[b].first == hk[a].first) ++b;
        std::vector<int64_t> leaders;
        for (size_t i = a; i < b; ++i) {
            const int64_t k = hk[i].second, n = npo[o0 + k];
            for (int64_t L : leaders)
                if (npo[o0 + L] == n &&
                    std::memcmp(t + off[L], t + off[k], 8 * (size_t)n) == 0) {
                    lead[(size_t)k] = L;
                    break;
                }
            if (lead[(size_t)k] < 0) {
                lead[(size_t)k] = k;
                leaders.push_back(k);
            }
        }
        a = b;
    }
    std::vector<std::vector<int64_t>> members((size_t)nb);
    for (int64_t k = 0; k < nb; ++k) members[(size_t)lead[(size_t)k]].push_back(k);
    Grouping g;
    for (int64_t k = 0; k < nb; ++k) {
        if (lead[(size_t)k] != k) continue;
        const auto &m = members[(size_t)k];
        for (size_t i = 0; i < m.size(); ++i) {
            g.order.push_back(m[i]);
            g.npo.push_back(npo[o0 + m[i]]);
            g.group.push_back(i == 0 ? (int)m.size() : 0);
        }
        if (m.size() > 1) g.any = true;
    }
    return g;
}

// Device pointers of one batch's workspace (run_device carves them from one
// allocation in this order; workspace_bytes sizes it).
struct Workspace {
    int64_t *off = nullptr;
    double *tt = nullptr;
    int *bad = nullptr;
    void *yc = nullptr, *wv = nullptr;
    double *yc64 = nullptr, *wv64 = nullptr;
    float2 *ydf = nullptr, *wdf = nullptr;
    double *chi0 = nullptr, *ymax = nullptr;
    int4 *items = nullptr;
    int *counters = nullptr;
    size_t n_counters = 0;
    unsigned char *near = nullptr, *slab = nullptr;
};

Workspace carve_workspace(unsigned char *base, const Plan &plan, int64_t n_obj, int64_t N,
                          int64_t n_freq, int prec)
{
    Workspace w;
    size_t cur = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + cur;
        cur += align16(bytes);
        return p;
    };
    w.off = (int64_t *)take(8 * (size_t)(n_obj + 1));
    w.tt = (double *)take(8 * (size_t)N);
    w.bad = (int *)take(4 * (size_t)n_obj);
    w.yc = take(rsize(prec) * (size_t)N);
    w.wv = take(rsize(prec) * (size_t)N);
    w.yc64 = plan.redo ? (double *)take(8 * (size_t)N) : nullptr;
    w.wv64 = plan.redo ? (double *)take(8 * (size_t)N) : nullptr;
    w.ydf = plan.redo ? (float2 *)take(8 * (size_t)N) : nullptr;
    w.wdf = plan.redo ? (float2 *)take(8 * (size_t)N) : nullptr;
    w.chi0 = (double *)take(8 * (size_t)n_obj);
    w.ymax = (double *)take(8 * (size_t)n_obj);
    w.items = (int4 *)take(sizeof(int4) * plan.items_total);
    w.n_counters = 2 * plan.buckets.size() + 2;
    w.counters = (int *)take(4 * w.n_counters);
    w.near = plan.redo ? (unsigned char *)take((size_t)n_obj * (size_t)n_freq) : nullptr;
    w.slab = base + cur;
    return w;
}

// CSR offsets and the work items of a plan, as the kernels read them
void plan_tables(const Plan &plan, const int64_t *npo, int64_t n_obj, std::vector<int64_t> &off,
                 std::vector<int4> &items)
{
    off.assign((size_t)n_obj + 1, 0);
    for (int64_t o = 0; o < n_obj; ++o) off[o + 1] = off[o] + npo[o];
    items.clear();
    items.reserve(plan.items_total);
    for (const Bucket &b : plan.buckets) items.insert(items.end(), b.items.begin(), b.items.end());
}

// what enqueue_pipeline tells its caller after each kernel it enqueues
enum LaunchKind { LK_PREP = 0, LK_PGRAM = 1, LK_ARGMAX = 2 };
struct LaunchHook {
    virtual void launched(LaunchKind k, const void *args) = 0;
};

// The device pipeline of one batch after its tables are on the device: the
// counters and flags cleared, prep, each length bucket's periodogram (and its
// FP64 recompute), argmax.  fbase (device, or null): object o's grid is
// freq[fbase[o] .. + n_freq); out_best_power (device, or null) receives each
// object's largest power.  prof: record the per-phase timers.
cudaError_t enqueue_pipeline(const Plan &plan, const Workspace &w, const double *t, const double *y,
                             const double *dy, int64_t n_obj, const double *freq, int64_t n_freq,
                             ssp_variant variant, const ssp_params &P, void *out_power,
                             double *out_best, cudaStream_t s, const int64_t *fbase,
                             double *out_best_power, bool prof, LaunchHook *hook)
{
    const int prec = (int)P.precision;
    const int kv = kernel_variant(variant, P);
    const bool per = P.periodic != 0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.counters, 0, 4 * w.n_counters, s))) return e;
    if (w.near && (e = cudaMemsetAsync(w.near, 0, (size_t)n_obj * (size_t)n_freq, s))) return e;
    PrepArgs pa{};
    pa.t = t;
    pa.y = y;
    pa.dy = dy;
    pa.off = w.off;
    pa.tt = w.tt;
    pa.yc = w.yc;
    pa.wv = w.wv;
    pa.yc64 = w.yc64;
    pa.wv64 = w.wv64;
    pa.ydf = w.ydf;
    pa.wdf = w.wdf;
    pa.chi0 = w.chi0;
    pa.ymax = w.ymax;
    pa.bad = w.bad;
    Mark mk;
    bool on = prof && prof_begin(SSP_PHASE_PREP, s, mk);
    if ((e = prep_launch(prec, pa, (int)n_obj, s))) {
        prof_drop(on, mk);
        return e;
    }
    if (hook) hook->launched(LK_PREP, &pa);
    prof_end(on, mk, s);
    size_t item_base = 0, slab_cur = 0, smo_cur = 0, redo_cur = 0;
    for (size_t k = 0; k < plan.buckets.size(); ++k) {
        const Bucket &b = plan.buckets[k];
        PgramArgs ga{};
        ga.off = w.off;
        ga.tt = w.tt;
        ga.yc = w.yc;
        ga.wv = w.wv;
        ga.chi0 = w.chi0;
        ga.ymax = w.ymax;
        ga.yc64 = w.yc64;
        ga.wv64 = w.wv64;
        ga.ydf = w.ydf;
        ga.wdf = w.wdf;
        ga.bad = w.bad;
        ga.freq = freq;
        ga.n_freq = n_freq;
        ga.items = w.items + item_base;
        ga.n_items = (int)b.items.size();
        ga.item_counter = w.counters + 2 * k;
        ga.power = out_power;
        ga.power_f32 = prec == SSP_FP32C;
        for (int i = 0; i < 3; ++i) ga.spans[i] = P.spans[i];
        ga.alpha = P.alpha;
        ga.slab = b.main.gmem ? w.slab + slab_cur : nullptr;
        ga.smo = b.main.smo_out ? w.slab + plan.slab_total + smo_cur : nullptr;
        ga.smo_stride = b.main.smo_stride;
        ga.smo_kmax = smo_rows(b.n_max, b.G);
        ga.smo_nmax = b.n_max;
        smo_cur += b.main.smo_stride * (size_t)b.main.grid;
        ga.redo_slab = b.main.redo_inline ? w.slab + plan.slab_total + plan.smo_total + redo_cur
                                          : nullptr;
        ga.redo_slab_bytes = b.main.redo_slab_bytes;
        redo_cur += b.main.redo_slab_bytes * (size_t)b.main.grid;
        ga.slab_bytes = b.main.slab_bytes;
        ga.cnt_smem = b.main.cnt_smem ? 1 : 0;
        ga.near = w.near;
        ga.near_ss = near_margin("SSP_NEAR_SS", ssp::kNearSS);
        ga.near_ss_abs = near_margin("SSP_NEAR_SS_ABS", ssp::kNearSSAbs);
        ga.near_sp = near_margin("SSP_NEAR_SP", ssp::kNearSP);
        ga.refit_frac = near_margin("SSP_REFIT_FRAC", ssp::kRefitFrac);
        ga.sens_ulps = near_margin("SSP_SENS_ULPS", ssp::kSensUlps);
        ga.sens_tau = near_margin("SSP_SENS_TAU", (float)ssp::kSensTau);
        ga.recompute = 0;
        ga.periodic = P.periodic;
        ga.span = P.span;
        ga.fbase = fbase;
        slab_cur += b.main.gmem ? b.main.slab_bytes * (size_t)b.main.grid : 0;
        const int ph = variant == SSP_SS ? SSP_PHASE_PGRAM_SS : SSP_PHASE_PGRAM_SP;
        on = prof && prof_begin(ph, s, mk);
        if ((e = pgram_launch(prec, kv, b.main.gmem, b.main.lng, per, b.shared, b.main.grid, b.G,
                              b.main.smem, ga, s))) {
            prof_drop(on, mk);
            return e;
        }
        if (hook) hook->launched(LK_PGRAM, &ga);
        prof_end(on, mk, s);
        if (plan.redo && !b.main.redo_inline) {
            // the same items through the FP64 kernel, flagged frequencies only
            ga.yc = w.yc64;
            ga.wv = w.wv64;
            ga.item_counter = w.counters + 2 * k + 1;
            ga.slab = b.redo.gmem ? w.slab + slab_cur : nullptr;
            ga.smo = nullptr;
            ga.redo_slab = nullptr;
            ga.slab_bytes = b.redo.slab_bytes;
            ga.cnt_smem = b.redo.cnt_smem ? 1 : 0;
            ga.recompute = 1;
            slab_cur += b.redo.gmem ? b.redo.slab_bytes * (size_t)b.redo.grid : 0;
            on = prof && prof_begin(SSP_PHASE_REDO, s, mk);
            if ((e = pgram_launch(kPrecRedo, kv, b.redo.gmem, b.redo.lng, per, b.shared, b.redo.grid,
                                  b.G_redo, b.redo.smem, ga, s))) {
                prof_drop(on, mk);
                return e;
            }
            if (hook) hook->launched(LK_PGRAM, &ga);
            prof_end(on, mk, s);
        }
        item_base += b.items.size();
    }
    ArgmaxArgs aa{};
    aa.power = out_power;
    aa.freq = freq;
    aa.fbase = fbase;
    aa.n_freq = n_freq;
    aa.bad = w.bad;
    aa.best_period = out_best;
    aa.best_power = out_best_power;
    on = prof && prof_begin(SSP_PHASE_ARGMAX, s, mk);
    if ((e = argmax_launch(prec, aa, (int)n_obj, s))) {
        prof_drop(on, mk);
        return e;
    }
    if (hook) hook->launched(LK_ARGMAX, &aa);
    prof_end(on, mk, s);
    return cudaSuccess;
}

int run_device(const double *t, const double *y, const double *dy, const int64_t *npo,
               int64_t n_obj, const double *freq, int64_t n_freq, ssp_variant variant,
               const ssp_params &P, void *out_power, double *out_best, cudaStream_t s,
               const int64_t *fbase = nullptr, double *out_best_power = nullptr,
               const int *group = nullptr)
{
    const int prec = (int)P.precision;
    Plan plan;
    int rc = build_plan(npo, n_obj, n_freq, prec, kernel_variant(variant, P), P.periodic != 0,
                        plan, group);
    if (rc) return rc;
    std::vector<int64_t> off;
    std::vector<int4> items;
    plan_tables(plan, npo, n_obj, off, items);
    const int64_t N = off[n_obj];
    const size_t ws = workspace_bytes(plan, n_obj, N, n_freq, prec);
    unsigned char *base = nullptr;
    cudaError_t e = ssp_internal::dev_alloc((void **)&base, ws, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SSP_ERR_NOMEM, "workspace of %zu bytes: %s", ws, cudaGetErrorString(e));
    }
    const Workspace w = carve_workspace(base, plan, n_obj, N, n_freq, prec);
    int status = SSP_OK;
    e = cudaMemcpyAsync(w.off, off.data(), 8 * off.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.items, items.data(), sizeof(int4) * items.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = enqueue_pipeline(plan, w, t, y, dy, n_obj, freq, n_freq, variant, P, out_power, out_best,
                             s, fbase, out_best_power, true, nullptr);
    if (e) status = cuda_fail(e, "enqueue");
    cudaError_t ef = cudaFreeAsync(base, s);
    if (status == SSP_OK && ef != cudaSuccess) status = cuda_fail(ef, "cudaFreeAsync");
    return status;
}


// ---- entry point without device allocation ----
// Scratch of ssp_periodogram_device_noalloc: a fixed array in device memory,
// set aside on every GPU that loads this library until the process exits.
// Host code may not use the name as an address; set-up takes the device
// address with cudaGetSymbolAddress, once per device.
constexpr size_t kNoAllocBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kNoAllocMaxDevices] = {};

int noalloc_scratch(unsigned char **out)
{
    int dev = 0;
    SSP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SSP_ERR_UNSUPPORTED, "device %d", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = (unsigned char *)p;
    }
    *out = g_noalloc_ptr[dev];
    return SSP_OK;
}

// run_device's launch sequence with the workspace carved from the fixed
// array; frames must fit shared memory (no per-CTA global slabs).
int run_device_noalloc(const double *t, const double *y, const double *dy, const int64_t *npo,
                       int64_t n_obj, const double *freq, int64_t n_freq, ssp_variant variant,
                       const ssp_params &P, void *out_power, double *out_best, cudaStream_t s)
{
    const int prec = (int)P.precision;
    Plan plan;
    const int kv = kernel_variant(variant, P);
    const bool per = P.periodic != 0;
    int rc = build_plan(npo, n_obj, n_freq, prec, kv, per, plan, nullptr, false);
    if (rc) return rc;
    for (const Bucket &b : plan.buckets)
        if (b.main.gmem || (plan.redo && b.redo.gmem))
            return fail(SSP_ERR_UNSUPPORTED,
                        "no-allocation entry point: object of %d points needs a frame in global "
                        "memory; at most about 2500 points per object are supported",
                        b.n_max);
    std::vector<int64_t> off((size_t)n_obj + 1, 0);
    for (int64_t o = 0; o < n_obj; ++o) off[o + 1] = off[o] + npo[o];
    const int64_t N = off[n_obj];
    const size_t ws = workspace_bytes(plan, n_obj, N, n_freq, prec);
    if (ws > kNoAllocBytes)
        return fail(SSP_ERR_UNSUPPORTED,
                    "no-allocation entry point: request needs %zu bytes of scratch, the fixed "
                    "array holds %zu",
                    ws, kNoAllocBytes);
    unsigned char *base = nullptr;
    rc = noalloc_scratch(&base);
    if (rc) return rc;
    size_t cur = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + cur;
        cur += align16(bytes);
        return p;
    };
    int64_t *d_off = (int64_t *)take(8 * (size_t)(n_obj + 1));
    double *d_tt = (double *)take(8 * (size_t)N);
    int *d_bad = (int *)take(4 * (size_t)n_obj);
    void *d_yc = take(rsize(prec) * (size_t)N);
    void *d_wv = take(rsize(prec) * (size_t)N);
    double *d_yc64 = plan.redo ? (double *)take(8 * (size_t)N) : nullptr;
    double *d_wv64 = plan.redo ? (double *)take(8 * (size_t)N) : nullptr;
    float2 *d_ydf = plan.redo ? (float2 *)take(8 * (size_t)N) : nullptr;
    float2 *d_wdf = plan.redo ? (float2 *)take(8 * (size_t)N) : nullptr;
    double *d_chi0 = (double *)take(8 * (size_t)n_obj);
    double *d_ymax = (double *)take(8 * (size_t)n_obj);
    int4 *d_items = (int4 *)take(sizeof(int4) * plan.items_total);
    const size_t n_counters = 2 * plan.buckets.size() + 2;
    int *d_counters = (int *)take(4 * n_counters);
    unsigned char *d_near =
        plan.redo ? (unsigned char *)take((size_t)n_obj * (size_t)n_freq) : nullptr;

    std::vector<int4> items;
    items.reserve(plan.items_total);
    for (const Bucket &b : plan.buckets) items.insert(items.end(), b.items.begin(), b.items.end());
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMemcpyAsync(d_off, off.data(), 8 * off.size(), cudaMemcpyHostToDevice, s))) break;
        if ((e = cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(),
                                 cudaMemcpyHostToDevice, s)))
            break;
        // the array keeps the previous call's contents: counters and flags restart at 0
        if ((e = cudaMemsetAsync(d_counters, 0, 4 * n_counters, s))) break;
        if (d_near && (e = cudaMemsetAsync(d_near, 0, (size_t)n_obj * (size_t)n_freq, s))) break;
        PrepArgs pa{};
        pa.t = t;
        pa.y = y;
        pa.dy = dy;
        pa.off = d_off;
        pa.tt = d_tt;
        pa.yc = d_yc;
        pa.wv = d_wv;
        pa.yc64 = d_yc64;
        pa.wv64 = d_wv64;
        pa.ydf = d_ydf;
        pa.wdf = d_wdf;
        pa.chi0 = d_chi0;
        pa.ymax = d_ymax;
        pa.bad = d_bad;
        if ((e = prep_launch(prec, pa, (int)n_obj, s))) break;
        size_t item_base = 0;
        for (size_t k = 0; k < plan.buckets.size(); ++k) {
            const Bucket &b = plan.buckets[k];
            PgramArgs ga{};
            ga.off = d_off;
            ga.tt = d_tt;
            ga.yc = d_yc;
            ga.wv = d_wv;
            ga.chi0 = d_chi0;
            ga.ymax = d_ymax;
            ga.yc64 = d_yc64;
            ga.wv64 = d_wv64;
            ga.ydf = d_ydf;
            ga.wdf = d_wdf;
            ga.bad = d_bad;
            ga.freq = freq;
            ga.n_freq = n_freq;
            ga.items = d_items + item_base;
            ga.n_items = (int)b.items.size();
            ga.item_counter = d_counters + 2 * k;
            ga.power = out_power;
            ga.power_f32 = prec == SSP_FP32C;
            for (int i = 0; i < 3; ++i) ga.spans[i] = P.spans[i];
            ga.alpha = P.alpha;
            ga.near = d_near;
            ga.near_ss = near_margin("SSP_NEAR_SS", ssp::kNearSS);
            ga.near_ss_abs = near_margin("SSP_NEAR_SS_ABS", ssp::kNearSSAbs);
            ga.near_sp = near_margin("SSP_NEAR_SP", ssp::kNearSP);
            ga.refit_frac = near_margin("SSP_REFIT_FRAC", ssp::kRefitFrac);
            ga.sens_ulps = near_margin("SSP_SENS_ULPS", ssp::kSensUlps);
            ga.sens_tau = near_margin("SSP_SENS_TAU", (float)ssp::kSensTau);
            ga.recompute = 0;
            ga.periodic = P.periodic;
            ga.span = P.span;
            if ((e = pgram_launch(prec, kv, false, b.main.lng, per, false, b.main.grid, b.G, b.main.smem, ga, s)))
                break;
            if (plan.redo) {
                ga.yc = d_yc64;
                ga.wv = d_wv64;
                ga.item_counter = d_counters + 2 * k + 1;
                ga.recompute = 1;
                if ((e = pgram_launch(kPrecRedo, kv, false, b.redo.lng, per, false, b.redo.grid, b.G_redo, b.redo.smem,
                                      ga, s)))
                    break;
            }
            item_base += b.items.size();
        }
        if (e) break;
        ArgmaxArgs aa{};
        aa.power = out_power;
        aa.freq = freq;
        aa.n_freq = n_freq;
        aa.bad = d_bad;
        aa.best_period = out_best;
        e = argmax_launch(prec, aa, (int)n_obj, s);
    } while (0);
    if (e) return cuda_fail(e, "enqueue");
    return SSP_OK;
}

std::once_flag g_pool_once;

}  // namespace

// entry points for the other translation units of the library (ssp_internal.h)
namespace ssp_internal {
int fail(int code, const char *msg) { return ::fail(code, "%s", msg); }
std::string last_error() { return g_err; }
void clear_error() { g_err.clear(); }
int check_params(const ssp_params &p) { return ::check_params(&p); }
int check_one_object(const ssp_params &p, const double *t, const double *y, const double *dy,
                     int64_t n)
{
    int rc = ::check_shape(&n, 1, 1, SSP_SS);
    if (rc) return rc;
    if (!t || !y || !dy) return ::fail(SSP_ERR_ARG, "NULL array argument");
    return ::check_values(t, y, dy, n, (int)p.precision);
}
int check_freq(const double *freq_grid, int64_t n_freq)
{
    if (!freq_grid) return ::fail(SSP_ERR_ARG, "NULL frequency grid");
    if (n_freq < 1 || n_freq > (int64_t)INT32_MAX) return ::fail(SSP_ERR_ARG, "n_freq out of range");
    for (int64_t q = 0; q < n_freq; ++q)
        if (!std::isfinite(freq_grid[q]) || !(freq_grid[q] > 0.0))
            return ::fail(SSP_ERR_ARG, "freq_grid[%lld] must be finite and > 0", (long long)q);
    return SSP_OK;
}
int64_t device_bytes(const int64_t *n_per_object, int64_t n_objects, int64_t n_freq,
                     ssp_variant variant, const ssp_params &p)
{
    Plan plan;
    const int rc = build_plan(n_per_object, n_objects, n_freq, (int)p.precision,
                              kernel_variant(variant, p), p.periodic != 0, plan);
    if (rc) return rc;
    int64_t N = 0;
    for (int64_t o = 0; o < n_objects; ++o) N += n_per_object[o];
    return (int64_t)workspace_bytes(plan, n_objects, N, n_freq, (int)p.precision);
}
int run(const double *t, const double *y, const double *dy, const int64_t *n_per_object,
        int64_t n_objects, const double *freq, int64_t n_freq, ssp_variant variant,
        const ssp_params &p, void *out_power, double *out_best, cudaStream_t s)
{
    std::call_once(g_pool_once, keep_pool_memory);
    return ::run_device(t, y, dy, n_per_object, n_objects, freq, n_freq, variant, p, out_power,
                        out_best, s);
}
}  // namespace ssp_internal

namespace {
// ---- launch plans: the device pipeline captured into a CUDA graph ----
struct PlanNode {
    cudaGraphNode_t node;
    LaunchKind kind;
    union {
        PrepArgs prep;
        PgramArgs pgram;
        ArgmaxArgs argmax;
    } args;
};

struct PlanRecorder : LaunchHook {
    cudaStream_t s = nullptr;
    std::vector<PlanNode> nodes;
    cudaError_t err = cudaSuccess;
    void launched(LaunchKind k, const void *a) override
    {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        const cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd);
        if (e != cudaSuccess || nd != 1) {
            if (err == cudaSuccess) err = e != cudaSuccess ? e : cudaErrorStreamCaptureUnsupported;
            return;
        }
        PlanNode pn{};
        pn.node = deps[0];   // the kernel just captured: the capture's only dependency
        pn.kind = k;
        if (k == LK_PREP) pn.args.prep = *(const PrepArgs *)a;
        else if (k == LK_PGRAM) pn.args.pgram = *(const PgramArgs *)a;
        else pn.args.argmax = *(const ArgmaxArgs *)a;
        nodes.push_back(pn);
    }
};

}  // namespace

struct ssp_plan {
    ssp_params P{};
    ssp_variant variant = SSP_SS;
    int64_t n_obj = 0, n_freq = 0;
    unsigned char *base = nullptr;   // workspace (cudaMalloc), held by the plan
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<PlanNode> nodes;
};

namespace {
void plan_free(ssp_plan *pl)
{
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->base) cudaFree(pl->base);
    delete pl;
}
}  // namespace


extern "C" {

void ssp_default_params(ssp_params *p)
{
    if (!p) return;
    p->spans[0] = 0.05;
    p->spans[1] = 0.2;
    p->spans[2] = 0.5;
    p->alpha = 9.0;
    p->periodic = 1;
    p->precision = SSP_FP32C;
    p->hbm_fraction = 0.75;
    p->span = 0.0;
}

const char *ssp_status_string(int status)
{
    switch (status) {
    case SSP_OK: return "ok";
    case SSP_ERR_ARG: return "invalid argument";
    case SSP_ERR_NOMEM: return "device memory budget exceeded";
    case SSP_ERR_CUDA: return "CUDA error";
    case SSP_ERR_TIMEOUT: return "bounded wait expired";
    case SSP_ERR_UNSUPPORTED: return "unsupported request";
    case SSP_ERR_BUSY: return "too many requests in flight";
    case SSP_PENDING: return "pending";
    default: return "unknown status";
    }
}

const char *ssp_last_error(void) { return g_err.c_str(); }

const char *ssp_version(void) { return "ssp 0.1 sm_103a"; }

int ssp_plan_create(const int64_t *n_per_object, int64_t n_objects, int64_t n_freq,
                    ssp_variant variant, const ssp_params *params, ssp_plan **out)
{
    g_err.clear();
    if (!out) return fail(SSP_ERR_ARG, "NULL plan handle pointer");
    *out = nullptr;
    ssp_params P;
    ssp_default_params(&P);
    if (params) P = *params;
    int rc = check_params(&P);
    if (rc) return rc;
    rc = check_shape(n_per_object, n_objects, n_freq, variant);
    if (rc) return rc;
    const int prec = (int)P.precision;
    Plan plan;
    rc = build_plan(n_per_object, n_objects, n_freq, prec, kernel_variant(variant, P),
                    P.periodic != 0, plan);
    if (rc) return rc;
    std::vector<int64_t> off;
    std::vector<int4> items;
    plan_tables(plan, n_per_object, n_objects, off, items);
    const int64_t N = off[n_objects];
    ssp_plan *pl = new ssp_plan;
    pl->P = P;
    pl->variant = variant;
    pl->n_obj = n_objects;
    pl->n_freq = n_freq;
    const size_t ws = workspace_bytes(plan, n_objects, N, n_freq, prec);
    cudaError_t e = cudaMalloc((void **)&pl->base, ws);
    if (e != cudaSuccess) {
        cudaGetLastError();
        pl->base = nullptr;
        plan_free(pl);
        return fail(SSP_ERR_NOMEM, "plan workspace of %zu bytes", ws);
    }
    const Workspace w = carve_workspace(pl->base, plan, n_objects, N, n_freq, prec);
    e = cudaMemcpy(w.off, off.data(), 8 * off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(w.items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    cudaStream_t s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    PlanRecorder rec;
    rec.s = s;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // placeholders for the caller's arrays: every execute sets them
        const cudaError_t ee = enqueue_pipeline(plan, w, nullptr, nullptr, nullptr, n_objects, nullptr,
                                                n_freq, variant, P, nullptr, nullptr, s, nullptr,
                                                nullptr, false, &rec);
        e = cudaStreamEndCapture(s, &pl->graph);
        if (e == cudaSuccess) e = ee;
        if (e == cudaSuccess) e = rec.err;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        plan_free(pl);
        return cuda_fail(e, "plan capture");
    }
    pl->nodes = std::move(rec.nodes);
    *out = pl;
    return SSP_OK;
}

int ssp_plan_execute(ssp_plan *pl, const double *t, const double *y, const double *dy,
                     const double *freq_grid, void *out_power, double *out_best_period,
                     void *stream)
{
    g_err.clear();
    if (!pl) return fail(SSP_ERR_ARG, "NULL plan");
    if (!t || !y || !dy || !freq_grid || !out_power || !out_best_period)
        return fail(SSP_ERR_ARG, "NULL array argument");
    for (PlanNode &pn : pl->nodes) {
        cudaKernelNodeParams kp;
        SSP_CUDA(cudaGraphKernelNodeGetParams(pn.node, &kp));
        PrepArgs pa;
        PgramArgs ga;
        ArgmaxArgs aa;
        void *argp[1];
        if (pn.kind == LK_PREP) {
            pa = pn.args.prep;
            pa.t = t;
            pa.y = y;
            pa.dy = dy;
            argp[0] = &pa;
        } else if (pn.kind == LK_PGRAM) {
            ga = pn.args.pgram;
            ga.freq = freq_grid;
            ga.power = out_power;
            argp[0] = &ga;
        } else {
            aa = pn.args.argmax;
            aa.power = out_power;
            aa.freq = freq_grid;
            aa.best_period = out_best_period;
            argp[0] = &aa;
        }
        kp.kernelParams = argp;
        kp.extra = nullptr;
        SSP_CUDA(cudaGraphExecKernelNodeSetParams(pl->exec, pn.node, &kp));
    }
    SSP_CUDA(cudaGraphLaunch(pl->exec, (cudaStream_t)stream));
    return SSP_OK;
}

int ssp_plan_destroy(ssp_plan *pl)
{
    g_err.clear();
    if (!pl) return fail(SSP_ERR_ARG, "NULL plan");
    plan_free(pl);
    return SSP_OK;
}

int ssp_test_fault(int kind, int count)
{
    g_err.clear();
    if (!ssp_internal::testing())
        return fail(SSP_ERR_UNSUPPORTED, "fault injection needs SSP_TESTING=1 in the environment");
    if (count < 0) return fail(SSP_ERR_ARG, "count must be >= 0");
    if (kind == SSP_FAULT_ALLOC) ssp_internal::g_fault_alloc.store(count);
    else if (kind == SSP_FAULT_STALL) ssp_internal::g_fault_stall.store(count);
    else if (kind == SSP_FAULT_UPLOAD) ssp_internal::g_fault_upload.store(count);
    else return fail(SSP_ERR_ARG, "unknown fault kind %d", kind);
    return SSP_OK;
}

int ssp_fold_fixed(const double *tt, int64_t n, double f, uint64_t *out)
{
    g_err.clear();
    if (n < 0 || (n > 0 && (!tt || !out))) return fail(SSP_ERR_ARG, "bad array arguments");
    if (!std::isfinite(f) || !(f > 0.0)) return fail(SSP_ERR_ARG, "f must be finite and > 0");
    const ssp::FoldFreq F = ssp::fold_freq(f);
    for (int64_t i = 0; i < n; ++i) {
        if (!std::isfinite(tt[i]) || tt[i] < 0.0)
            return fail(SSP_ERR_ARG, "tt[%lld] must be finite and >= 0", (long long)i);
        out[i] = ssp::fold_fixed64_fast(tt[i], F);
    }
    return SSP_OK;
}

void ssp_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
}

int ssp_profile_read(ssp_phase_time out[SSP_N_PHASES], int reset)
{
    g_err.clear();
    if (!out) return fail(SSP_ERR_ARG, "NULL output");
    for (int k = 0; k < SSP_N_PHASES; ++k) out[k] = ssp_phase_time{0, 0.0};
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int status = SSP_OK;
    for (Mark &m : g_marks) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(m.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, m.a, m.b);
        if (e != cudaSuccess) {
            status = cuda_fail(e, "profile event");
            continue;
        }
        out[m.phase].launches += 1;
        out[m.phase].ms += ms;
    }
    if (reset) {
        for (Mark &m : g_marks) {
            cudaEventDestroy(m.a);
            cudaEventDestroy(m.b);
        }
        g_marks.clear();
    }
    return status;
}

int ssp_periodogram_device(const double *t, const double *y, const double *dy,
                           const int64_t *n_per_object, int64_t n_objects,
                           const double *freq_grid, int64_t n_freq, ssp_variant variant,
                           const ssp_params *params, void *out_power, double *out_best_period,
                           void *stream)
{
    g_err.clear();
    ssp_params P;
    ssp_default_params(&P);
    if (params) P = *params;
    int rc = check_params(&P);
    if (rc) return rc;
    rc = check_shape(n_per_object, n_objects, n_freq, variant);
    if (rc) return rc;
    if (!t || !y || !dy || !freq_grid || !out_power || !out_best_period)
        return fail(SSP_ERR_ARG, "NULL array argument");
    std::call_once(g_pool_once, keep_pool_memory);
    return run_device(t, y, dy, n_per_object, n_objects, freq_grid, n_freq, variant, P, out_power,
                      out_best_period, (cudaStream_t)stream);
}

int ssp_periodogram_device_noalloc(const double *t, const double *y, const double *dy,
                                   const int64_t *n_per_object, int64_t n_objects,
                                   const double *freq_grid, int64_t n_freq, ssp_variant variant,
                                   const ssp_params *params, void *out_power,
                                   double *out_best_period, void *stream)
{
    g_err.clear();
    ssp_params P;
    ssp_default_params(&P);
    if (params) P = *params;
    int rc = check_params(&P);
    if (rc) return rc;
    rc = check_shape(n_per_object, n_objects, n_freq, variant);
    if (rc) return rc;
    if (!t || !y || !dy || !freq_grid || !out_power || !out_best_period)
        return fail(SSP_ERR_ARG, "NULL array argument");
    return run_device_noalloc(t, y, dy, n_per_object, n_objects, freq_grid, n_freq, variant, P,
                              out_power, out_best_period, (cudaStream_t)stream);
}

int ssp_periodogram(const double *t, const double *y, const double *dy,
                    const int64_t *n_per_object, int64_t n_objects, const double *freq_grid,
                    int64_t n_freq, ssp_variant variant, const ssp_params *params,
                    void *out_power, double *out_best_period)
{
    g_err.clear();
    ssp_params P;
    ssp_default_params(&P);
    if (params) P = *params;
    int rc = check_params(&P);
    if (rc) return rc;
    rc = check_shape(n_per_object, n_objects, n_freq, variant);
    if (rc) return rc;
    if (!t || !y || !dy || !freq_grid || !out_power || !out_best_period)
        return fail(SSP_ERR_ARG, "NULL array argument");
    int64_t N = 0;
    for (int64_t o = 0; o < n_objects; ++o) N += n_per_object[o];
    rc = check_values(t, y, dy, N, (int)P.precision);
    if (rc) return rc;
    for (int64_t q = 0; q < n_freq; ++q)
        if (!std::isfinite(freq_grid[q]) || !(freq_grid[q] > 0.0))
            return fail(SSP_ERR_ARG, "freq_grid[%lld] must be finite and > 0", (long long)q);
    std::call_once(g_pool_once, keep_pool_memory);

    cudaStream_t s;
    SSP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    const size_t rs = P.precision == SSP_FP64 ? 8 : 4;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaStreamDestroy(s);
        return cuda_fail(cudaGetLastError(), "cudaMemGetInfo");
    }
    const double budget = P.hbm_fraction * (double)free_b;
    // batch objects so that inputs, outputs and working storage fit the budget
    int status = SSP_OK;
    double *d_freq = nullptr;
    cudaError_t e = ssp_internal::dev_alloc((void **)&d_freq, 8 * (size_t)n_freq, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_freq, freq_grid, 8 * (size_t)n_freq, cudaMemcpyHostToDevice, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        status = fail(SSP_ERR_NOMEM, "frequency grid of %lld values", (long long)n_freq);
    } else if (e != cudaSuccess) {
        status = cuda_fail(e, "frequency grid");
    }
    int64_t o0 = 0, p0 = 0;
    while (status == SSP_OK && o0 < n_objects) {
        // grow the batch while its estimate fits
        int64_t o1 = o0, pts = 0;
        double need = 0.0;
        while (o1 < n_objects) {
            const double add = (double)n_per_object[o1] * (24.0 + 8.0 + 2.0 * rs) +
                               (double)n_freq * rs + 64.0;
            if (o1 > o0 && need + add > budget - kSlabReserve) break;
            need += add;
            pts += n_per_object[o1];
            ++o1;
        }
        const int64_t nb = o1 - o0;
        unsigned char *blk = nullptr;
        const size_t in_b = 8 * (size_t)pts, pw_b = rs * (size_t)nb * (size_t)n_freq;
        e = ssp_internal::dev_alloc((void **)&blk, 3 * align16(in_b) + align16(pw_b) + align16(8 * nb), s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            status = fail(SSP_ERR_NOMEM, "batch of %lld objects does not fit", (long long)nb);
            break;
        }
        double *d_t = (double *)blk, *d_y = (double *)(blk + align16(in_b)),
               *d_dy = (double *)(blk + 2 * align16(in_b));
        void *d_pw = blk + 3 * align16(in_b);
        double *d_best = (double *)(blk + 3 * align16(in_b) + align16(pw_b));
        // (shared sorts are built for periodic windows)
        const Grouping gp = P.periodic ? group_by_times(t, n_per_object, o0, o1, p0) : Grouping{};
        if (gp.any) {
            // objects sharing their times run next to each other, leader first
            std::vector<double> st((size_t)pts), sy((size_t)pts), sdy((size_t)pts);
            std::vector<int64_t> off((size_t)nb + 1, p0);
            for (int64_t k = 0; k < nb; ++k) off[k + 1] = off[k] + n_per_object[o0 + k];
            size_t at = 0;
            for (int64_t k : gp.order) {
                const size_t n = (size_t)n_per_object[o0 + k];
                std::memcpy(&st[at], t + off[k], 8 * n);
                std::memcpy(&sy[at], y + off[k], 8 * n);
                std::memcpy(&sdy[at], dy + off[k], 8 * n);
                at += n;
            }
            std::vector<unsigned char> hpw(pw_b);
            std::vector<double> hbest((size_t)nb);
            do {
                if ((e = cudaMemcpyAsync(d_t, st.data(), in_b, cudaMemcpyHostToDevice, s))) break;
                if ((e = cudaMemcpyAsync(d_y, sy.data(), in_b, cudaMemcpyHostToDevice, s))) break;
                if ((e = cudaMemcpyAsync(d_dy, sdy.data(), in_b, cudaMemcpyHostToDevice, s))) break;
                status = run_device(d_t, d_y, d_dy, gp.npo.data(), nb, d_freq, n_freq, variant, P,
                                    d_pw, d_best, s, nullptr, nullptr, gp.group.data());
                if (status) break;
                if ((e = cudaMemcpyAsync(hpw.data(), d_pw, pw_b, cudaMemcpyDeviceToHost, s))) break;
                if ((e = cudaMemcpyAsync(hbest.data(), d_best, 8 * (size_t)nb,
                                         cudaMemcpyDeviceToHost, s)))
                    break;
                if ((e = cudaStreamSynchronize(s))) break;
                const size_t row = rs * (size_t)n_freq;
                for (int64_t k = 0; k < nb; ++k) {
                    const int64_t o = o0 + gp.order[(size_t)k];
                    std::memcpy((unsigned char *)out_power + row * (size_t)o,
                                hpw.data() + row * (size_t)k, row);
                    out_best_period[o] = hbest[(size_t)k];
                }
            } while (0);
            if (e && status == SSP_OK) status = cuda_fail(e, "batch with shared times");
            cudaFreeAsync(blk, s);
            o0 = o1;
            p0 += pts;
            continue;
        }
        do {
            if ((e = cudaMemcpyAsync(d_t, t + p0, in_b, cudaMemcpyHostToDevice, s))) break;
            if ((e = cudaMemcpyAsync(d_y, y + p0, in_b, cudaMemcpyHostToDevice, s))) break;
            if ((e = cudaMemcpyAsync(d_dy, dy + p0, in_b, cudaMemcpyHostToDevice, s))) break;
        } while (0);
        if (e) {
            status = cuda_fail(e, "input copy");
        } else {
            status = run_device(d_t, d_y, d_dy, n_per_object + o0, nb, d_freq, n_freq, variant, P,
                                d_pw, d_best, s);
            if (status == SSP_OK) {
                e = cudaMemcpyAsync((unsigned char *)out_power + rs * (size_t)o0 * (size_t)n_freq,
                                    d_pw, pw_b, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(out_best_period + o0, d_best, 8 * (size_t)nb,
                                        cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) status = cuda_fail(e, "output copy");
            }
        }
        cudaFreeAsync(blk, s);
        o0 = o1;
        p0 += pts;
    }
    if (d_freq) cudaFreeAsync(d_freq, s);
    e = cudaStreamSynchronize(s);
    if (status == SSP_OK && e != cudaSuccess) status = cuda_fail(e, "synchronize");
    cudaStreamDestroy(s);
    return status;
}

// ---------------------------------------------------------------------------
// autotuning of the threads per CTA, per length range
// ---------------------------------------------------------------------------
int ssp_autotune(const double *t, const double *y, const double *dy, const int64_t *n_per_object,
                 int64_t n_objects, const double *freq_grid, int64_t n_freq, ssp_variant variant,
                 const ssp_params *params, double budget_ptf, int32_t *out_group_sizes)
{
    g_err.clear();
    ssp_params P;
    ssp_default_params(&P);
    if (params) P = *params;
    int rc = check_params(&P);
    if (rc) return rc;
    rc = check_shape(n_per_object, n_objects, n_freq, variant);
    if (rc) return rc;
    if (!t || !y || !dy || !freq_grid) return fail(SSP_ERR_ARG, "NULL array argument");
    if (!(budget_ptf > 0.0)) budget_ptf = 2.0e9;
    std::vector<int64_t> off((size_t)n_objects + 1, 0);
    for (int64_t o = 0; o < n_objects; ++o) off[o + 1] = off[o] + n_per_object[o];
    rc = check_values(t, y, dy, off[n_objects], (int)P.precision);
    if (rc) return rc;
    for (int64_t q = 0; q < n_freq; ++q)
        if (!std::isfinite(freq_grid[q]) || !(freq_grid[q] > 0.0))
            return fail(SSP_ERR_ARG, "freq_grid[%lld] must be finite and > 0", (long long)q);
    std::call_once(g_pool_once, keep_pool_memory);
    const int pi = P.precision == SSP_FP64 ? 0 : 1, vi = kernel_variant(variant, P);
    const size_t rs = rsize((int)P.precision);
    cudaStream_t s;
    SSP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int status = SSP_OK;
    for (int r = 0; r < kRanges && status == SSP_OK; ++r) {
        std::vector<int64_t> objs;
        for (int64_t o = 0; o < n_objects; ++o)
            if (range_of((int)n_per_object[o]) == r) objs.push_back(o);
        if (objs.empty()) continue;
        // the range's objects (in order, up to the budget at 64 frequencies
        // each) on an evenly spaced sample of the grid: enough (object,
        // frequency) pairs to fill the GPU, about budget_ptf of work
        std::vector<int64_t> npo;
        int64_t pts = 0;
        int n_max = 0;
        for (int64_t o : objs) {
            if (!npo.empty() && (double)(pts + n_per_object[o]) * 64.0 > budget_ptf) break;
            npo.push_back(n_per_object[o]);
            pts += n_per_object[o];
            n_max = std::max(n_max, (int)n_per_object[o]);
        }
        const int64_t nob = (int64_t)npo.size();
        int64_t F = (int64_t)(budget_ptf / (double)pts);
        F = std::max<int64_t>(F, (4096 + nob - 1) / nob);
        F = std::max<int64_t>(64, std::min<int64_t>(F, n_freq));
        std::vector<double> ht((size_t)pts), hy((size_t)pts), hdy((size_t)pts), hf((size_t)F);
        int64_t at = 0;
        for (size_t k = 0; k < npo.size(); ++k) {
            const int64_t o = objs[k], n = n_per_object[o];
            std::memcpy(&ht[(size_t)at], t + off[o], 8 * (size_t)n);
            std::memcpy(&hy[(size_t)at], y + off[o], 8 * (size_t)n);
            std::memcpy(&hdy[(size_t)at], dy + off[o], 8 * (size_t)n);
            at += n;
        }
        for (int64_t q = 0; q < F; ++q) hf[(size_t)q] = freq_grid[(q * n_freq) / F];
        unsigned char *blk = nullptr;
        const size_t a = align16(8 * (size_t)pts), bf = align16(8 * (size_t)F),
                     bp = align16(rs * (size_t)nob * (size_t)F), bb = align16(8 * (size_t)nob);
        cudaError_t e = ssp_internal::dev_alloc((void **)&blk, 3 * a + bf + bp + bb, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            status = fail(SSP_ERR_NOMEM, "autotune sample does not fit");
            break;
        }
        double *dt = (double *)blk, *dyv = (double *)(blk + a), *ddy = (double *)(blk + 2 * a);
        double *df = (double *)(blk + 3 * a);
        void *dpw = blk + 3 * a + bf;
        double *dbest = (double *)(blk + 3 * a + bf + bp);
        cudaMemcpyAsync(dt, ht.data(), 8 * (size_t)pts, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dyv, hy.data(), 8 * (size_t)pts, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(ddy, hdy.data(), 8 * (size_t)pts, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(df, hf.data(), 8 * (size_t)F, cudaMemcpyHostToDevice, s);
        // candidates around the rule: half, same, double, within 32..512 and
        // with at least two centres per thread
        const int g0 = group_size_rule(n_max, vi, (int)P.precision);
        std::vector<int> cand;
        for (int g : {g0 / 2, g0, g0 * 2})
            if (g >= 32 && g <= 512 && (g == g0 || 2 * g <= std::max(64, n_max))) cand.push_back(g);
        const int prev = g_tuned[pi][vi][r].load();
        int best_g = g0;
        float best_ms = 0.f;
        for (int g : cand) {
            g_tuned[pi][vi][r].store(g);
            float ms = 0.f;
            for (int rep = 0; rep < 3 && status == SSP_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, s);
                rc = run_device(dt, dyv, ddy, npo.data(), nob, df, F, variant, P, dpw, dbest, s);
                if (rc) status = rc;
            }
            if (status != SSP_OK) break;
            cudaEventRecord(e1, s);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                status = cuda_fail(e, "autotune timing");
                break;
            }
            cudaEventElapsedTime(&ms, e0, e1);
            if (best_ms == 0.f || ms < best_ms) {
                best_ms = ms;
                best_g = g;
            }
        }
        g_tuned[pi][vi][r].store(status == SSP_OK ? best_g : prev);
        cudaFreeAsync(blk, s);
    }
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (out_group_sizes)
        for (int r = 0; r < kRanges; ++r) {
            const int tg = g_tuned[pi][vi][r].load();
            out_group_sizes[r] = tg ? tg : group_size_rule(kRangeMax[r], vi, (int)P.precision);
        }
    return status;
}

void ssp_autotune_clear(void)
{
    for (auto &a : g_tuned)
        for (auto &b : a)
            for (auto &c : b) c.store(0);
}

// ---------------------------------------------------------------------------
// search-and-refine
// ---------------------------------------------------------------------------
int ssp_search_refine(const double *t, const double *y, const double *dy,
                      const int64_t *n_per_object, int64_t n_objects, const double *coarse_grid,
                      int64_t n_coarse, ssp_variant coarse_variant, ssp_variant fine_variant,
                      int n_peaks, int n_fine, const ssp_params *params, double *out_best_period,
                      double *out_best_power)
{
    g_err.clear();
    ssp_params P;
    ssp_default_params(&P);
    if (params) P = *params;
    int rc = check_params(&P);
    if (rc) return rc;
    if (P.span > 0.0) return fail(SSP_ERR_ARG, "search-and-refine needs the variable span");
    rc = check_shape(n_per_object, n_objects, n_coarse, coarse_variant);
    if (rc) return rc;
    rc = check_shape(n_per_object, n_objects, 1, fine_variant);
    if (rc) return rc;
    if (!t || !y || !dy || !coarse_grid || !out_best_period || !out_best_power)
        return fail(SSP_ERR_ARG, "NULL array argument");
    if (n_coarse < 2) return fail(SSP_ERR_ARG, "the coarse grid needs at least 2 frequencies");
    if (n_peaks < 1 || n_peaks > 64) return fail(SSP_ERR_ARG, "n_peaks must be in 1..64");
    if (n_fine < 1 || (int64_t)n_peaks * n_fine > (int64_t)1 << 22)
        return fail(SSP_ERR_ARG, "n_fine must be >= 1 with n_peaks * n_fine <= 2^22");
    for (int64_t q = 0; q < n_coarse; ++q) {
        if (!std::isfinite(coarse_grid[q]) || !(coarse_grid[q] > 0.0))
            return fail(SSP_ERR_ARG, "coarse_grid[%lld] must be finite and > 0", (long long)q);
        if (q > 0 && !(coarse_grid[q] > coarse_grid[q - 1]))
            return fail(SSP_ERR_ARG, "the coarse grid must increase strictly");
    }
    int64_t N = 0;
    for (int64_t o = 0; o < n_objects; ++o) N += n_per_object[o];
    rc = check_values(t, y, dy, N, (int)P.precision);
    if (rc) return rc;
    std::call_once(g_pool_once, keep_pool_memory);
    const int prec = (int)P.precision;
    const size_t rs = rsize(prec);
    const int64_t nf = (int64_t)n_peaks * n_fine;
    cudaStream_t s;
    SSP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double budget = P.hbm_fraction * (double)free_b - kSlabReserve;
    int status = SSP_OK;
    double *d_coarse = nullptr;
    cudaError_t e = ssp_internal::dev_alloc((void **)&d_coarse, 8 * (size_t)n_coarse, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_coarse, coarse_grid, 8 * (size_t)n_coarse, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) status = cuda_fail(e, "coarse grid");
    int64_t o0 = 0, p0 = 0;
    while (status == SSP_OK && o0 < n_objects) {
        // objects per batch: inputs, coarse and fine powers and grids in the budget
        int64_t o1 = o0, pts = 0;
        double need = 0.0;
        while (o1 < n_objects) {
            const double add = (double)n_per_object[o1] * (24.0 + 8.0 + 2.0 * (double)rs) +
                               (double)(n_coarse + nf) * (double)rs + 8.0 * (double)nf + 96.0;
            if (o1 > o0 && need + add > budget) break;
            need += add;
            pts += n_per_object[o1];
            ++o1;
        }
        const int64_t nb = o1 - o0;
        const size_t in_b = align16(8 * (size_t)pts), cp_b = align16(rs * (size_t)(nb * n_coarse));
        const size_t fp_b = align16(rs * (size_t)(nb * nf)), fg_b = align16(8 * (size_t)(nb * nf));
        const size_t ob_b = align16(8 * (size_t)nb);
        unsigned char *blk = nullptr;
        e = ssp_internal::dev_alloc((void **)&blk, 3 * in_b + cp_b + fp_b + fg_b + 4 * ob_b, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            status = fail(SSP_ERR_NOMEM, "batch of %lld objects does not fit", (long long)nb);
            break;
        }
        double *d_t = (double *)blk, *d_y = (double *)(blk + in_b), *d_dy = (double *)(blk + 2 * in_b);
        void *d_cp = blk + 3 * in_b, *d_fp = blk + 3 * in_b + cp_b;
        double *d_fg = (double *)(blk + 3 * in_b + cp_b + fp_b);
        unsigned char *tail = blk + 3 * in_b + cp_b + fp_b + fg_b;
        double *d_cbest = (double *)tail, *d_fbest = (double *)(tail + ob_b);
        double *d_fpow = (double *)(tail + 2 * ob_b);
        int64_t *d_fbase = (int64_t *)(tail + 3 * ob_b);
        std::vector<int64_t> fbase((size_t)nb);
        for (int64_t i = 0; i < nb; ++i) fbase[(size_t)i] = i * nf;
        do {
            if ((e = cudaMemcpyAsync(d_t, t + p0, 8 * (size_t)pts, cudaMemcpyHostToDevice, s))) break;
            if ((e = cudaMemcpyAsync(d_y, y + p0, 8 * (size_t)pts, cudaMemcpyHostToDevice, s))) break;
            if ((e = cudaMemcpyAsync(d_dy, dy + p0, 8 * (size_t)pts, cudaMemcpyHostToDevice, s))) break;
            if ((e = cudaMemcpyAsync(d_fbase, fbase.data(), 8 * (size_t)nb, cudaMemcpyHostToDevice, s)))
                break;
            // coarse search
            status = run_device(d_t, d_y, d_dy, n_per_object + o0, nb, d_coarse, n_coarse,
                                coarse_variant, P, d_cp, d_cbest, s);
            if (status) break;
            PeaksArgs pa{};
            pa.power = d_cp;
            pa.coarse = d_coarse;
            pa.n_coarse = n_coarse;
            pa.k = n_peaks;
            pa.n_fine = n_fine;
            pa.fine = d_fg;
            if ((e = peaks_launch(prec, pa, (int)nb, s))) break;
            // refine on each object's own grids
            status = run_device(d_t, d_y, d_dy, n_per_object + o0, nb, d_fg, nf, fine_variant, P,
                                d_fp, d_fbest, s, d_fbase, d_fpow);
            if (status) break;
            if ((e = cudaMemcpyAsync(out_best_period + o0, d_fbest, 8 * (size_t)nb,
                                     cudaMemcpyDeviceToHost, s)))
                break;
            if ((e = cudaMemcpyAsync(out_best_power + o0, d_fpow, 8 * (size_t)nb,
                                     cudaMemcpyDeviceToHost, s)))
                break;
        } while (0);
        if (e != cudaSuccess && status == SSP_OK) status = cuda_fail(e, "search-and-refine");
        cudaFreeAsync(blk, s);
        if (status == SSP_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess)
            status = cuda_fail(e, "search-and-refine");
        o0 = o1;
        p0 += pts;
    }
    if (d_coarse) cudaFreeAsync(d_coarse, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return status;
}

}  // extern "C"
