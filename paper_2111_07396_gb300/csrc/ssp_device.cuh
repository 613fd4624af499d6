// ssp_device.cuh -- device code of the Super Smoother periodogram (arXiv
// 2111.07396) for sm_103a.
//
// One CTA processes one (object, trial frequency) at a time, looping over
// work items (object, frequency range) taken from a global counter.  For
// each frequency everything stays in the CTA's frame (shared memory, or a
// per-CTA global slab for objects too large for shared memory):
//
//   fold    phase = frac(tt*f) (Alg. 1, computePhasedTime), bit-identical to
//           the rounded binary64 product: the FP64 path multiplies in FP64,
//           the FP32C path emulates the same IEEE multiply with integers
//           (ssp_fold.h) and keeps the phase as a 64-bit fixed-point number.
//   sort    stable argsort by phase (Alg. 1, argsort + mapArgsort): one
//           counting pass into ~n/2 buckets by the top phase bits, then each
//           element ranks itself inside its bucket; CTA-wide bitonic sort if
//           a bucket is crowded.
//   smooth  running lines (the `smoothkernel` of Listing 1; Friedman 1984):
//           the n centres are split into one contiguous chunk per thread;
//           each thread builds its first window from per-chunk aggregates
//           plus the ragged ends, then slides the window through its chunk
//           with add/remove updates of sums taken about a local origin.
//           SS = Listing 1 as four sweeps (three spans with CV, smoothed
//           residuals with span choice and bass, smoothed spans with the
//           interpolation, final tweeter pass with chi2); SP = one sweep with
//           three windows and the generalized-validation span choice.
//   reduce  chi2 per frequency, power = 1 - chi2/chi0 (computePgram).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ssp_fold.h"

namespace ssp {

// kernel variants: SS (Listing 1), SP (Sec. 3), and Listing 1's fixed-span
// single smooth, which is the same computation for both
enum { VAR_SS = 0, VAR_SP = 1, VAR_FIXED = 2, VAR_SPG = 3 };
// SPG: relative gap between two spans' scores below which FP32C sends the
// frequency to the FP64 recompute (the scores' FP32 error is ~1e-6)
constexpr double kNearSPG = 1e-5;
constexpr int kMaxThreads = 512;
constexpr int kBucketRankMax = 64;   // larger buckets switch to the bitonic sort

// FP32C decisions closer than these margins to their thresholds are re-taken
// in FP64: the frequency is flagged and recomputed by the FP64 kernel.
//  - SS: tweeter vs midrange smoothed residuals closer than
//    kNearSS * min(1, 256/n) * min(1, 512/n) relative (the FP32 error of a
//    smoothed residual, and the effect of one flipped choice on the power,
//    both fall as the windows grow with n), up to kNearSSMaxN points;
//  - a cross-validated residual whose 1 - leverage is below kNearLev, and a
//    window spread within kNearSlope of vsmlsq.
// SP choices are settled in place instead: where the tweeter and midrange
// generalized-validation residuals are closer than kNearSP * eps_fp32 times
// the magnitude scale (the larger of the point's and the object's largest
// centred magnitude), and the other choice could move the power by more than
// kSensTau, the warp refits the three span windows beyond FP32 precision
// (double-float sums of exact products) from the exact phases and the inputs
// split into double-float pairs, and takes the choice from those in double-float
// arithmetic.  Over C1-C4-shaped catalogs (3.5e5 settles) every choice the
// settle reversed had its residuals within 16 of these units of each other,
// and the settles spread evenly over |g0 - g1| (half of them in the top
// octave of the margin): kNearSP keeps twice the largest distance seen.
constexpr float kNearSS = 1e-6f;
constexpr float kNearSSAbs = 8.f;
// Above this many points the SS tweeter/midrange margin flags nothing: one
// choice decided either way moves the power by little there.  Measured by
// recomputing every flagged frequency in binary64 (3.6e4 of them, catalogs of
// 256-4,096 points): the largest change was 5e-4 at 256-511 points, 1.3e-4
// at 512-1,023, 3.5e-5 at 1,024-2,047 and 1.3e-5 at 2,048-4,095, against
// the 2e-4 tolerance; on the 3,000-point seasonal object the recomputes took
// 18% of the SS time and moved no power by more than 7e-6.
constexpr int kNearSSMaxN = 2048;
constexpr float kNearSP = 32.f;
constexpr float kNearLev = 1e-4f;
constexpr float kNearSlope = 1e-4f;
constexpr float kRefitFrac = 1.f / 128.f;  // history guard of the sliding sums
// windows of at most this many points are initialised by direct summation
constexpr int kDirectInit = 32;
// SS launches whose objects exceed this many points use the kernel that
// initialises windows out of line (FP32C)
constexpr int kLongN = 1536;
// SP: a point whose fit could move the power by more than kSensTau through
// the FP32 error of its residuals (bass enhancement divides by the smallest;
// each residual is taken to err by its slope times the rounding of X plus
// kSensUlps ulps of its magnitude scale) is settled by the warp's refit as
// well
constexpr double kSensTau = 1e-6;
constexpr float kSensUlps = 2.f;

struct PgramArgs {
    const int64_t *off;     // [n_obj + 1] CSR offsets
    const double *tt;       // [N] t - min t (binary64, both paths)
    const void *yc;         // [N] centred magnitudes, R
    const void *wv;         // [N] weights dy^-2, R
    const double *chi0;     // [n_obj]
    const double *ymax;     // [n_obj] largest centred magnitude
    const double *yc64, *wv64;  // [N] binary64 inputs (FP32C: exact SP refits)
    const float2 *ydf, *wdf;    // [N] the same as double-float pairs (hi, lo) (FP32C)
    const int *bad;         // [n_obj] nonzero: invalid input, NaN output
    const double *freq;     // [n_freq]
    int64_t n_freq;
    const int4 *items;      // (object, q0, q1, -)
    int n_items;
    int *item_counter;      // work-queue head, zero before launch
    void *power;            // [n_obj][n_freq] R
    double spans[3];
    double alpha;
    unsigned char *slab;    // per-CTA frames when they do not fit shared memory
    size_t slab_bytes;
    int cnt_smem;           // slab frames: sort bucket counts in shared memory
    unsigned char *near;    // [n_obj][n_freq] FP32C: decision near a threshold
    int recompute;          // FP64 kernel: only flagged (o, q), float power out
    int periodic;           // 1: periodic windows; 0: windows clamped inside the data
    double span;            // > 0: Listing 1's fixed-span single smooth
    const int64_t *fbase;   // null: one grid; else object o's grid starts at freq[fbase[o]]
    int power_f32;          // power array holds float
    float near_ss;          // SS margin for n <= 256 (scaled down above)
    float near_ss_abs;      // SS margin in units of eps_fp32 * the object's largest magnitude
    float near_sp;          // SP margin in units of eps_fp32 * magnitude scale
    float refit_frac;       // refit windows whose spread fell below this part of hiB
    float sens_ulps;        // SP sensitivity: rounding of a residual, in ulps of its scale
    double sens_tau;        // SP sensitivity: power budget per point
    // SS: the three smooths of pass A, read back only at their own centre in
    // pass C, live in a per-CTA global slab instead of the frame (null: in
    // the frame).  Layout per CTA: [column][k][thread] for the k-th centre of
    // a thread's chunk while k < smo_kmax (a warp's accesses are adjacent),
    // then [column][point] for the centres of longer chunks.
    void *smo;
    size_t smo_stride;      // bytes per CTA
    int smo_kmax, smo_nmax;
    // FP32C SS, long objects: a flagged frequency is recomputed in binary64
    // by the same CTA right away (null: flags for the recompute launch).
    // Per-CTA binary64 frames in global memory of redo_slab_bytes each.
    unsigned char *redo_slab;
    size_t redo_slab_bytes;
};

// rows of the smooth slab's per-thread part: twice the mean chunk length
// plus slack (chunks grow past the mean only over runs of tied phases)
__host__ __device__ inline int smo_rows(int n, int G) { return 2 * ((n + G - 1) / G) + 4; }
__host__ __device__ inline size_t smo_bytes(int n, int G, size_t rsize)
{
    return 3 * ((size_t)smo_rows(n, G) * (size_t)G + (size_t)n) * rsize;
}

// ---------------------------------------------------------------------------
// frame layout (per CTA, sized for the largest n of a launch)
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }
// counting-sort buckets: a power of two >= n/2 (about two keys per bucket)
__host__ __device__ inline int bucket_count(int n)
{
    int nb = 32;
    while (2 * nb < n) nb <<= 1;
    return nb;
}
__host__ __device__ inline int pow2_at_least(int n)
{
    int p = 32;
    while (p < n) p <<= 1;
    return p;
}

// (phase, weight) of one point, read and written together
template <typename R> struct Vec2;
template <> struct Vec2<float> { typedef float2 T; };
template <> struct Vec2<double> { typedef double2 T; };
template <typename R>
__device__ inline typename Vec2<R>::T vec2(R a, R b)
{
    typename Vec2<R>::T v;
    v.x = a;
    v.y = b;
    return v;
}

template <typename R>
struct Frame {
    typename Vec2<R>::T *XW;  // sorted phase (x) and weight (y)
    R *Y;                     // centred magnitude
    R *C[7];                // smoother columns
    uint32_t *tie;          // bit j: sorted points j and j+1 have the same
                            // folded phase (exact fold output, not rounded X)
    uint64_t *key;          // phase as 64-bit fixed point: by original index
                            // after the fold, in sorted order after the sort
    uint64_t *sk;           // sort scratch: keys by bucket position
    uint16_t *slot, *tmp, *perm;  // sort scratch; perm: original index of
                                  // each sorted point (n <= 65535)
    uint32_t *cnt;          // bucket counts / starts
    double *ph;             // FP64 phase by original index
    int per;                // windows wrap (periodic) or are clamped inside [0, n-1]
};

// first slot of the 2h+1-point window of centre j: j - h with periodic
// wrap, else the window slid to lie inside the data (Listing 1 iper = 1)
__device__ inline int win_lo_mode(int per, int j, int h, int n)
{
    if (per) return j - h;
    const int lo = j - h;
    return lo < 0 ? 0 : (lo > n - 1 - 2 * h ? n - 1 - 2 * h : lo);
}
template <typename R>
__device__ inline int win_lo(const Frame<R> &fr, int j, int h, int n)
{
    return win_lo_mode(fr.per, j, h, n);
}

__host__ __device__ inline size_t tie_words(int n) { return ((size_t)n + 31) / 32; }

// Frame layout.  XW (phase and weight, interleaved) and Y come first; while
// the phases are sorted that region holds the scatter scratch instead (keys
// by bucket position, slots and scattered indices).  The sort region follows: the 64-bit keys (the fold
// output by original index, then the keys in sorted order), perm, the bucket
// counts and, for FP64, the phases by original index.  SS columns C0..C6 also
// follow XW, Y and overlay the sort region, which is dead once the gather
// has run; SP keeps the sorted keys for its exact refits.  The tie bitmask
// follows whichever region ends later, because the gather writes it while it
// still reads the sort's output.
template <typename R>
__host__ __device__ inline size_t xwy_bytes(int n)
{
    const size_t col = align16(sizeof(R) * (size_t)n);
    const size_t scat = align16(4 * (size_t)n) * 2 + align16(2 * (size_t)n) * 2;
    return 3 * col > scat ? 3 * col : scat;
}

template <typename R>
__host__ __device__ inline size_t sort_end(int n)
{
    size_t s = xwy_bytes<R>(n) + align16(4 * (size_t)n) * 2 +
               align16(2 * (size_t)pow2_at_least(n)) + align16(4 * (size_t)bucket_count(n));
    if (sizeof(R) == 8) s += align16(8 * (size_t)n);
    return s;
}

template <typename R>
__host__ __device__ inline size_t tie_offset(int n, int ncols)
{
    const size_t cols = xwy_bytes<R>(n) + align16(sizeof(R) * (size_t)n) * (size_t)(ncols - 3);
    const size_t s = sort_end<R>(n);
    return cols > s ? cols : s;
}

// columns a variant keeps: SS uses XW (two columns), Y and C0..C6 (C1, C3, C5,
// C6 only when the smooths C0, C2, C4 live in the global slab); SP only XW, Y
__host__ __device__ inline int frame_cols(int variant, bool smo_out = false)
{
    return variant == VAR_SS ? (smo_out ? 7 : 10) : 3;
}

// keep_perm: objects with identical times share one sort (their frame keeps
// perm for every member's gather); an SS frame then holds perm past the tie
// bitmask, clear of the smoother columns that overlay the sort region -- or,
// when the smooths live in the global slab (smo_out), in that slab too, so
// that two CTAs still share an SM
template <typename R>
__host__ __device__ inline size_t frame_bytes(int n, int variant, bool keep_perm = false,
                                              bool smo_out = false)
{
    size_t b = tie_offset<R>(n, frame_cols(variant, smo_out)) + align16(4 * tie_words(n));
    if (keep_perm && variant == VAR_SS && !smo_out) b += align16(2 * (size_t)pow2_at_least(n));
    return b;
}
// bytes of the kept perm in the smooth slab (shared sorts, smo_out)
__host__ __device__ inline size_t kept_perm_bytes(int n) { return align16(2 * (size_t)pow2_at_least(n)); }

template <typename R>
__device__ inline Frame<R> carve_frame(unsigned char *base, int n, int variant,
                                       bool keep_perm = false, bool smo_out = false,
                                       uint16_t *perm_slab = nullptr)
{
    Frame<R> f;
    const size_t col = align16(sizeof(R) * (size_t)n), xwy = xwy_bytes<R>(n);
    const size_t a4 = align16(4 * (size_t)n), a2 = align16(2 * (size_t)n);
    const size_t ap = align16(2 * (size_t)pow2_at_least(n));
    f.XW = (typename Vec2<R>::T *)base;   // 2 n sizeof(R) bytes <= 2 col
    f.Y = (R *)(base + 2 * col);
    f.sk = (uint64_t *)base;   // 8n bytes <= 2 a4
    f.slot = (uint16_t *)(base + 2 * a4);
    f.tmp = (uint16_t *)(base + 2 * a4 + a2);
    if (smo_out && variant == VAR_SS) {
        // C1, C3, C5, C6 in the frame; the smooths C0, C2, C4 in the slab
        const int slot[7] = {-1, 0, -1, 1, -1, 2, 3};
        for (int k = 0; k < 7; ++k) f.C[k] = slot[k] < 0 ? nullptr : (R *)(base + xwy + slot[k] * col);
    } else {
        for (int k = 0; k < 7; ++k) f.C[k] = (R *)(base + xwy + k * col);
    }
    unsigned char *s = base + xwy;
    f.key = (uint64_t *)s;     // 8n bytes <= 2 a4
    f.perm = (uint16_t *)(s + 2 * a4);
    f.cnt = (uint32_t *)(s + 2 * a4 + ap);
    f.ph = (double *)(s + 2 * a4 + ap + align16(4 * (size_t)bucket_count(n)));
    f.tie = (uint32_t *)(base + tie_offset<R>(n, frame_cols(variant, smo_out)));
    if (keep_perm && variant == VAR_SS)
        f.perm = smo_out ? perm_slab
                         : (uint16_t *)(base + tie_offset<R>(n, frame_cols(variant, smo_out)) +
                                        align16(4 * tie_words(n)));
    f.per = 1;
    return f;
}

// ---------------------------------------------------------------------------
// extended-precision accumulator for the window prefixes: an unevaluated sum
// hi + lo of two numbers of the working type (double-float, ~48 bits, on the
// FP32 path; double-double, ~104 bits, on the FP64 path), added with Knuth's
// two-sum and multiplied with an FMA-exact product (Dekker's error-free
// transformations)
// ---------------------------------------------------------------------------
template <typename T>
struct xacc {
    T hi, lo;
};
typedef xacc<float> df;
typedef xacc<double> dd;
__device__ inline float fma_x(float a, float b, float c) { return fmaf(a, b, c); }
__device__ inline double fma_x(double a, double b, double c) { return fma(a, b, c); }
template <typename T>
__device__ inline xacc<T> x_two_sum(T a, T b)
{
    const T s = a + b;
    const T bb = s - a;
    return xacc<T>{s, (a - (s - bb)) + (b - bb)};
}
template <typename T>
__device__ inline xacc<T> x_fast(T a, T b)
{
    const T s = a + b;
    return xacc<T>{s, b - (s - a)};
}
template <typename T>
__device__ inline xacc<T> acc_add(xacc<T> x, xacc<T> y)
{
    xacc<T> s = x_two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return x_fast(s.hi, s.lo);
}
template <typename T>
__device__ inline xacc<T> acc_neg(xacc<T> x) { return xacc<T>{-x.hi, -x.lo}; }
template <typename T>
__device__ inline xacc<T> acc_mul(xacc<T> x, T b)
{
    const T p = x.hi * b;
    const T e = fma_x(x.hi, b, -p);
    return x_fast(p, fma_x(x.lo, b, e));
}
template <typename T>
__device__ inline T acc_to(xacc<T> x) { return x.hi + x.lo; }
template <typename T>
__device__ inline xacc<T> acc_shfl_up(xacc<T> x, int k)
{
    return xacc<T>{__shfl_up_sync(0xffffffffu, x.hi, k), __shfl_up_sync(0xffffffffu, x.lo, k)};
}
template <typename T>
__device__ inline xacc<T> acc_shfl_xor(xacc<T> x, int k)
{
    return xacc<T>{__shfl_xor_sync(0xffffffffu, x.hi, k), __shfl_xor_sync(0xffffffffu, x.lo, k)};
}
template <typename T>
__device__ inline xacc<T> acc_shfl_idx(xacc<T> x, int k)
{
    return xacc<T>{__shfl_sync(0xffffffffu, x.hi, k), __shfl_sync(0xffffffffu, x.lo, k)};
}

// plain accumulator (the FP64 recompute of flagged FP32C frequencies, whose
// results only have to meet the FP32C tolerance)
__device__ inline double acc_add(double x, double y) { return x + y; }
__device__ inline double acc_neg(double x) { return -x; }
__device__ inline double acc_mul(double x, double b) { return x * b; }
__device__ inline double acc_to(double x) { return x; }
__device__ inline double acc_shfl_up(double x, int k) { return __shfl_up_sync(0xffffffffu, x, k); }
__device__ inline double acc_shfl_xor(double x, int k) { return __shfl_xor_sync(0xffffffffu, x, k); }
__device__ inline double acc_shfl_idx(double x, int k) { return __shfl_sync(0xffffffffu, x, k); }

// smallest window B / total weight whose prefix-based sums keep the accuracy
// stated in win_init
template <typename A> __device__ constexpr double acc_keep();
template <> __device__ constexpr double acc_keep<xacc<float> >() { return 16.0 / 16777216.0; }
template <> __device__ constexpr double acc_keep<xacc<double> >() { return 16.0 / 17592186044416.0; }
template <> __device__ constexpr double acc_keep<double>() { return 16.0 / 8388608.0; }

// accumulator of a kernel: extended unless PLAIN
template <typename R, bool PLAIN> struct AccSel { typedef xacc<R> T; };
template <typename R> struct AccSel<R, true> { typedef R T; };
template <typename A> struct R_of { typedef A type; };
template <typename T> struct R_of<xacc<T> > { typedef T type; };
template <typename A> struct AccFrom {
    __device__ static A get(typename R_of<A>::type a) { return A{a, typename R_of<A>::type(0)}; }
};
template <> struct AccFrom<double> {
    __device__ static double get(double a) { return a; }
};
template <typename A>
__device__ inline A acc_from(typename R_of<A>::type a) { return AccFrom<A>::get(a); }

// Exact floor(a / n) for 0 <= a < 2^26 and 1 <= n <= 65535 by one 64-bit
// multiply and a shift (Granlund-Montgomery): with L = ceil(log2 n), s = 26 + L
// and m = floor(2^s / n) + 1, a m / 2^s exceeds a / n by less than
// a / 2^s < 2^-L <= 1/n, which never reaches the next integer.  The GPU has no
// integer divider: a plain division compiles to float reciprocals and
// conversions, and conversions issue on the FP64 pipe, at 1/64 of the FP32
// rate on this chip.
struct DivN {
    uint32_t m;
    int s;
};
__host__ __device__ inline DivN divn_make(int n)
{
    int L = 0;
    while ((1 << L) < n) ++L;
    DivN d;
    d.s = 26 + L;
    d.m = (uint32_t)((1ull << d.s) / (uint64_t)n) + 1u;
    return d;
}
__host__ __device__ inline int divn(uint32_t a, DivN d)
{
    return (int)(((uint64_t)a * d.m) >> d.s);
}

// per-frequency chunk table, window prefixes and reduction scratch (always
// shared memory).  px: exclusive prefixes over chunks of the raw moments
// sum w, sum w x, sum w x^2 (x about 0); pc: per channel sum w v and
// sum w x v.  Entry u is the sum over chunks 0..u-1; entry G the total.
template <typename R, typename A>
struct Small {
    int *cs;       // [G + 1] chunk starts
    A *px;         // [3][G + 1]
    A *pc;         // [2 * nch][G + 1]
    A *scan;       // [16][8] warp totals of a scan
    double *red;   // [96] reduction scratch
    int *ired;     // [32]
    int *flags;    // [4]
    DivN dn;       // division by the item's n (chunk lookups)
};

// channels a variant smooths at once: SS pass B smooths three residual
// columns and their difference; SP only y
__host__ __device__ inline int max_channels(int variant) { return variant == VAR_SS ? 4 : 1; }

template <typename A>
__host__ __device__ inline size_t small_bytes(int G, int variant)
{
    const size_t a = sizeof(A);
    return align16(4 * (size_t)(G + 1)) + align16(a * 3 * (size_t)(G + 1)) +
           align16(a * 2 * (size_t)max_channels(variant) * (size_t)(G + 1)) + 16 * 8 * a +
           96 * 8 + 32 * 4 + 16;
}

template <typename R, typename A>
__device__ inline Small<R, A> carve_small(unsigned char *base, int G, int variant)
{
    Small<R, A> s;
    s.cs = (int *)base;
    base += align16(4 * (size_t)(G + 1));
    s.px = (A *)base;
    base += align16(sizeof(A) * 3 * (size_t)(G + 1));
    s.pc = (A *)base;
    base += align16(sizeof(A) * 2 * (size_t)max_channels(variant) * (size_t)(G + 1));
    s.scan = (A *)base;
    base += 16 * 8 * sizeof(A);
    s.red = (double *)base;
    s.ired = (int *)(base + 768);
    s.flags = (int *)(base + 768 + 128);
    return s;
}

// ---------------------------------------------------------------------------
// block helpers
// ---------------------------------------------------------------------------
__device__ inline double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < nw; ++k) t += red[k];
        red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}

// exclusive scan of cnt[0..nb) in place; returns the largest count
__device__ inline int block_exclusive_scan(uint32_t *cnt, int nb, int *ired)
{
    const int G = blockDim.x, tid = threadIdx.x;
    const int per = nb > G ? nb >> (__ffs(G) - 1) : 1;   // nb and G are powers of two
    const int a = min(nb, tid * per), len = min(nb, a + per) - a;
    // Blocks of 16 or more counts: each thread walks its block starting at
    // offset sk, so that the lanes of a warp, whose blocks lie per words
    // apart, read 32 different banks; head is the sum of the counts before
    // sk.  (nb and G are powers of two, so a non-empty block holds exactly
    // per counts; any other shape walks in order.)  Shorter blocks conflict
    // at most 8 ways and walk in order: there the rotation costs more than
    // it saves.
    const int lg = __ffs(per) - 1;   // log2(per) when per is a power of two
    const int sk = (per >= 16 && len == per && (per & (per - 1)) == 0)
                       ? (tid >> (lg >= 5 ? 0 : 5 - lg)) & (per - 1) : 0;
    uint32_t sum = 0, mx = 0, head = 0;
    if (sk == 0) {
        for (int i = a; i < a + len; ++i) {
            const uint32_t c = cnt[i];
            sum += c;
            mx = c > mx ? c : mx;
        }
    } else {
        for (int k = 0; k < len; ++k) {
            const int r = k + sk < len ? k + sk : k + sk - len;
            const uint32_t c = cnt[a + r];
            sum += c;
            mx = c > mx ? c : mx;
            head += r < sk ? c : 0u;
        }
    }
    // inclusive warp scan of per-thread sums
    const int lane = tid & 31, warp = tid >> 5, nw = (G + 31) >> 5;
    uint32_t inc = sum;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if (lane == 31) ired[warp] = (int)inc;
    if (lane == 0) ired[16 + warp] = (int)mx;
    __syncthreads();
    uint32_t wbase = 0;
    for (int k = 0; k < warp; ++k) wbase += (uint32_t)ired[k];
    int gmax = 0;
    for (int k = 0; k < nw; ++k) gmax = max(gmax, ired[16 + k]);
    const uint32_t start = wbase + inc - sum;   // exclusive prefix at a
    uint32_t run = start + head;                 // ... and at a + sk
    if (sk == 0) {
        for (int i = a; i < a + len; ++i) {
            const uint32_t c = cnt[i];
            cnt[i] = run;
            run += c;
        }
    } else {
        for (int k = 0; k < len; ++k) {
            int r = k + sk;
            if (r >= len) {
                r -= len;
                if (r == 0) run = start;
            }
            const uint32_t c = cnt[a + r];
            cnt[a + r] = run;
            run += c;
        }
    }
    __syncthreads();
    return gmax;
}

// The phase k 2^-64 of a 64-bit fixed-point key, truncated to float (round
// toward zero), built from the key's bits: the exponent from the position of
// its leading one, the significand from the 23 bits below it.  (An integer to
// float conversion instruction would issue on the FP64 pipe.)
__device__ inline float key_to_float_rz(uint64_t k)
{
    if (k == 0) return 0.f;
    const int e = 63 - __clzll((long long)k);   // leading one: value in [2^(e-64), 2^(e-63))
    const uint32_t mant = (uint32_t)((e >= 23 ? k >> (e - 23) : k << (23 - e)) & 0x7fffffu);
    return __int_as_float(((e + 63) << 23) | (int)mant);   // exponent field (e - 64) + 127
}

// ---------------------------------------------------------------------------
// fold (Alg. 1 computePhasedTime)
// ---------------------------------------------------------------------------
// FP64: the binary64 product rounded once, then its fraction (exact).
__device__ inline double fold_fp64(double tt, double f)
{
    double p = __dmul_rn(tt, f);
    return __dsub_rn(p, floor(p));
}

// ---------------------------------------------------------------------------
// stable argsort of the folded phases: perm[j] = index of the j-th smallest
// ---------------------------------------------------------------------------
template <typename R>
__device__ inline bool key_less(const Frame<R> &fr, uint32_t i, uint32_t j)
{
    const uint64_t ki = fr.key[i], kj = fr.key[j];
    if (ki != kj) return ki < kj;
    if (sizeof(R) == 8) {
        const double a = fr.ph[i], b = fr.ph[j];
        if (a != b) return a < b;   // phases below 2^-64 apart (tiny phases only)
    }
    return i < j;
}

template <typename R>
__device__ __noinline__ void bitonic_argsort(const Frame<R> fr, int n)
{
    const int tid = threadIdx.x, G = blockDim.x;
    const int np2 = pow2_at_least(n);
    for (int p = tid; p < np2; p += G) fr.perm[p] = (p < n) ? (uint16_t)p : (uint16_t)0xffff;
    __syncthreads();
    for (int k = 2; k <= np2; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int p = tid; p < np2; p += G) {
                const int q = p ^ jj;
                if (q > p) {
                    const uint16_t a = fr.perm[p], b = fr.perm[q];
                    const bool up = ((p & k) == 0);
                    // padding (0xffff, never a real index since n <= 65535) sorts last
                    const bool a_gt_b = (a == 0xffff) ? (b != 0xffff)
                                      : (b == 0xffff) ? false : key_less(fr, b, a);
                    if (a_gt_b == up) {
                        fr.perm[p] = b;
                        fr.perm[q] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Fold (Alg. 1 computePhasedTime) and stable argsort of the phases: a
// counting sort on the top bits of the 64-bit fixed-point phase into about
// n/2 buckets, each bucket ranked by full key, then original index (FP64:
// binary64 phase between equal keys, then index); buckets more crowded than
// kBucketRankMax fall back to a bitonic sort.  On return perm holds the
// original index of each sorted point and key the sorted keys.
template <typename R, typename A>
__device__ void fold_and_sort(const Frame<R> &fr, int n, const Small<R, A> &sm, const double *tt,
                              double f)
{
    const FoldFreq F = fold_freq(f);
    const int tid = threadIdx.x, G = blockDim.x;
    const int nb = bucket_count(n);
    const int shift = 32 - (31 - __clz(nb));
    for (int b = tid; b < nb; b += G) fr.cnt[b] = 0u;
    __syncthreads();
    for (int i = tid; i < n; i += G) {
        uint64_t fx;
        if (sizeof(R) == 8) {
            const double ph = fold_fp64(tt[i], f);
            fr.ph[i] = ph;
            fx = __double2ull_rz(ph * 18446744073709551616.0);
        } else {
            fx = fold_fixed64_fast(tt[i], F);
        }
        fr.key[i] = fx;
        fr.slot[i] = (uint16_t)atomicAdd(&fr.cnt[(uint32_t)(fx >> 32) >> shift], 1u);
    }
    __syncthreads();
    const int crowd = block_exclusive_scan(fr.cnt, nb, sm.ired);
    if (crowd > kBucketRankMax) {
        bitonic_argsort(fr, n);
        // sorted keys by way of the scatter scratch
        for (int p = tid; p < n; p += G) {
            const uint32_t i = fr.perm[p];
            fr.sk[p] = fr.key[i];
        }
        __syncthreads();
        for (int p = tid; p < n; p += G) fr.key[p] = fr.sk[p];
        __syncthreads();
        return;
    }
    // scatter index and key to the bucket's slots
    for (int i = tid; i < n; i += G) {
        const uint64_t k = fr.key[i];
        const int p = (int)fr.cnt[(uint32_t)(k >> 32) >> shift] + fr.slot[i];
        fr.tmp[p] = (uint16_t)i;
        fr.sk[p] = k;
    }
    __syncthreads();
    // rank within the bucket (its members sit next to each other)
    for (int p = tid; p < n; p += G) {
        const uint32_t i = fr.tmp[p];
        const uint64_t k = fr.sk[p];
        const uint32_t b = (uint32_t)(k >> 32) >> shift;
        const int lo = (int)fr.cnt[b];
        const int hi = (b + 1 < (uint32_t)nb) ? (int)fr.cnt[b + 1] : n;
        int rank = 0;
        for (int q = lo; q < hi; ++q) {
            const uint64_t qk = fr.sk[q];
            bool less = qk < k;
            if (qk == k) {
                const uint32_t iq = fr.tmp[q];
                less = iq < i;
                if (sizeof(R) == 8 && fr.ph[iq] != fr.ph[i]) less = fr.ph[iq] < fr.ph[i];
            }
            rank += less ? 1 : 0;
        }
        fr.perm[lo + rank] = (uint16_t)i;
        fr.key[lo + rank] = k;
    }
    __syncthreads();
}


// ---------------------------------------------------------------------------
// running-line machinery
// ---------------------------------------------------------------------------
// Neighbours per side (Friedman 1984): trunc(0.5*span*n + 0.5), >= 2, and at
// most (n-1)/2 so that no window holds a point twice.  Rounded exactly as the
// binary64 expression reads (no contraction).
__device__ inline int half_width(int n, double span)
{
    int ibw = (int)__dadd_rn(__dmul_rn(__dmul_rn(0.5, span), (double)n), 0.5);
    if (ibw < 2) ibw = 2;
    if (2 * ibw + 1 > n) ibw = (n - 1) / 2;
    return ibw;
}

// sums of a window about origin o: W = sum w, A = sum w dx, B = sum w dx^2,
// C[c] = sum w v_c, D[c] = sum w dx v_c, dx = x - o
template <typename R, int NCH>
struct Win {
    R W, A, B, C[NCH], D[NCH];
    R hiB;   // largest B the sums have held: the scale of their rounding error
    __device__ inline void zero()
    {
        W = A = B = hiB = R(0);
#pragma unroll
        for (int c = 0; c < NCH; ++c) C[c] = D[c] = R(0);
    }
};

// FP32C divides with the approximate reciprocal (about 1 ulp), far cheaper
// than an IEEE division and inside the path's error budget; FP64 divides
// exactly.
__device__ inline float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ inline double fdiv(double a, double b) { return a / b; }

// window slot e (may lie one period before 0 or after n-1) -> point, shift
__device__ inline int slot_point(int e, int n, int &sh)
{
    if (e < 0) { sh = -1; return e + n; }
    if (e >= n) { sh = 1; return e - n; }
    sh = 0;
    return e;
}
template <typename R>
__device__ inline int slot_point_r(int e, int n, R &shift)
{
    const int lo = e < 0, hi = e >= n;
    shift = lo ? R(-1) : (hi ? R(1) : R(0));
    return e + (lo ? n : 0) - (hi ? n : 0);
}

// Channel c at point p.  With DIFF the last channel is not stored: it is
// channel 0 minus channel 1, smoothed directly so that its sign is exact where
// the two smooths round to the same value (the running line is linear).
template <typename R, int NCH, bool DIFF>
__device__ inline R chan(const R *const *v, int c, int p)
{
    if (DIFF && c == NCH - 1) return v[0][p] - v[1][p];
    return v[c][p];
}

template <typename R, int NCH, bool DIFF = false>
__device__ inline void win_add(Win<R, NCH> &s, const Frame<R> &fr, const R *const *v, int e,
                               int n, R o, R sign)
{
    R shf;
    const int p = slot_point_r<R>(e, n, shf);
    const typename Vec2<R>::T xw = fr.XW[p];
    const R dx = (xw.x - o) + shf;
    const R w = sign * xw.y;
    const R wdx = w * dx;
    s.W += w;
    s.A += wdx;
    s.B += wdx * dx;
    if (sizeof(R) == 4) s.hiB = fmax(s.hiB, s.B);
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        R vc = chan<R, NCH, DIFF>(v, c, p);
        s.C[c] += w * vc;
        s.D[c] += wdx * vc;
    }
}

// Exclusive block-wide scan of Q accumulator values per thread (one entry per
// chunk): out[q][t] = sum over threads < t, out[q][G] = total.  Warps scan
// with shuffles and publish their totals; after one barrier every warp sums
// the totals of the warps before it itself (a shuffle reduction over at most
// 16 lanes), so no warp waits on a serial second-level scan.  The caller
// synchronises before reading out, and that barrier also orders this scan's
// reads of scratch before the next scan's writes.
template <typename A, int Q>
__device__ void block_scan_store(A (&v)[Q], A *const (&out)[Q], A *scratch)
{
    typedef typename R_of<A>::type T;
    const int G = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = G >> 5;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const A y = acc_shfl_up(v[q], k);
            if (lane >= k) v[q] = acc_add(v[q], y);
        }
    }
    A ex[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        ex[q] = acc_shfl_up(v[q], 1);
        if (lane == 0) ex[q] = acc_from<A>(T(0));
    }
    if (nw == 1) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            out[q][tid] = ex[q];
            if (lane == 31) out[q][G] = v[q];
        }
        return;
    }
    if (lane == 31) {
#pragma unroll
        for (int q = 0; q < Q; ++q) scratch[warp * 8 + q] = v[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        // offset of this warp: the totals of warps 0 .. warp-1, summed over
        // lanes 0 .. nw-1 (nw is a power of two, so the butterflies below
        // never mix in lanes >= nw)
        A b = lane < warp ? scratch[lane * 8 + q] : acc_from<A>(T(0));
        for (int k = 1; k < nw; k <<= 1) b = acc_add(b, acc_shfl_xor(b, k));
        b = acc_shfl_idx(b, 0);
        out[q][tid] = acc_add(b, ex[q]);
        if (tid == G - 1) out[q][G] = acc_add(b, v[q]);
    }
}

// The same scan with warp 0 scanning the warp totals between two barriers:
// more waiting, but fewer registers live across the barriers, which the SS
// kernels for short objects (few warps per CTA) need to keep their occupancy.
template <typename A, int Q>
__device__ void block_scan_store_serial(A (&v)[Q], A *const (&out)[Q], A *scratch)
{
    typedef typename R_of<A>::type T;
    const int G = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = G >> 5;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const A y = acc_shfl_up(v[q], k);
            if (lane >= k) v[q] = acc_add(v[q], y);
        }
    }
    A ex[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        ex[q] = acc_shfl_up(v[q], 1);
        if (lane == 0) ex[q] = acc_from<A>(T(0));
    }
    if (nw == 1) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            out[q][tid] = ex[q];
            if (lane == 31) out[q][G] = v[q];
        }
        return;
    }
    __syncthreads();   // the previous scan has finished reading scratch
    if (lane == 31) {
#pragma unroll
        for (int q = 0; q < Q; ++q) scratch[warp * 8 + q] = v[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            A t = lane < nw ? scratch[lane * 8 + q] : acc_from<A>(T(0));
            for (int k = 1; k < nw; k <<= 1) {
                const A y = acc_shfl_up(t, k);
                if (lane >= k) t = acc_add(t, y);
            }
            A b = acc_shfl_up(t, 1);
            if (lane == 0) b = acc_from<A>(T(0));
            if (lane < nw) scratch[lane * 8 + q] = b;
            if (lane == nw - 1) out[q][G] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) out[q][tid] = acc_add(scratch[warp * 8 + q], ex[q]);
}

// x-moment prefixes of the chunks together with the prefixes of one channel
// (sum w v, sum w x v), all about 0
template <typename R, bool SERIAL = false, typename A>
__device__ void build_xy_prefix(const Frame<R> &fr, const Small<R, A> &sm, const R *vy, int c0,
                                int c1, R o)
{
    const int L = blockDim.x + 1;
    R w_ = R(0), a_ = R(0), b_ = R(0), sc = R(0), sd = R(0);
    for (int j = c0; j < c1; ++j) {
        const typename Vec2<R>::T xw = fr.XW[j];
        const R w = xw.y, d = xw.x - o, wv = w * vy[j];
        w_ += w;
        a_ += w * d;
        b_ += w * d * d;
        sc += wv;
        sd += wv * d;
    }
    // about 0: sum w x = a + o W, sum w x^2 = b + 2 o a + o^2 W, sum w x v = d + o c
    A v[5];
    v[0] = acc_from<A>(w_);
    v[1] = acc_add(acc_from<A>(a_), acc_mul(acc_from<A>(w_), o));
    v[2] = acc_add(acc_add(acc_from<A>(b_), acc_mul(acc_from<A>(a_), R(2) * o)),
                   acc_mul(acc_mul(acc_from<A>(w_), o), o));
    v[3] = acc_from<A>(sc);
    v[4] = acc_add(acc_from<A>(sd), acc_mul(acc_from<A>(sc), o));
    A *const out[5] = {sm.px, sm.px + L, sm.px + 2 * L, sm.pc, sm.pc + L};
    if (SERIAL) block_scan_store_serial<A, 5>(v, out, sm.scan);
    else block_scan_store<A, 5>(v, out, sm.scan);
}

// channel prefixes of the chunks (each later pass).  With FIX, a stored
// channel value below 0 (a CV residual whose leverage reached 1) is first
// replaced by the previous centre's (0 at the first centre), as Listing 1
// does; a value read from a neighbouring chunk while its owner resolves it is
// either still negative (the walk goes on) or already the value the walk
// would find.
template <typename R, int NCH, bool DIFF = false, bool FIX = false, bool SERIAL = false, typename A>
__device__ void build_channel_prefix(const Frame<R> &fr, const Small<R, A> &sm, const R *const *vv,
                                     int c0, int c1, R o)
{
    constexpr int NS = DIFF ? NCH - 1 : NCH;   // stored channels
    const int L = blockDim.x + 1;
    R sc[NCH], sd[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) sc[ch] = sd[ch] = R(0);
    for (int j = c0; j < c1; ++j) {
        const typename Vec2<R>::T xw = fr.XW[j];
        const R w = xw.y, d = xw.x - o;
        R val[NCH];
#pragma unroll
        for (int ch = 0; ch < NS; ++ch) {
            R x = vv[ch][j];
            if (FIX && x < R(0)) {
                int q = j - 1;
                while (q >= 0 && vv[ch][q] < R(0)) --q;
                x = (q >= 0) ? vv[ch][q] : R(0);
                const_cast<R *>(vv[ch])[j] = x;
            }
            val[ch] = x;
        }
        if (DIFF) val[NCH - 1] = val[0] - val[1];
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            const R wv = w * val[ch];
            sc[ch] += wv;
            sd[ch] += wv * d;
        }
    }
    A v[2 * NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        v[2 * ch] = acc_from<A>(sc[ch]);
        v[2 * ch + 1] = acc_add(acc_from<A>(sd[ch]), acc_mul(acc_from<A>(sc[ch]), o));  // sum w x v about 0
    }
    A *out[2 * NCH];
#pragma unroll
    for (int q = 0; q < 2 * NCH; ++q) out[q] = sm.pc + q * L;
    if (SERIAL) block_scan_store_serial<A, 2 * NCH>(v, out, sm.scan);
    else block_scan_store<A, 2 * NCH>(v, out, sm.scan);
}

// Chunk u starts at cs[u] = floor(u n / G), moved forward past a run of ties
// it would split, so cs[u] >= floor(u n / G): the arithmetic guess below is
// never too low, and the correction walks down over tie-emptied chunks only.
// First chunk starting at or after p (0 <= p <= n):
__device__ inline int chunk_lower(const int *cs, int G, int n, DivN dn, int p)
{
    int u = divn((unsigned)(p * G) + (unsigned)(n - 1), dn);   // ceil(p G / n): cs[u] >= p
    while (u > 0 && cs[u - 1] >= p) --u;
    return u;
}
// Last chunk boundary at or before q (0 <= q <= n):
__device__ inline int chunk_upper(const int *cs, int G, int n, DivN dn, int q)
{
    int u = divn((unsigned)((q + 1) * G) + (unsigned)(n - 1), dn) - 1;   // floor(u n / G) <= q
    if (u > G) u = G;
    while (cs[u] > q) --u;
    return u;
}

// one point at slot p (0 <= p < n) with abscissa shift sh (-1, 0, +1)
template <typename R, int NCH, bool DIFF>
__device__ inline void win_add_slot(Win<R, NCH> &s, const Frame<R> &fr, const R *const *v, int p,
                                    R sh, R o, R sgn)
{
    const typename Vec2<R>::T xw = fr.XW[p];
    const R dx = (xw.x - o) + sh;
    const R w = sgn * xw.y;
    const R wdx = w * dx;
    s.W += w;
    s.A += wdx;
    s.B += wdx * dx;
    if (sizeof(R) == 4) s.hiB = fmax(s.hiB, s.B);
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        R vc = chan<R, NCH, DIFF>(v, c, p);
        s.C[c] += w * vc;
        s.D[c] += wdx * vc;
    }
}

// Prefix of the chunks before chunk boundary u of period k (-1, 0, +1) of the
// periodic extension, in extended slot order: with P_u the prefix of period 0
// and T the total, Q = P_u for k = 0, T + P_u with x -> x + 1 for k = +1 and
// (P_u - T) with x -> x - 1 for k = -1 (the slots of period -1 before the
// boundary are those of chunks u.. of period 0, counted negatively).  The
// moments transform as sum w (x+k) = S1 + k W, sum w (x+k)^2 = S2 + 2k S1 + W,
// sum w (x+k) v = D + k C.
template <typename R, int NCH, typename A>
__device__ inline void ext_prefix(const Small<R, A> &sm, int u, int k, A &W, A &S1, A &S2,
                                  A (&C)[NCH], A (&D)[NCH])
{
    const int L = blockDim.x + 1, G = blockDim.x;
    W = sm.px[0 * L + u];
    S1 = sm.px[1 * L + u];
    S2 = sm.px[2 * L + u];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        C[ch] = sm.pc[(2 * ch) * L + u];
        D[ch] = sm.pc[(2 * ch + 1) * L + u];
    }
    if (k == 0) return;
    if (k < 0) {
        W = acc_add(W, acc_neg(sm.px[0 * L + G]));
        S1 = acc_add(S1, acc_neg(sm.px[1 * L + G]));
        S2 = acc_add(S2, acc_neg(sm.px[2 * L + G]));
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            C[ch] = acc_add(C[ch], acc_neg(sm.pc[(2 * ch) * L + G]));
            D[ch] = acc_add(D[ch], acc_neg(sm.pc[(2 * ch + 1) * L + G]));
        }
    }
    const R sg = k < 0 ? R(-1) : R(1);
    S2 = acc_add(S2, acc_add(acc_mul(S1, R(2) * sg), W));
    S1 = acc_add(S1, acc_mul(W, sg));
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) D[ch] = acc_add(D[ch], acc_mul(C[ch], sg));
    if (k > 0) {
        W = acc_add(W, sm.px[0 * L + G]);
        S1 = acc_add(S1, sm.px[1 * L + G]);
        S2 = acc_add(S2, sm.px[2 * L + G]);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            C[ch] = acc_add(C[ch], sm.pc[(2 * ch) * L + G]);
            D[ch] = acc_add(D[ch], sm.pc[(2 * ch + 1) * L + G]);
        }
    }
}

// Chunk boundary nearest to position p (0 <= p <= n) of one period: the
// first boundary at or after p, or the one before it when that is closer.
__device__ inline int chunk_nearest(const int *cs, int G, int n, DivN dn, int p)
{
    const int u = chunk_lower(cs, G, n, dn, p);
    return (u > 0 && p - cs[u - 1] < cs[u] - p) ? u - 1 : u;
}

// Sums of the window [c - h, c + h] about origin o.  In the periodic
// extension of the sorted points (slot e is point e mod n with x shifted by
// floor(e / n)), each end of the window is taken to its nearest chunk
// boundary; the whole chunks between the two boundaries come from the
// extended-precision prefixes (raw moments about 0, ext_prefix), and the
// points between each end and its boundary are added or subtracted one by
// one, both ends in one loop.  The sums are then moved to origin o in the
// extended type and rounded once.
template <typename R, int NCH, bool DIFF = false, typename A>
__device__ inline void win_init_body(Win<R, NCH> &s, const Frame<R> &fr, const Small<R, A> &sm,
                                     const R *const *v, int c, int h, int n, R o)
{
    const int G = blockDim.x, L = G + 1;
    s.zero();
    const int ea = win_lo(fr, c, h, n), eb = ea + 2 * h;
    if (2 * h + 1 <= kDirectInit) {
        // a short window costs less summed point by point than from prefixes
        for (int e = ea; e <= eb; ++e) win_add<R, NCH, DIFF>(s, fr, v, e, n, o, R(1));
        return;
    }
    // ends of the half-open slot range [ea, eb + 1): period and position
    // (-n < ea < n and 0 < eb + 1 < 2n; clamped windows lie in period 0)
    const int ka = ea < 0 ? -1 : 0, kb = eb + 1 > n ? 1 : 0;
    const int pa = ea - ka * n, pb = eb + 1 - kb * n;
    const int ua = chunk_nearest(sm.cs, G, n, sm.dn, pa);
    const int ub = chunk_nearest(sm.cs, G, n, sm.dn, pb);
    A W, S1, S2, C[NCH], D[NCH];
    {
        A W0, S10, S20, C0[NCH], D0[NCH];
        ext_prefix<R, NCH, A>(sm, ua, ka, W0, S10, S20, C0, D0);
        ext_prefix<R, NCH, A>(sm, ub, kb, W, S1, S2, C, D);
        W = acc_add(W, acc_neg(W0));
        S1 = acc_add(S1, acc_neg(S10));
        S2 = acc_add(S2, acc_neg(S20));
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            C[ch] = acc_add(C[ch], acc_neg(C0[ch]));
            D[ch] = acc_add(D[ch], acc_neg(D0[ch]));
        }
    }
    // ragged ends, both in one loop: points [la, la + nl) of period ka with
    // sign sl, points [lb, lb + nr) of period kb with sign sr
    const int qa = sm.cs[ua], qb = sm.cs[ub];
    const int la = qa >= pa ? pa : qa, nl = qa >= pa ? qa - pa : pa - qa;
    const int lb = qb <= pb ? qb : pb, nr = qb <= pb ? pb - qb : qb - pb;
    const R sl = qa >= pa ? R(1) : R(-1), sr = qb <= pb ? R(1) : R(-1);
    const R sha = (R)ka, shb = (R)kb;
    const int nm = nl > nr ? nl : nr;
    for (int k = 0; k < nm; ++k) {
        if (k < nl) win_add_slot<R, NCH, DIFF>(s, fr, v, la + k, sha, o, sl);
        if (k < nr) win_add_slot<R, NCH, DIFF>(s, fr, v, lb + k, shb, o, sr);
    }
    // about o: A = S1 - o W, B = S2 - 2 o S1 + o^2 W, D = D - o C
    const A oW = acc_mul(W, o);
    const R wr = acc_to(W);
    const R ar = acc_to(acc_add(S1, acc_neg(oW)));
    const R br = acc_to(acc_add(acc_add(S2, acc_neg(acc_mul(S1, R(2) * o))), acc_mul(oW, o)));
    // Every prefix term is bounded by 16 x (total weight): |x| <= 2 after a
    // wrap and |o| < 1.  The accumulator's rounding therefore leaves B with a
    // relative error below eps_acc * 16 tW / B; where that could exceed about
    // 2^-24 (double-float), 2^-56 (double-double) or 2^-30 (plain binary64,
    // FP64 recompute) of B, the window is clustered so tightly that it is
    // summed point by point about o instead.
    const R tw = acc_to(sm.px[0 * L + G]);
    const R keep = R(acc_keep<A>());
    if (!(br > tw * keep)) {
        s.zero();
        for (int e = ea; e <= eb; ++e) win_add<R, NCH, DIFF>(s, fr, v, e, n, o, R(1));
        return;
    }
    s.W += wr;
    s.A += ar;
    s.B += br;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        s.C[ch] += acc_to(C[ch]);
        s.D[ch] += acc_to(acc_add(D[ch], acc_neg(acc_mul(C[ch], o))));
    }
    if (sizeof(R) == 4) s.hiB = fmax(s.hiB, s.B);
}

// Window initialisation, in line or (OOL) out of line.  Out of line there is
// one copy of the code per channel layout instead of one per call site, which
// keeps the SS passes' instruction footprint small; the call takes only what
// the initialisation reads (phases and weights, window mode, channels, chunk
// starts and prefixes), but saves and restores the caller's live registers.
// Long objects (few centres per thread, long windows) gain: C2 SS runs 7%
// faster.  Short ones lose (C3 SS 4% slower), so the kernels for them keep
// it in line.
template <typename R, int NCH>
struct Chans {
    const R *p[NCH];
};
template <typename R, int NCH, bool DIFF, typename A>
__device__ __noinline__ Win<R, NCH> win_init_ool(const typename Vec2<R>::T *XW, int per,
                                                 const Chans<R, NCH> cv, int *cs, A *px, A *pc,
                                                 DivN dn, int c, int h, int n, R o)
{
    Frame<R> fr{};
    fr.XW = const_cast<typename Vec2<R>::T *>(XW);
    fr.per = per;
    Small<R, A> sm{};
    sm.cs = cs;
    sm.px = px;
    sm.pc = pc;
    sm.dn = dn;
    const R *v[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) v[ch] = cv.p[ch];
    Win<R, NCH> s;
    win_init_body<R, NCH, DIFF>(s, fr, sm, v, c, h, n, o);
    return s;
}
template <typename R, int NCH, bool DIFF = false, bool OOL = false, typename A>
__device__ inline void win_init(Win<R, NCH> &s, const Frame<R> &fr, const Small<R, A> &sm,
                                const R *const *v, int c, int h, int n, R o)
{
    if constexpr (OOL) {
        Chans<R, NCH> cv;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) cv.p[ch] = (DIFF && ch == NCH - 1) ? nullptr : v[ch];
        s = win_init_ool<R, NCH, DIFF, A>(fr.XW, fr.per, cv, sm.cs, sm.px, sm.pc, sm.dn, c, h, n, o);
    } else {
        win_init_body<R, NCH, DIFF>(s, fr, sm, v, c, h, n, o);
    }
}

// the line fit of a window evaluated at the centre j
template <typename R, int NCH>
struct Fit {
    R rW, rS, dxj;   // 1/W, 1/Sxx (0 when the slope is dropped), x_j - xbar
    R sxx;
    bool slope;
    R s[NCH];        // fit at the centre
    R b[NCH];        // its slope
};

template <typename R, int NCH>
__device__ inline void win_fit(Fit<R, NCH> &f, const Win<R, NCH> &s, R xj_minus_o, R vsmlsq)
{
    f.rW = fdiv(R(1), s.W);
    const R xb = s.A * f.rW;
    const R sxx = s.B - xb * s.A;
    f.slope = sxx > vsmlsq;
    f.rS = f.slope ? fdiv(R(1), sxx) : R(0);
    f.sxx = sxx;
    f.dxj = xj_minus_o - xb;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const R sxv = s.D[c] - xb * s.C[c];
        f.b[c] = sxv * f.rS;
        f.s[c] = s.C[c] * f.rW + f.b[c] * f.dxj;
    }
}

// FP32C guard: the sliding sums carry absolute errors of order eps times the
// largest moment they have held; where the centred spread is below a fixed
// part of that (a tight cluster after wide windows, or a far origin), this
// centre's window is refitted directly in FP64.
// (out of line, taking only the pointers it reads, by value: the rare call
// must not force the caller's fits, frame or channel table into local memory,
// nor put a frame copy in the hot loop's code)
template <typename R, int NCH, bool DIFF = false>
__device__ __noinline__ Fit<R, NCH> win_refit_fp64(const typename Vec2<R>::T *XW, int per,
                                                   const Chans<R, NCH> cv, int j, int h, int n,
                                                   double vsmlsq)
{
    const R *v[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) v[c] = cv.p[c];
    Fit<R, NCH> f;
    const int lo = win_lo_mode(per, j, h, n);
    double sw = 0.0, swx = 0.0, swv[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) swv[c] = 0.0;
    for (int e = lo; e <= lo + 2 * h; ++e) {
        int sh;
        int p = slot_point(e, n, sh);
        const typename Vec2<R>::T xw = XW[p];
        double w = (double)xw.y, x = (double)xw.x + sh;
        sw += w;
        swx += w * x;
#pragma unroll
        for (int c = 0; c < NCH; ++c) swv[c] += w * (double)chan<R, NCH, DIFF>(v, c, p);
    }
    const double xm = swx / sw;
    double sxx = 0.0, sxv[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) sxv[c] = 0.0;
    for (int e = lo; e <= lo + 2 * h; ++e) {
        int sh;
        int p = slot_point(e, n, sh);
        const typename Vec2<R>::T xw = XW[p];
        double w = (double)xw.y, dx = (double)xw.x + sh - xm;
        sxx += w * dx * dx;
#pragma unroll
        for (int c = 0; c < NCH; ++c) sxv[c] += w * dx * (double)chan<R, NCH, DIFF>(v, c, p);
    }
    const bool slope = sxx > vsmlsq;
    const double dxj = (double)XW[j].x - xm;
    f.rW = (R)(1.0 / sw);
    f.slope = slope;
    f.rS = slope ? (R)(1.0 / sxx) : R(0);
    f.dxj = (R)dxj;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        f.b[c] = (R)(slope ? sxv[c] / sxx : 0.0);
        f.s[c] = (R)(swv[c] / sw + (slope ? sxv[c] / sxx : 0.0) * dxj);
    }
    f.sxx = (R)sxx;
    return f;
}

template <typename R, int NCH, bool DIFF = false>
__device__ inline void win_fit_checked(Fit<R, NCH> &f, const Win<R, NCH> &s, const Frame<R> &fr,
                                       const R *const *v, int j, int h, int n, R o, R vsmlsq,
                                       bool &near, R refit_frac)
{
    win_fit<R, NCH>(f, s, fr.XW[j].x - o, vsmlsq);
    if (sizeof(R) == 4) {
        const R sxx = f.sxx;
        if (sxx < s.hiB * refit_frac && s.hiB > R(0)) {
            Chans<R, NCH> cv;
#pragma unroll
            for (int c = 0; c < NCH; ++c) cv.p[c] = (DIFF && c == NCH - 1) ? nullptr : v[c];
            f = win_refit_fp64<R, NCH, DIFF>(fr.XW, fr.per, cv, j, h, n, (double)vsmlsq);
            f.sxx = sxx;
        }
        if (fabs(sxx - vsmlsq) <= (R)kNearSlope * vsmlsq) near = true;
    }
}

// slide a window from centre j to j + 1
template <typename R, int NCH, bool DIFF = false>
__device__ inline void win_slide(Win<R, NCH> &s, const Frame<R> &fr, const R *const *v, int j,
                                 int h, int n, R o)
{
    // a window clamped inside the data moves only while h <= j <= n - 2 - h,
    // and then exactly as a periodic one does
    if (!fr.per && (j < h || j > n - 2 - h)) return;
    win_add<R, NCH, DIFF>(s, fr, v, j - h, n, o, R(-1));
    win_add<R, NCH, DIFF>(s, fr, v, j + h + 1, n, o, R(1));
}

// Binary64 kernels: the fit of the window of centre j recomputed in two
// passes (weighted means, then centred sums), and 1 - w_j h_j from it.
template <typename R>
__device__ inline void cv_refit(Fit<R, 1> &f, R &d, const Frame<R> &fr, const R *const *v, int j,
                                int h, int n, R vsmlsq, R wj)
{
    Chans<R, 1> cv;
    cv.p[0] = v[0];
    f = win_refit_fp64<R, 1, false>(fr.XW, fr.per, cv, j, h, n, (double)vsmlsq);
    d = R(1) - wj * (f.rW + f.dxj * f.dxj * f.rS);
}

// ---------------------------------------------------------------------------
// Listing 1 pieces shared by SS and SP
// ---------------------------------------------------------------------------
// Span constants of one frequency in the compute precision (built once, so
// the per-centre code does no binary64 arithmetic in the FP32C kernels).
template <typename R>
struct SpanK {
    R s0, s1, s2, inv01, inv21, ex;
    bool bass;   // 0 < alpha <= 10
};
template <typename R>
__device__ inline SpanK<R> span_consts(const double *spans, double alpha)
{
    SpanK<R> k;
    k.s0 = (R)spans[0];
    k.s1 = (R)spans[1];
    k.s2 = (R)spans[2];
    k.inv01 = R(1) / (k.s0 - k.s1);
    k.inv21 = R(1) / (k.s2 - k.s1);
    k.ex = (R)(10.0 - alpha);
    k.bass = alpha > 0.0 && alpha <= 10.0;
    return k;
}

// Span choice at one centre: first strict minimum of the three residuals,
// then bass enhancement toward the woofer span.  Listing 1 enhances only when
// the minimum is strictly below the woofer's residual; as the two approach,
// the enhanced span tends to the woofer's, and exactly at equality it drops
// back.  Two different windows agree exactly only by rounding, and FP32
// rounds far more often than binary64, so for R = float an exact tie between
// different windows (lim_k: window k differs from the woofer's) takes the
// limit value instead.
// d01 (when use_d01) is the directly smoothed r0 - r1: it settles tweeter
// against midrange where r0 and r1 round to the same value.
// (residual ratio)^(10 - alpha) for alpha other than 9: out of line, so that
// the inlined power function does not sit in the per-point loops that take
// the default alpha's plain ratio
static __device__ __noinline__ float span_pow(float x, float e) { return powf(x, e); }
static __device__ __noinline__ double span_pow(double x, double e) { return pow(x, e); }

template <typename R>
__device__ inline R choose_span(const SpanK<R> &K, R r0, R r1, R r2, R res_woof, R fallback,
                                bool lim0, bool lim1, bool use_d01 = false, R d01 = R(0))
{
    R resmin = R(1.0e20), s = fallback;
    int k = -1;
    if (r0 < resmin) { resmin = r0; s = K.s0; k = 0; }
    const bool mid_wins = (use_d01 && k == 0 && r1 < R(1.0e20)) ? (d01 > R(0)) : (r1 < resmin);
    if (mid_wins) { resmin = r1; s = K.s1; k = 1; }
    if (r2 < resmin) { resmin = r2; s = K.s2; k = 2; }
    bool below = resmin < res_woof;
    if (sizeof(R) == 4 && !below && resmin == res_woof && ((k == 0 && lim0) || (k == 1 && lim1)))
        below = true;
    if (K.bass && below && resmin > R(0)) {
        R tmp = fdiv(resmin, res_woof);
        if (tmp < R(1.0e-7)) tmp = R(1.0e-7);
        const R pw = (K.ex == R(1)) ? tmp : span_pow(tmp, K.ex);
        s += (K.s2 - s) * pw;
    }
    return s;
}

// tweeter and midrange residuals so close that FP32 rounding could reorder them
// (diff is their directly smoothed difference).  Each CV residual carries
// an FP32 error of a few ulps of the magnitudes its window sums held, not of
// the residual itself, so the margin has a relative part and an absolute
// one at the object's magnitude scale.
template <typename R>
__device__ inline bool span_contested(R diff, R r0, R r1, float margin, float margin_abs)
{
    return sizeof(R) == 4 && (fabs(diff) <= (R)margin * fmax(r0, r1) || fabs(diff) <= (R)margin_abs);
}

template <typename R>
__device__ inline R interpolate_span(const SpanK<R> &K, R s, R tw, R mid, R woof)
{
    if (s <= K.s0) s = K.s0;
    if (s >= K.s2) s = K.s2;
    R f = s - K.s1;
    if (f < R(0)) {
        f = (sizeof(R) == 8) ? f / (K.s0 - K.s1) : f * K.inv01;
        return (R(1) - f) * mid + f * tw;
    }
    f = (sizeof(R) == 8) ? f / (K.s2 - K.s1) : f * K.inv21;
    return (R(1) - f) * mid + f * woof;
}

// Kahan-compensated running sum (FP32C chi2)
template <typename R>
struct KSum {
    R s = R(0), c = R(0);
    __device__ inline void add(R v)
    {
        if (sizeof(R) == 8) { s += v; return; }
        R y = v - c;
        R t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ inline double value() const { return (double)s - (double)c; }
};

// Run bookkeeping for the averaging step of every running line: centres with
// equal phases get the weighted mean of their values.  Chunks never split a
// run, so a thread sees each run whole.
template <typename R, int K>
struct RunAvg {
    int start;
    R w, s[K];
    __device__ inline void reset(int j)
    {
        start = j;
        w = R(0);
#pragma unroll
        for (int k = 0; k < K; ++k) s[k] = R(0);
    }
};

template <typename R>
__device__ inline bool tie_next(const Frame<R> &fr, int j)
{
    return (fr.tie[j >> 5] >> (j & 31)) & 1u;
}

// Whether the window (half width h) of centre j holds j alone beside points
// that all share one abscissa: then the leave-one-out line does not exist and,
// with the slope in use, j's leverage is exactly 1.  Only a clamped window's
// first or last point can be so (in a centred window the centre lies between
// its neighbours' abscissae, which would then equal its own; a periodic
// window's wrapped points sit a period away); the tie bits tell.
template <typename R>
__device__ inline bool lev_one_end(const Frame<R> &fr, int j, int h, int n)
{
    if (fr.per) return false;
    const int lo = win_lo(fr, j, h, n);
    int a, b;   // pairs (i, i + 1) for i in [a, b) must all be tied
    if (j == lo) { a = lo + 1; b = lo + 2 * h; }
    else if (j == lo + 2 * h) { a = lo; b = lo + 2 * h - 1; }
    else return false;
    for (int i = a; i < b; ++i)
        if (!tie_next(fr, i)) return false;
    return true;
}

template <typename R, int K, typename Emit>
__device__ inline void run_push(RunAvg<R, K> &ra, const Frame<R> &fr, int j, bool ties,
                                const R (&vals)[K], Emit &&emit)
{
    if (!ties) {
        emit(j, vals);
        return;
    }
    const R wj = fr.XW[j].y;
    ra.w += wj;
#pragma unroll
    for (int k = 0; k < K; ++k) ra.s[k] += wj * vals[k];
    if (tie_next(fr, j)) return;   // run continues
    if (ra.start == j) {
        emit(j, vals);
    } else {
        R avg[K];
#pragma unroll
        for (int k = 0; k < K; ++k) avg[k] = ra.s[k] / ra.w;
        for (int i = ra.start; i <= j; ++i) emit(i, avg);
    }
    ra.reset(j + 1);
}


// Error-free pieces of the SP settle.  u22f: an integer below 2^23 as a float,
// exactly, by way of its bit pattern (no conversion instruction).
__device__ inline float u22f(uint32_t m) { return __int_as_float(0x4b000000 | m) - 8388608.0f; }
// (kp - kj) 2^-64 + sh as a double-float, exact to about 2^-48 relative: the
// 64-bit difference of two fixed-point phases is split into three pieces that
// floats hold exactly and summed with an error-free addition.
__device__ inline df key_diff_df(uint64_t kp, uint64_t kj, int sh)
{
    const bool ge = kp >= kj;
    const uint64_t m = ge ? kp - kj : kj - kp;
    const float f2 = u22f((uint32_t)(m >> 44)) * 0x1p-20f;
    const float f1 = u22f((uint32_t)(m >> 22) & 0x3fffffu) * 0x1p-42f;
    const float f0 = u22f((uint32_t)m & 0x3fffffu) * 0x1p-64f;
    df v = x_two_sum(f2, f1);
    v = x_fast(v.hi, v.lo + f0);
    if (!ge) v = df{-v.hi, -v.lo};
    if (sh) v = acc_add(df{(float)sh, 0.f}, v);
    return v;
}
// product of two double-floats, rounded once to a double-float (FMA-exact
// leading product plus the cross terms)
__device__ inline df df_mul(df a, df b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return x_fast(p, e);
}
// running sum: the leading parts add error-free, the low parts and the
// errors collect in lo (renormalised once at the end)
__device__ inline void df_acc(df &s, df x)
{
    const df t = x_two_sum(s.hi, x.hi);
    s.hi = t.hi;
    s.lo += t.lo + x.lo;
}
__device__ inline double df_to_double(df x) { return (double)x.hi + (double)x.lo; }
// quotient of two double-floats to about 2^-44 relative: an approximate
// quotient q1, the residual a - q1 b (its leading part exact by an FMA, the
// difference a.hi - q1 b.hi exact by Sterbenz's lemma), and its quotient as
// the correction
__device__ inline df df_div(df a, df b)
{
    const float q1 = __fdividef(a.hi, b.hi);
    const float p = q1 * b.hi;
    const float e = fmaf(q1, b.hi, -p);
    const float r = fmaf(-q1, b.lo, ((a.hi - p) - e) + a.lo);
    return x_fast(q1, __fdividef(r, b.hi));
}
__device__ inline df df_sub(df a, df b) { return acc_add(a, acc_neg(b)); }
// a < b for normalised double-floats (|lo| at most half an ulp of hi)
__device__ inline bool df_less(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ inline df df_abs(df a) { return a.hi < 0.f ? acc_neg(a) : a; }

// Settles one contested SP centre je beyond FP32 precision: the line fits of
// its span windows from the exact phases (the sorted 64-bit fixed-point keys)
// and the inputs as double-float pairs read through perm, and the residual
// comparisons of the span choice, all in double-float arithmetic on the FP32
// pipe (about 2^-44 relative, against binary64's 2^-53; the FP64 pipe issues
// at 1/64 of the FP32 rate on this chip).  Once the choice is taken, bass
// enhancement and interpolation depend on the residuals and fits only
// continuously, and run in FP32 like every other centre's.  The windows share
// their centre and nest (h0 <= h1 <= h2, periodic or clamped), so each point
// is loaded and summed once: into the tweeter window, or the ring the
// midrange window adds around it, or the woofer's ring around that (each
// ring's two segments in one walk); the wider windows' sums are running
// totals.  sl: bit k set when span k's fit kept its slope, which picks the
// validation factor as in the FP32 choice.  Bit 3 of sl asks for the woofer
// window too.  Without it (a near-tie whose smaller residual lies more than
// 1e-4 relative below the woofer's) the woofer's FP32 fit s2f and residual
// g2f stand in: the span then depends on them only continuously, and the
// woofer's ring, the longest walk, is skipped.
// The code runs rarely, from a cold instruction cache, so it is out of line
// and written once per step (only the walk is unrolled).  All lanes of the
// warp call it together with the same centre; every lane returns the smooth.
template <typename R>
__device__ __noinline__ float sp_settle(const Frame<R> fr, const float2 *ydf, const float2 *wdf,
                                        int je, int h0, int h1, int h2, int n, int qi, int qj,
                                        int sl, const SpanK<float> K, float s2f, float g2f)
{
    // bit 3 of sl: refit the woofer window as well, else take its FP32 fit
    const int nk = (sl & 8) ? 3 : 2;
    const uint64_t *key = fr.key;
    // Listing 1's vsmlsq = 1e-6 scale^2 from the exact phases at the scale
    // indices qi, qj (1e-6 as a double-float: the binary64 constant split)
    const df sq = key_diff_df(key[qj], key[qi], 0);
    const df vsm = df_mul(df_mul(sq, sq), df{1.0e-6f, 2.5247572e-15f});
    const uint16_t *perm = fr.perm;
    const uint64_t kj = key[je];
    const int lo[3] = {win_lo(fr, je, h0, n), win_lo(fr, je, h1, n), win_lo(fr, je, h2, n)};
    const int hw[3] = {h0, h1, h2};
    const float2 y2e = ydf[perm[je]];
    const df ye{y2e.x, y2e.y};
    df sw{0.f, 0.f}, sa = sw, sb = sw, sc = sw, sd = sw;
    df e[3];
    float fit[3];
    fit[2] = s2f;
    e[2] = df{g2f, 0.f};
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        const int hi = lo[k] + 2 * hw[k];
        // slots [ea, ea + na) and [eb, eb + nb): window 0, or ring k
        const int ea = lo[k], na = k ? lo[k - 1] - lo[k] : 2 * hw[0] + 1;
        const int eb = k ? lo[k - 1] + 2 * hw[k - 1] + 1 : 0, nb = k ? hi - (eb - 1) : 0;
        df aw{0.f, 0.f}, aa = aw, ab = aw, ac = aw, ad = aw;
#pragma unroll 2
        for (int v = (int)(threadIdx.x & 31); v < na + nb; v += 32) {
            const int e_ = v < na ? ea + v : eb + (v - na);
            int sh;
            const int p = slot_point(e_, n, sh);
            const uint32_t i = perm[p];
            const df dx = key_diff_df(key[p], kj, sh);
            const float2 w2 = wdf[i], y2 = ydf[i];
            const df w{w2.x, w2.y}, y{y2.x, y2.y};
            const df wdx = df_mul(w, dx);
            df_acc(aw, w);
            df_acc(aa, wdx);
            df_acc(ab, df_mul(wdx, dx));
            df_acc(ac, df_mul(w, y));
            df_acc(ad, df_mul(wdx, y));
        }
        df q[5] = {aw, aa, ab, ac, ad};
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            q[m] = x_two_sum(q[m].hi, q[m].lo);
#pragma unroll 1
            for (int o = 16; o > 0; o >>= 1) q[m] = acc_add(q[m], acc_shfl_xor(q[m], o));
        }
        sw = acc_add(sw, q[0]);
        sa = acc_add(sa, q[1]);
        sb = acc_add(sb, q[2]);
        sc = acc_add(sc, q[3]);
        sd = acc_add(sd, q[4]);
        // x about x_j: xbar - x_j = sa / sw; the fit at x_j
        const df xb = df_div(sa, sw);
        const df sxx = df_sub(sb, df_mul(xb, sa));
        df f = df_div(sc, sw);
        if (df_less(vsm, sxx)) f = df_sub(f, df_mul(df_div(df_sub(sd, df_mul(xb, sc)), sxx), xb));
        fit[k] = f.hi + f.lo;
        // generalized-validation residual |y_j - fit| / (1 - nu/m)
        const float m = u22f((uint32_t)(2 * hw[k] + 1));
        const df d = df_sub(df{1.f, 0.f}, df_div(df{((sl >> k) & 1) ? 2.f : 1.f, 0.f}, df{m, 0.f}));
        e[k] = df_div(df_abs(df_sub(ye, f)), d);
    }
    // the choice as Listing 1 takes it (first strict minimum; bass only below
    // the woofer's residual), on the double-float residuals
    df resmin{1.0e20f, 0.f};
    float s = K.s2;
    if (df_less(e[0], resmin)) { resmin = e[0]; s = K.s0; }
    if (df_less(e[1], resmin)) { resmin = e[1]; s = K.s1; }
    if (df_less(e[2], resmin)) { resmin = e[2]; s = K.s2; }
    if (K.bass && df_less(resmin, e[2]) && resmin.hi > 0.f) {
        float tmp = fdiv(resmin.hi, e[2].hi);
        if (tmp < 1.0e-7f) tmp = 1.0e-7f;
        const float pw = (K.ex == 1.f) ? tmp : span_pow(tmp, K.ex);
        s += (K.s2 - s) * pw;
    }
    return interpolate_span<float>(K, s, fit[0], fit[1], fit[2]);
}

// Where pass A leaves the three smooths for pass C: the frame's columns C0,
// C2, C4, or this CTA's part of the global slab (coalesced across a warp:
// every thread of a warp is at the same k of its chunk at the same time).
// SLAB false: always the frame columns (kernels for objects too short to use
// the slab carry no slab addressing).
template <typename R, bool SLAB>
struct SmoCols {
    R *slab;        // null: frame columns
    R *col[3];      // frame columns C0, C2, C4
    int kmax, G, nmax, tid, c0;
    __device__ inline R *at(int c, int i) const
    {
        if (!SLAB || !slab) return col[c] + i;
        const int k = i - c0;
        return k < kmax ? slab + ((size_t)(c * kmax + k) * G + tid)
                        : slab + (size_t)3 * kmax * G + (size_t)c * nmax + i;
    }
};

struct FreqResult {
    double chi2;
    bool near;   // FP32C: some decision fell within its margin
};

// Per-object constants of a work item, computed once per item so that the
// per-frequency code does no binary64 arithmetic on the FP32C path: Listing
// 1's window half widths (binary64 expressions), the span constants, the SS
// tweeter/midrange margin at this n, and the SP sensitivity budget.
template <typename R>
struct ObjK {
    int h0, h1, h2, hs;   // half widths of the three spans, and of the fixed span
    bool lim0, lim1;      // the tweeter's / midrange's window differs from the woofer's
    SpanK<R> K;
    // generalized-validation factors 1 / (1 - nu/m) of the three windows (m
    // points) for a line (nu = 2) and a constant (nu = 1)
    R gl0, gc0, gl1, gc1, gl2, gc2;

    float margin;         // SS: tweeter-vs-midrange margin, relative
    float margin_abs;     // and absolute (the residuals' FP32 error scale)
    R sens_lim, ymax;     // SP: chi2 budget per point, largest centred magnitude
};
template <typename R>
__device__ inline ObjK<R> obj_consts(const PgramArgs &a, int n, int obj)
{
    ObjK<R> k;
    k.h0 = half_width(n, a.spans[0]);
    k.h1 = half_width(n, a.spans[1]);
    k.h2 = half_width(n, a.spans[2]);
    k.hs = a.span > 0.0 ? half_width(n, a.span) : 0;
    k.lim0 = k.h0 != k.h2;
    k.lim1 = k.h1 != k.h2;
    const R m0 = (R)(2 * k.h0 + 1), m1 = (R)(2 * k.h1 + 1), m2 = (R)(2 * k.h2 + 1);
    k.gl0 = R(1) / (R(1) - R(2) / m0);
    k.gc0 = R(1) / (R(1) - R(1) / m0);
    k.gl1 = R(1) / (R(1) - R(2) / m1);
    k.gc1 = R(1) / (R(1) - R(1) / m1);
    k.gl2 = R(1) / (R(1) - R(2) / m2);
    k.gc2 = R(1) / (R(1) - R(1) / m2);
    k.K = span_consts<R>(a.spans, a.alpha);
    // both parts shrink with n as the effect of one flipped choice does
    const float shrink = fminf(1.f, 256.f / (float)n) * fminf(1.f, 512.f / (float)n);
    k.margin = n > kNearSSMaxN ? -1.f : a.near_ss * shrink;
    k.margin_abs = n > kNearSSMaxN ? -1.f : a.near_ss_abs * shrink * 1.1920929e-7f * (float)a.ymax[obj];
    k.sens_lim = (R)(a.sens_tau * a.chi0[obj]);
    k.ymax = (R)a.ymax[obj];
    return k;
}

// Sum of the threads' compensated chi2 sums and OR of their near flags, valid
// on thread 0 only (the one that stores the result).  One barrier.  FP32C
// combines the (sum, -compensation) pairs as double-float numbers with
// error-free additions on the FP32 pipe; thread 0 converts the total once.
// NQ sums at once (SPG scores three spans twice).
template <int NQ>
__device__ inline void block_reduce0(const KSum<float> (&k)[NQ], bool near, double *red, int *ired,
                                     double (&out)[NQ], bool &near0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    df v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        v[q] = df{k[q].s, -k[q].c};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const df y{__shfl_xor_sync(0xffffffffu, v[q].hi, o),
                       __shfl_xor_sync(0xffffffffu, v[q].lo, o)};
            v[q] = acc_add(v[q], y);
        }
    }
    const bool wn = __any_sync(0xffffffffu, near);
    float2 *rf = (float2 *)red;   // 32 slots
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) rf[q * 16 + warp] = make_float2(v[q].hi, v[q].lo);
        ired[warp] = wn ? 1 : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nr = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            df t{0.f, 0.f};
            for (int w = 0; w < nw; ++w) {
                const float2 e = rf[q * 16 + w];
                t = acc_add(t, df{e.x, e.y});
            }
            out[q] = (double)t.hi + (double)t.lo;
        }
        for (int w = 0; w < nw; ++w) nr |= ired[w];
        near0 = nr != 0;
    }
}
template <int NQ>
__device__ inline void block_reduce0(const KSum<double> (&k)[NQ], bool near, double *red, int *ired,
                                     double (&out)[NQ], bool &near0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        v[q] = k[q].value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    const bool wn = __any_sync(0xffffffffu, near);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[q * 16 + warp] = v[q];
        ired[warp] = wn ? 1 : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nr = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += red[q * 16 + w];
            out[q] = t;
        }
        for (int w = 0; w < nw; ++w) nr |= ired[w];
        near0 = nr != 0;
    }
}
template <typename R>
__device__ inline FreqResult chi2_result(const KSum<R> &chi2, bool near, double *red, int *ired)
{
    const KSum<R> k[1] = {chi2};
    double out[1] = {0.0};
    bool n0 = false;
    block_reduce0<1>(k, near, red, ired, out, n0);
    return FreqResult{out[0], n0};
}

// Listing 1's fixed-span mode: one running-line smooth of y with span
// a.span, no cross-validation, then chi2 (its own kernel variant).
template <typename R, typename A>
__device__ inline FreqResult fixed_span_pass(const ObjK<R> &ok, const Frame<R> &fr,
                                             const Small<R, A> &sm, int n, int c0, int c1, R o,
                                             R vsmlsq, bool ties, R rf)
{
    const int hs = ok.hs;
    const R *vy[1] = {fr.Y};
    KSum<R> chi2;
    bool near = false;
    build_xy_prefix(fr, sm, fr.Y, c0, c1, o);
    __syncthreads();
    if (c0 < c1) {
        Win<R, 1> w;
        win_init<R, 1>(w, fr, sm, vy, c0, hs, n, o);
        RunAvg<R, 1> ra;
        ra.reset(c0);
        auto emit = [&](int i, const R (&v)[1]) {
            const R d = fr.Y[i] - v[0];
            chi2.add(fr.XW[i].y * d * d);
        };
        for (int j = c0; j < c1; ++j) {
            Fit<R, 1> f1;
            win_fit_checked<R, 1>(f1, w, fr, vy, j, hs, n, o, vsmlsq, near, rf);
            const R val[1] = {f1.s[0]};
            run_push<R, 1>(ra, fr, j, ties, val, emit);
            if (j + 1 < c1) win_slide<R, 1>(w, fr, vy, j, hs, n, o);
        }
    }
    return chi2_result(chi2, near, sm.red, sm.ired);
}

// ---------------------------------------------------------------------------
// one (object, frequency)
// ---------------------------------------------------------------------------
// The result is valid on thread 0 only.
template <typename R, int VARIANT, bool LONG, typename A>
__device__ FreqResult process_frequency(const PgramArgs &a, const ObjK<R> &ok, int obj, int lead,
                                        int n, double f, const Frame<R> &fr, const Small<R, A> &sm,
                                        bool reuse)
{
    const int tid = threadIdx.x, G = blockDim.x;
    const int64_t base = a.off[obj];
    const R *yc = (const R *)a.yc + base;
    const R *wv = (const R *)a.wv + base;
    bool ties, flat;
    if (reuse) {
        // the group leader's sort holds: X, the tie bits and perm are those
        // of this object's identical times; only y and w are its own
        for (int j = tid; j < n; j += G) {
            const uint32_t i = fr.perm[j];
            fr.XW[j].y = wv[i];
            fr.Y[j] = yc[i];
        }
        __syncthreads();
        ties = sm.flags[0] != 0;
        flat = sm.flags[1] != 0;
    } else {
    const double *tt = a.tt + a.off[lead];

    // ---- fold and sort ----
    fold_and_sort(fr, n, sm, tt, f);

    // ---- gather ----
    // tie bits and the degenerate test use the exact fold output, so runs of
    // equal abscissae are those of the binary64 phases, whatever X rounds to
    int tie = 0;
    for (int j0 = tid - (tid & 31); j0 < n; j0 += G) {
        const int j = j0 + (tid & 31);
        bool tj = false;
        if (j < n) {
            const uint32_t i = fr.perm[j];
            const uint64_t kj = fr.key[j];
            const uint32_t kh = (uint32_t)(kj >> 32);
            R x;
            if (sizeof(R) == 8) {
                x = (R)fr.ph[i];
            } else {
                // X = the phase truncated to float.  From 2^-8 up, the top
                // word alone holds the float's 24 bits (its own truncation is
                // the same); only tiny phases need the 64-bit conversion.
                x = (R)key_to_float_rz(kj);
            }
            fr.XW[j] = vec2<R>(x, wv[i]);
            fr.Y[j] = yc[i];
            if (j + 1 < n) {
                tj = (sizeof(R) == 8) ? (fr.ph[i] == fr.ph[fr.perm[j + 1]])
                                      : (kj == fr.key[j + 1]);
            }
        }
        const uint32_t word = __ballot_sync(0xffffffffu, tj);
        if ((tid & 31) == 0) fr.tie[j0 >> 5] = word;
        tie |= tj;
    }
    ties = __syncthreads_or(tie) != 0;
    flat = (sizeof(R) == 8) ? !(fr.ph[fr.perm[n - 1]] > fr.ph[fr.perm[0]])
                            : (fr.key[n - 1] == fr.key[0]);
    if (tid == 0) {   // for the group's later objects
        sm.flags[0] = ties;
        sm.flags[1] = flat;
    }
    }

    // ---- degenerate abscissae: weighted mean (Listing 1) ----
    if (flat) {
        double sw = 0.0, swy = 0.0;
        for (int j = tid; j < n; j += G) {
            sw += (double)fr.XW[j].y;
            swy += (double)fr.XW[j].y * (double)fr.Y[j];
        }
        sw = block_sum(sw, sm.red);
        swy = block_sum(swy, sm.red);
        const R m = (R)(sw > 0.0 ? swy / sw : 0.0);
        double c2 = 0.0;
        for (int j = tid; j < n; j += G) {
            const double d = (double)(fr.Y[j] - m);
            c2 += (double)fr.XW[j].y * d * d;
        }
        return FreqResult{block_sum(c2, sm.red), false};
    }

    const int qi = n / 4 - 1, qj = 3 * (qi + 1) - 1;
    const R scale = fr.XW[qj].x - fr.XW[qi].x;
    const R vsmlsq = (R)1.0e-6 * scale * scale;
    const int h0 = ok.h0, h1 = ok.h1, h2 = ok.h2;
    const bool lim0 = ok.lim0, lim1 = ok.lim1;
    const SpanK<R> &K = ok.K;
    // the span constants in FP32, for the SP settle's continuous steps
    const SpanK<float> K32{(float)K.s0, (float)K.s1, (float)K.s2, (float)K.inv01,
                           (float)K.inv21, (float)K.ex, K.bass};

    // ---- chunks: contiguous centre ranges that never split a run of ties ----
    {
        int c = (int)((unsigned)(tid * n) >> (__ffs(G) - 1));   // floor(tid n / G), G a power of two
        if (ties)
            while (c > 0 && c < n && tie_next(fr, c - 1)) ++c;
        sm.cs[tid] = c;
        if (tid == 0) sm.cs[G] = n;
    }
    __syncthreads();
    const int c0 = sm.cs[tid], c1 = sm.cs[tid + 1];
    const R o = (c0 < c1) ? fr.XW[c0].x : R(0);

    KSum<R> chi2;
    bool near = false;
    const R rf = (R)a.refit_frac;

    if (VARIANT == VAR_FIXED)   // Listing 1's single smooth of y
        return fixed_span_pass<R, A>(ok, fr, sm, n, c0, c1, o, vsmlsq, ties, rf);

    if (VARIANT == VAR_SPG) {
        // Sec. 3, global generalized validation: three windows in one
        // sweep; each span scores sum w g^2 over the frequency and the least
        // score's smooth gives chi2
        const R *vy[1] = {fr.Y};
        build_xy_prefix(fr, sm, fr.Y, c0, c1, o);
        __syncthreads();
        KSum<R> gs[3], xs[3];
        if (c0 < c1) {
            Win<R, 1> w0, w1, w2;
            win_init<R, 1>(w0, fr, sm, vy, c0, h0, n, o);
            win_init<R, 1>(w1, fr, sm, vy, c0, h1, n, o);
            win_init<R, 1>(w2, fr, sm, vy, c0, h2, n, o);
            const R gl0 = ok.gl0, gc0 = ok.gc0, gl1 = ok.gl1, gc1 = ok.gc1, gl2 = ok.gl2, gc2 = ok.gc2;
            RunAvg<R, 3> ra;
            ra.reset(c0);
            auto emit = [&](int i, const R (&v)[3]) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const R d = fr.Y[i] - v[k];
                    xs[k].add(fr.XW[i].y * d * d);
                }
            };
            for (int j = c0; j < c1; ++j) {
                Fit<R, 1> f0, f1, f2;
                win_fit_checked<R, 1>(f0, w0, fr, vy, j, h0, n, o, vsmlsq, near, rf);
                win_fit_checked<R, 1>(f1, w1, fr, vy, j, h1, n, o, vsmlsq, near, rf);
                win_fit_checked<R, 1>(f2, w2, fr, vy, j, h2, n, o, vsmlsq, near, rf);
                const R yj = fr.Y[j], wj = fr.XW[j].y;
                const R g0 = fabs(yj - f0.s[0]) * (f0.slope ? gl0 : gc0);
                const R g1 = fabs(yj - f1.s[0]) * (f1.slope ? gl1 : gc1);
                const R g2 = fabs(yj - f2.s[0]) * (f2.slope ? gl2 : gc2);
                gs[0].add(wj * g0 * g0);
                gs[1].add(wj * g1 * g1);
                gs[2].add(wj * g2 * g2);
                const R val[3] = {f0.s[0], f1.s[0], f2.s[0]};
                run_push<R, 3>(ra, fr, j, ties, val, emit);
                if (j + 1 < c1) {
                    win_slide<R, 1>(w0, fr, vy, j, h0, n, o);
                    win_slide<R, 1>(w1, fr, vy, j, h1, n, o);
                    win_slide<R, 1>(w2, fr, vy, j, h2, n, o);
                }
            }
        }
        const KSum<R> all[6] = {gs[0], gs[1], gs[2], xs[0], xs[1], xs[2]};
        double tot[6] = {0, 0, 0, 0, 0, 0};
        bool n0 = false;
        block_reduce0<6>(all, near, sm.red, sm.ired, tot, n0);
        // thread 0 picks the span (the result is read on thread 0 only)
        int kbest = 0;
        for (int k = 1; k < 3; ++k)
            if (tot[k] < tot[kbest]) kbest = k;
        if (sizeof(R) == 4)
            for (int k = 0; k < 3; ++k)
                if (k != kbest && fabs(tot[k] - tot[kbest]) <= kNearSPG * fabs(tot[kbest])) n0 = true;
        return FreqResult{tot[3 + kbest], n0};
    }

    if (VARIANT == VAR_SP) {
        // one sweep, three windows on y, generalized validation (Sec. 3)
        const R *vy[1] = {fr.Y};
        build_xy_prefix(fr, sm, fr.Y, c0, c1, o);
        __syncthreads();
        const int lane = tid & 31;
        const int len = c1 - c0;
        // warp-uniform trip count: contested centres are settled by the warp
        const int kmax = __reduce_max_sync(0xffffffffu, len);
        Win<R, 1> w0, w1, w2;
        if (len > 0) {
            win_init<R, 1>(w0, fr, sm, vy, c0, h0, n, o);
            win_init<R, 1>(w1, fr, sm, vy, c0, h1, n, o);
            win_init<R, 1>(w2, fr, sm, vy, c0, h2, n, o);
        }
        // 1 / (1 - nu/m) for a line (nu = 2) and a constant (nu = 1)
        const R gl0 = ok.gl0, gc0 = ok.gc0, gl1 = ok.gl1, gc1 = ok.gc1, gl2 = ok.gl2, gc2 = ok.gc2;
        const float2 *y64 = a.ydf ? a.ydf + base : nullptr;
        const float2 *w64 = a.wdf ? a.wdf + base : nullptr;
        // a point whose bound E on its chi2 change exceeds this is refitted
        const R sens_lim = ok.sens_lim;
        const R ymax = ok.ymax;
        RunAvg<R, 1> ra;
        ra.reset(c0);
        auto emit = [&](int i, const R (&v)[1]) {
            const R d = fr.Y[i] - v[0];
            chi2.add(fr.XW[i].y * d * d);
        };
        for (int k = 0; k < kmax; ++k) {
            const bool act = k < len;
            const int j = c0 + k;
            R val[1] = {R(0)};
            bool contested = false;
            R s0 = R(0), s1 = R(0), s2 = R(0), g2 = R(0);
            bool sl0 = false, sl1 = false, sl2 = false;
            // the settle refits the woofer window too unless its FP32 fit is
            // enough: a near-tie settle whose minimum lies clearly below the
            // woofer's residual (bass enhancement and interpolation depend on
            // the woofer's fit continuously there)
            bool need2 = true;
            if (act) {
                Fit<R, 1> f0, f1, f2;
                win_fit_checked<R, 1>(f0, w0, fr, vy, j, h0, n, o, vsmlsq, near, rf);
                win_fit_checked<R, 1>(f1, w1, fr, vy, j, h1, n, o, vsmlsq, near, rf);
                win_fit_checked<R, 1>(f2, w2, fr, vy, j, h2, n, o, vsmlsq, near, rf);
                const R yj = fr.Y[j];
                s0 = f0.s[0];
                s1 = f1.s[0];
                s2 = f2.s[0];
                sl0 = f0.slope;
                sl1 = f1.slope;
                sl2 = f2.slope;
                const R g0 = fabs(yj - s0) * (f0.slope ? gl0 : gc0);
                const R g1 = fabs(yj - s1) * (f1.slope ? gl1 : gc1);
                g2 = fabs(yj - s2) * (f2.slope ? gl2 : gc2);
                const R sp = choose_span<R>(K, g0, g1, g2, g2, K.s2, lim0, lim1);
                val[0] = interpolate_span<R>(K, sp, s0, s1, s2);
                if (sizeof(R) == 4 && y64) {
                    const R scale = fmax(fmax(fabs(yj), fabs(s0)), fabs(s1));
                    // a tweeter/midrange near-tie: the window sums round at the
                    // magnitudes they slide over, which the object's largest
                    // centred magnitude bounds.  Settling the choice in binary64
                    // only matters if the other choice could move chi2 by more
                    // than the per-point budget: the smooth lies between the
                    // three fits, so it moves by at most their spread R, and
                    // w (y - v)^2 by at most w R (2 |y - v| + R).  A tie run
                    // spreads the change over its members: always settled.
                    if (fabs(g0 - g1) <= (R)a.near_sp * (R)1.1920929e-7 * fmax(scale, ymax)) {
                        const R rs = fmax(fmax(s0, s1), s2) - fmin(fmin(s0, s1), s2);
                        const bool in_run = ties && (tie_next(fr, j) || (j > 0 && tie_next(fr, j - 1)));
                        contested = in_run || fr.XW[j].y * rs * (R(2) * fabs(yj - val[0]) + rs) > sens_lim;
                        need2 = !(g2 - fmin(g0, g1) > (R)1e-4 * g2);
                    }
                    // bound on the power change from the FP32 error of the
                    // residuals through bass enhancement and interpolation:
                    // each residual's error is its slope times the rounding
                    // of X plus the sums' rounding at the magnitude scale
                    const R gm = fmin(g0, g1);
                    if (!contested && K.bass && gm < g2 && gm > R(0)) {
                        const R eps = (R)1.1920929e-7;
                        const R ul = (R)a.sens_ulps;
                        const R ge = (gm == g0) ? (fabs(f0.b[0]) * eps + ul * eps * scale) * (sl0 ? gl0 : gc0)
                                                : (fabs(f1.b[0]) * eps + ul * eps * scale) * (sl1 ? gl1 : gc1);
                        const R sc2 = fmax(fabs(yj), fabs(s2));
                        const R we = (fabs(f2.b[0]) * eps + ul * eps * sc2) * (sl2 ? gl2 : gc2);
                        const R tmp = gm / g2;
                        const R sk = (gm == g0) ? K.s0 : K.s1;
                        const R sp_ = sp;
                        const R dvds = (sp_ - K.s1 < R(0)) ? fabs(s0 - s1) * (-K.inv01)
                                                           : fabs(s2 - s1) * K.inv21;
                        const R E = R(2) * fr.XW[j].y * fabs(yj - val[0]) *
                                    ((K.s2 - sk) * dvds * tmp * (ge / gm + we / g2));
                        if (E > sens_lim) {
                            contested = true;
                            need2 = true;
                        }
                    }
                }
            }
            unsigned todo = __ballot_sync(0xffffffffu, contested);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int je = __shfl_sync(0xffffffffu, j, src);
                const int sl = __shfl_sync(0xffffffffu, (sl0 ? 1 : 0) | (sl1 ? 2 : 0) | (sl2 ? 4 : 0) |
                                                            (need2 ? 8 : 0), src);
                const float s2f = __shfl_sync(0xffffffffu, (float)s2, src);
                const float g2f = __shfl_sync(0xffffffffu, (float)g2, src);
                const float v = sp_settle<R>(fr, y64, w64, je, h0, h1, h2, n, qi, qj, sl, K32, s2f, g2f);
                if (lane == src) val[0] = (R)v;
            }
            if (act) {
                run_push<R, 1>(ra, fr, j, ties, val, emit);
                if (j + 1 < c1) {
                    win_slide<R, 1>(w0, fr, vy, j, h0, n, o);
                    win_slide<R, 1>(w1, fr, vy, j, h1, n, o);
                    win_slide<R, 1>(w2, fr, vy, j, h2, n, o);
                }
            }
        }
        return chi2_result(chi2, near, sm.red, sm.ired);
    }

    // ===== SS, Listing 1 =====
    SmoCols<R, LONG> smo;
    smo.slab = (LONG && a.smo) ? (R *)((unsigned char *)a.smo + (size_t)blockIdx.x * a.smo_stride)
                               : nullptr;
    smo.col[0] = fr.C[0];
    smo.col[1] = fr.C[2];
    smo.col[2] = fr.C[4];
    smo.kmax = a.smo_kmax;
    smo.G = G;
    smo.nmax = a.smo_nmax;
    smo.tid = tid;
    smo.c0 = c0;
    // pass A: the three spans on y with cross-validation.  C0/C2/C4 = smooths
    // (tweeter/midrange/woofer), C1/C3/C5 = CV residuals (-1 marks a centre
    // whose leverage reached 1; resolved below).
    {
        const R *vy[1] = {fr.Y};
        build_xy_prefix<R, !LONG>(fr, sm, fr.Y, c0, c1, o);
        __syncthreads();
        if (c0 < c1) {
            Win<R, 1> w0, w1, w2;
            win_init<R, 1, false, LONG>(w0, fr, sm, vy, c0, h0, n, o);
            win_init<R, 1, false, LONG>(w1, fr, sm, vy, c0, h1, n, o);
            win_init<R, 1, false, LONG>(w2, fr, sm, vy, c0, h2, n, o);
            RunAvg<R, 3> ra;
            ra.reset(c0);
            auto emit = [&](int i, const R (&v)[3]) {
                *smo.at(0, i) = v[0];
                *smo.at(1, i) = v[1];
                *smo.at(2, i) = v[2];
            };
            for (int j = c0; j < c1; ++j) {
                Fit<R, 1> f0, f1, f2;
                win_fit_checked<R, 1>(f0, w0, fr, vy, j, h0, n, o, vsmlsq, near, rf);
                win_fit_checked<R, 1>(f1, w1, fr, vy, j, h1, n, o, vsmlsq, near, rf);
                win_fit_checked<R, 1>(f2, w2, fr, vy, j, h2, n, o, vsmlsq, near, rf);
                const R yj = fr.Y[j], wj = fr.XW[j].y;
                R d0 = R(1) - wj * (f0.rW + f0.dxj * f0.dxj * f0.rS);
                R d1 = R(1) - wj * (f1.rW + f1.dxj * f1.dxj * f1.rS);
                R d2 = R(1) - wj * (f2.rW + f2.dxj * f2.dxj * f2.rS);
                if (sizeof(R) == 4 && fmin(fmin(fabs(d0), fabs(d1)), fabs(d2)) < (R)kNearLev)
                    near = true;
                if (sizeof(R) == 8) {
                    // 1 - w h near 0: its sliding-sum value carries the sums'
                    // history; refit that window in two passes, as the
                    // definition reads, before the leverage test below
                    if (d0 < R(1e-6)) cv_refit<R>(f0, d0, fr, vy, j, h0, n, vsmlsq, wj);
                    if (d1 < R(1e-6)) cv_refit<R>(f1, d1, fr, vy, j, h1, n, vsmlsq, wj);
                    if (d2 < R(1e-6)) cv_refit<R>(f2, d2, fr, vy, j, h2, n, vsmlsq, wj);
                }
                // Leverage 1 is decided exactly: the slope in use and every
                // other point of the window tied (only a clamped window's end
                // point can be alone so), where 1 - w h is rounding noise; or
                // 1 - w h rounding to 0 or below.  FP32C flags any 1 - w h
                // below kNearLev for the FP64 recompute as well.
                const bool l0 = ties && f0.slope && lev_one_end(fr, j, h0, n);
                const bool l1 = ties && f1.slope && lev_one_end(fr, j, h1, n);
                const bool l2 = ties && f2.slope && lev_one_end(fr, j, h2, n);
                fr.C[1][j] = (d0 > R(0) && !l0) ? fdiv(fabs(yj - f0.s[0]), d0) : R(-1);
                fr.C[3][j] = (d1 > R(0) && !l1) ? fdiv(fabs(yj - f1.s[0]), d1) : R(-1);
                fr.C[5][j] = (d2 > R(0) && !l2) ? fdiv(fabs(yj - f2.s[0]), d2) : R(-1);
                const R val[3] = {f0.s[0], f1.s[0], f2.s[0]};
                run_push<R, 3>(ra, fr, j, ties, val, emit);
                if (j + 1 < c1) {
                    win_slide<R, 1>(w0, fr, vy, j, h0, n, o);
                    win_slide<R, 1>(w1, fr, vy, j, h1, n, o);
                    win_slide<R, 1>(w2, fr, vy, j, h2, n, o);
                }
            }
        }
    }
    __syncthreads();

    // pass B: midrange smooth of the three residual columns (and, FP32C, of the
    // tweeter-minus-midrange difference), span choice with bass enhancement
    // -> C6
    {
        constexpr bool DIFF = sizeof(R) == 4;
        constexpr int NB = DIFF ? 4 : 3;
        const R *vr[3] = {fr.C[1], fr.C[3], fr.C[5]};
        const float margin = ok.margin, margin_abs = ok.margin_abs;
        // resolves the -1 residuals of pass A while it sums them
        build_channel_prefix<R, NB, DIFF, true, !LONG>(fr, sm, vr, c0, c1, o);
        __syncthreads();
        if (c0 < c1) {
            Win<R, NB> w1;
            win_init<R, NB, DIFF, LONG>(w1, fr, sm, vr, c0, h1, n, o);
            RunAvg<R, NB> ra;
            ra.reset(c0);
            auto emit = [&](int i, const R (&v)[NB]) {
                const R d01 = DIFF ? v[NB - 1] : v[0] - v[1];
                if (span_contested(d01, v[0], v[1], margin, margin_abs)) near = true;
                // when no residual is below 1e20 the span column keeps the
                // woofer's CV residual, as Listing 1's column 6 does
                fr.C[6][i] = choose_span<R>(K, v[0], v[1], v[2], v[2], fr.C[5][i], lim0, lim1,
                                            DIFF, d01);
            };
            for (int j = c0; j < c1; ++j) {
                Fit<R, NB> f1;
                win_fit_checked<R, NB, DIFF>(f1, w1, fr, vr, j, h1, n, o, vsmlsq, near, rf);
                R val[NB];
#pragma unroll
                for (int c = 0; c < NB; ++c) val[c] = f1.s[c];
                run_push<R, NB>(ra, fr, j, ties, val, emit);
                if (j + 1 < c1) win_slide<R, NB, DIFF>(w1, fr, vr, j, h1, n, o);
            }
        }
    }
    // No barrier here, nor after pass C: the next pass's prefix build reads
    // only this thread's own chunk, and its scan's barrier comes before any
    // thread reads another's columns or overwrites what this pass reads (the
    // barrier after pass A stays: its leverage-1 fix-up reads the previous
    // chunk).

    // pass C: midrange smooth of the chosen spans, clamp and interpolate -> C1
    {
        const R *vs[1] = {fr.C[6]};
        // LONG (smooths in the global slab, where they come from L2): pass A's
        // smooths at the next two centres are loaded ahead of their use, the
        // first two before the prefix scan, then each two centres before it
        // is interpolated
        R q0[3] = {R(0), R(0), R(0)}, q1[3] = {R(0), R(0), R(0)};
        if (LONG && c0 < c1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) q0[c] = *smo.at(c, c0);
            if (c0 + 1 < c1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) q1[c] = *smo.at(c, c0 + 1);
            }
        }
        build_channel_prefix<R, 1, false, false, !LONG>(fr, sm, vs, c0, c1, o);
        __syncthreads();
        if (c0 < c1) {
            Win<R, 1> w1;
            win_init<R, 1, false, LONG>(w1, fr, sm, vs, c0, h1, n, o);
            RunAvg<R, 1> ra;
            ra.reset(c0);
            auto emit = [&](int i, const R (&v)[1]) {
                fr.C[1][i] = interpolate_span<R>(K, v[0], *smo.at(0, i), *smo.at(1, i), *smo.at(2, i));
            };
            for (int j = c0; j < c1; ++j) {
                Fit<R, 1> f1;
                win_fit_checked<R, 1>(f1, w1, fr, vs, j, h1, n, o, vsmlsq, near, rf);
                if (LONG && !ties) {
                    fr.C[1][j] = interpolate_span<R>(K, f1.s[0], q0[0], q0[1], q0[2]);
                } else {
                    const R val[1] = {f1.s[0]};
                    run_push<R, 1>(ra, fr, j, ties, val, emit);
                }
                if (LONG) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) q0[c] = q1[c];
                    if (j + 2 < c1) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) q1[c] = *smo.at(c, j + 2);
                    }
                }
                if (j + 1 < c1) win_slide<R, 1>(w1, fr, vs, j, h1, n, o);
            }
        }
    }

    // pass D: final tweeter smooth and chi2
    {
        const R *vv[1] = {fr.C[1]};
        build_channel_prefix<R, 1, false, false, !LONG>(fr, sm, vv, c0, c1, o);
        __syncthreads();
        if (c0 < c1) {
            Win<R, 1> w0;
            win_init<R, 1, false, LONG>(w0, fr, sm, vv, c0, h0, n, o);
            RunAvg<R, 1> ra;
            ra.reset(c0);
            auto emit = [&](int i, const R (&v)[1]) {
                const R d = fr.Y[i] - v[0];
                chi2.add(fr.XW[i].y * d * d);
            };
            for (int j = c0; j < c1; ++j) {
                Fit<R, 1> f0;
                win_fit_checked<R, 1>(f0, w0, fr, vv, j, h0, n, o, vsmlsq, near, rf);
                const R val[1] = {f0.s[0]};
                run_push<R, 1>(ra, fr, j, ties, val, emit);
                if (j + 1 < c1) win_slide<R, 1>(w0, fr, vv, j, h0, n, o);
            }
        }
    }
    return chi2_result(chi2, near, sm.red, sm.ired);
}

// The binary64 recompute of one flagged SS frequency inside an FP32C kernel
// (long objects), on the binary64 inputs: the same code path, launch shape and
// therefore results as the separate recompute launch, but run by the CTA that
// flagged the frequency, right away.  Its FP64-pipe work then overlaps other
// CTAs' FP32 work instead of a launch of its own whose time is the latency of
// one frequency on one SM.  The frame lives in this CTA's global slab, the
// chunk table and prefixes in the shared region of the FP32 path (the same
// size: both accumulate in 8-byte numbers).  The chi2 is valid on thread 0.
template <bool PER>
__device__ __noinline__ double redo_ss_binary64(const PgramArgs a, int obj, int lead, int n, double f,
                                                unsigned char *smem, unsigned char *slab)
{
    Small<double, double> sm = carve_small<double, double>(smem, blockDim.x, VAR_SS);
    sm.dn = divn_make(n);
    Frame<double> fr = carve_frame<double>(slab, n, VAR_SS, false, false);
    fr.per = PER;
    PgramArgs b = a;
    b.yc = a.yc64;
    b.wv = a.wv64;
    b.smo = nullptr;
    const ObjK<double> ok = obj_consts<double>(b, n, obj);
    return process_frequency<double, VAR_SS, false, double>(b, ok, obj, lead, n, f, fr, sm, false).chi2;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// Persistent CTAs take work items (object, frequency range) from a counter.
// FP32C launches flag frequencies whose decisions came within their margins;
// the FP64 kernel's recompute launch then redoes exactly those frequencies
// and overwrites their (float) power.
// LONG: SS initialises its windows out of line (objects of many points)
template <typename R, int VARIANT, bool GMEM, bool PLAIN, bool PER, bool SHARED, bool LONG = false>
__global__ void __launch_bounds__(kMaxThreads) pgram_kernel(PgramArgs a)
{
    typedef typename AccSel<R, PLAIN>::T A;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item, s_redo;
    const int G = blockDim.x;
    Small<R, A> sm = carve_small<R, A>(smem, G, VARIANT);
    unsigned char *big = GMEM ? a.slab + (size_t)blockIdx.x * a.slab_bytes
                              : smem + align16(small_bytes<A>(G, VARIANT));
    if (threadIdx.x == 0) s_redo = 0;   // (the item fetch's barrier orders this)
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.item_counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= a.n_items) break;
        const int4 item = a.items[it];
        const int o = item.x;                 // first object of the item
        // SHARED: objects o..o+m-1 share their times, and with them each
        // frequency's fold and sort
        const int m = SHARED && item.w > 1 ? item.w : 1;
        const int n = (int)(a.off[o + 1] - a.off[o]);
        // only the kernels for long objects address the smooth slab; a shared
        // sort keeps its perm there, past the three smooth columns
        const bool smo_out = LONG && a.smo != nullptr;
        uint16_t *perm_slab =
            smo_out ? (uint16_t *)((unsigned char *)a.smo + (size_t)blockIdx.x * a.smo_stride +
                                   smo_bytes(a.smo_nmax, G, sizeof(R)))
                    : nullptr;
        Frame<R> fr = carve_frame<R>(big, n, VARIANT, SHARED, smo_out, perm_slab);
        sm.dn = divn_make(n);
        ObjK<R> ok = obj_consts<R>(a, n, o);
        fr.per = PER;
        // a frame in global memory still counts its sort buckets in shared
        // memory: the counting pass is one atomic per point
        if (GMEM && a.cnt_smem) fr.cnt = (uint32_t *)(smem + align16(small_bytes<A>(G, VARIANT)));
        for (int q = item.y; q < item.z; ++q) {
            bool sorted = false;
            for (int k = 0; k < m; ++k) {
                const int obj = o + k;
                const int64_t at = (int64_t)obj * a.n_freq + q;
                const bool bad = a.bad[obj] != 0;
                if (a.recompute && (bad || a.near[at] == 0)) continue;   // block-uniform
                double pw = 0.0;
                bool near = false;
                const double fq = a.freq[(a.fbase ? a.fbase[o] : 0) + q];
                if (bad) {
                    pw = __longlong_as_double(0x7ff8000000000000LL);
                } else {
                    if (SHARED && k > 0) ok = obj_consts<R>(a, n, obj);
                    const FreqResult r = process_frequency<R, VARIANT, LONG>(a, ok, obj, o, n, fq, fr,
                                                                             sm, SHARED && sorted);
                    sorted = true;
                    // the result is valid on thread 0, the one that stores it
                    if (threadIdx.x == 0) {
                        const double c0 = a.chi0[obj];
                        pw = (c0 > 0.0) ? 1.0 - r.chi2 / c0 : 0.0;
                        near = r.near;
                    }
                }
                constexpr bool kInline = LONG && VARIANT == VAR_SS && sizeof(R) == 4;
                const bool inl = kInline && a.redo_slab != nullptr;
                if (threadIdx.x == 0) {
                    if (a.power_f32) ((float *)a.power)[at] = (float)pw;
                    else ((double *)a.power)[at] = pw;
                    if (near && inl) s_redo = 1;
                    else if (near && a.near) a.near[at] = 1;
                }
                __syncthreads();
                if constexpr (kInline) {
                    if (inl && s_redo) {   // block-uniform
                        const double c2 = redo_ss_binary64<PER>(
                            a, obj, o, n, fq, smem, a.redo_slab + (size_t)blockIdx.x * a.redo_slab_bytes);
                        if (threadIdx.x == 0) {
                            const double c0 = a.chi0[obj];
                            ((float *)a.power)[at] = (float)((c0 > 0.0) ? 1.0 - c2 / c0 : 0.0);
                            s_redo = 0;
                        }
                        sorted = false;    // the recompute used the shared scratch
                        __syncthreads();
                    }
                }
            }
        }
    }
}

}  // namespace ssp
