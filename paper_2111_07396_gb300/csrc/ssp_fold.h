// ssp_fold.h -- the phase fold of Alg. 1 (computePhasedTime), phase =
// frac(tt * f), evaluated without the FP64 pipe.
//
// fold_fixed64 returns floor(frac(fl(tt * f)) * 2^64), where fl() is the
// binary64 product rounded to nearest even exactly as an IEEE multiply rounds
// it.  The 53-bit significands are multiplied as integers (exact 106-bit
// product), rounded to 53 bits, and the fraction bits below the binary point
// are returned as a 64-bit fixed-point number.  For every phase >= 2^-11 the
// result is the binary64 phase exactly (its bits all lie at or above 2^-64),
// so sort order and equality of phases are those of the binary64 fold.
// Products below 2^-64 (including every subnormal product) give 0.
//
// Host and device share this code, so the host entry point ssp_fold_fixed
// reproduces the kernels' fold bit for bit.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define SSP_HD __host__ __device__
#else
#define SSP_HD
#endif

namespace ssp {

SSP_HD inline uint64_t dbl_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

SSP_HD inline uint64_t mulhi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    const uint64_t a0 = a & 0xffffffffu, a1 = a >> 32, b0 = b & 0xffffffffu, b1 = b >> 32;
    const uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    const uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffu) + (p10 & 0xffffffffu);
    return p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
#endif
}

SSP_HD inline int clz64(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// tt >= 0 finite, f > 0 finite (the library validates both)
SSP_HD inline uint64_t fold_fixed64(double tt, double f)
{
    const uint64_t bt = dbl_bits(tt), bf = dbl_bits(f);
    int et = (int)((bt >> 52) & 0x7ff), ef = (int)((bf >> 52) & 0x7ff);
    uint64_t mt = bt & 0xfffffffffffffull, mf = bf & 0xfffffffffffffull;
    if (et == 0) {
        if (mt == 0) return 0;
        et = 1;
    } else {
        mt |= 1ull << 52;
    }
    if (ef == 0) ef = 1;
    else mf |= 1ull << 52;
    // tt * f = (mt * mf) * 2^q exactly
    const uint64_t lo = mt * mf, hi = mulhi64(mt, mf);
    int q = et + ef - 2 * 1075;
    const int nbits = hi ? 128 - clz64(hi) : 64 - clz64(lo);
    if (q + nbits <= -64) return 0;  // product below 2^-64
    // round the significand to 53 bits, nearest even
    uint64_t m;
    const int sh = nbits > 53 ? nbits - 53 : 0;
    if (sh == 0) {
        m = lo;
    } else {
        bool guard, sticky;
        if (sh >= 64) {
            m = hi >> (sh - 64);
            const int g = sh - 1;  // guard bit index in the 128-bit product
            guard = g >= 64 ? ((hi >> (g - 64)) & 1) : ((lo >> g) & 1);
            sticky = g >= 64 ? (lo != 0 || (hi & ((1ull << (g - 64)) - 1)) != 0)
                             : (lo & ((1ull << g) - 1)) != 0;
        } else {
            m = (hi << (64 - sh)) | (lo >> sh);
            guard = (lo >> (sh - 1)) & 1;
            sticky = sh >= 2 ? (lo & ((1ull << (sh - 1)) - 1)) != 0 : false;
        }
        if (guard && (sticky || (m & 1))) {
            ++m;
            if (m == (1ull << 53)) {
                m >>= 1;
                ++q;
            }
        }
        q += sh;
    }
    // value = m * 2^q; the fraction is the bits below 2^0
    if (q >= 0) return 0;
    const int fb = -q;  // fraction bits in m
    const uint64_t frac = fb >= 64 ? m : (m & ((1ull << fb) - 1));
    const int up = 64 - fb;  // position of m's lsb in the 64-bit fixed point
    if (up >= 0) return frac << up;
    if (up <= -64) return 0;
    return frac >> (-up);
}


// The trial frequency's part of the fold, taken apart once per frequency.
struct FoldFreq {
    double f;
    uint64_t mf;   // 53-bit significand with its leading bit
    int ef;        // biased exponent; 0 (a subnormal f) takes the general path
};

SSP_HD inline FoldFreq fold_freq(double f)
{
    const uint64_t bf = dbl_bits(f);
    FoldFreq r;
    r.f = f;
    r.ef = (int)((bf >> 52) & 0x7ff);
    r.mf = (bf & 0xfffffffffffffull) | (1ull << 52);
    return r;
}

// fold_fixed64 for a normal tt and a normal f with no data-dependent
// branches on the common path: both significands carry their leading bit, so
// the exact product lies in [2^104, 2^106) and the rounding point is one of
// two fixed bit positions.  The 64-bit fixed-point fraction of m 2^q is then
// (m 2^(q+64)) mod 2^64: the integer part shifts out.  Returns exactly what
// fold_fixed64 returns (zero and subnormal operands go through it).
SSP_HD inline uint64_t fold_fixed64_fast(double tt, const FoldFreq &F)
{
    const uint64_t bt = dbl_bits(tt);
    const int et = (int)(bt >> 52);   // tt >= 0: the sign bit is clear
    if (et == 0 || F.ef == 0) return bt == 0 ? 0 : fold_fixed64(tt, F.f);
    const uint64_t mt = (bt & 0xfffffffffffffull) | (1ull << 52);
    const uint64_t lo = mt * F.mf, hi = mulhi64(mt, F.mf);
    const int top = (int)(hi >> 41);   // bit 105 of the product
    const int sh = 52 + top;           // significant bits below the kept 53
    int q = et + F.ef - 2150;          // product = (hi:lo) 2^q
    if (q + sh + 53 <= -64) return 0;  // product below 2^-64
    uint64_t m = top ? ((hi << 11) | (lo >> 53)) : ((hi << 12) | (lo >> 52));
    const uint64_t g = top ? (1ull << 52) : (1ull << 51);
    const bool guard = (lo & g) != 0, sticky = (lo & (g - 1)) != 0;
    q += sh;
    if (guard && (sticky || (m & 1))) {
        ++m;
        if (m == (1ull << 53)) {
            m >>= 1;
            ++q;
        }
    }
    const int s = q + 64;
    if (s >= 64) return 0;
    if (s >= 0) return m << s;
    if (s <= -64) return 0;
    return m >> (-s);
}

}  // namespace ssp
