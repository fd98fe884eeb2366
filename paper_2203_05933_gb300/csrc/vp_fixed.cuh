// Conversions between float64 and the fixed-point form of the correction apply
// (per-row values and per-group densities as integers of at most 52 bits, exact
// 128-bit sums), by integer operations on the bits: on GB300 the FP64 unit
// (2 lanes per clock per SM) would hold each such warp instruction for about 64
// cycles, while these take a few integer instructions.
#pragma once

#include <cuda_runtime.h>

namespace vp {

// x 2^(52-e) rounded to the nearest integer (ties away from zero), for |x| < 2^e
// and e >= -1021 (so |result| <= 2^52): x = M 2^(E'-1075) with the significand
// M (the implicit bit added for normal numbers) and E' = max(E, 1) for the
// biased exponent E, so the result is M 2^-sh, sh = 1023 + e - E' >= 1.
__device__ __forceinline__ long long fixed52(double x, int e)
{
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ff);
    long long M = b & 0xfffffffffffffLL;
    if (E) M |= 1LL << 52;
    const int sh = 1023 + e - (E > 1 ? E : 1);
    const long long q = sh >= 64 ? 0LL : (M + (1LL << (sh - 1))) >> sh;
    return b < 0 ? -q : q;
}

// The biased exponent field of x (0 for zeros and subnormals, 2047 for infinities
// and NaN); e = max(E, 1) - 1022 over a set of values bounds them all by 2^e.
__device__ __forceinline__ unsigned exponent_field(double x)
{
    return (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu;
}

// x 2^sh rounded to the nearest 128-bit integer (ties away from zero), for
// |x 2^sh| < 2^125: the significand shifted left, or right with rounding.
__device__ __forceinline__ __int128 fixed128(double x, int sh)
{
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ff);
    unsigned long long M = (unsigned long long)b & 0xfffffffffffffULL;
    if (E) M |= 1ULL << 52;
    const int t = (E > 1 ? E : 1) - 1075 + sh;  // x 2^sh = M 2^t, t <= 72 by the bound
    unsigned __int128 q;
    if (t >= 0) {
        q = (unsigned __int128)M << t;
    } else {
        const int r = -t;
        q = r >= 64 ? 0 : (unsigned __int128)((M + (1ULL << (r - 1))) >> r);
    }
    return b < 0 ? -(__int128)q : (__int128)q;
}

// t 2^s as float64 for a 128-bit two's-complement integer t, rounded to the
// nearest (ties away from zero): the magnitude's leading 53 bits, rounded, become
// the significand and s plus the shift the exponent field; results outside the
// normal range (overflow, subnormal) go through ldexp of the rounded significand.
__device__ __forceinline__ double int128_ldexp(__int128 t, int s)
{
    const bool neg = t < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
    if (a == 0) return 0.0;
    const unsigned long long ah = (unsigned long long)(a >> 64), al = (unsigned long long)a;
    const int n = ah ? 128 - __clzll((long long)ah) : 64 - __clzll((long long)al);  // bit length
    int sh = n - 53;
    unsigned long long mant;
    if (sh <= 0) {
        mant = al << (-sh);
    } else {
        mant = (unsigned long long)((a + ((unsigned __int128)1 << (sh - 1))) >> sh);
        if (mant >> 53) {  // rounded up to 2^53
            mant >>= 1;
            ++sh;
        }
    }
    const int E = sh + s + 1075;  // value = mant 2^(sh + s), mant in [2^52, 2^53)
    if (E >= 1 && E <= 2046)
        return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)E << 52) |
                                                (mant & 0xfffffffffffffULL)));
    return ldexp(neg ? -(double)mant : (double)mant, sh + s);
}

}  // namespace vp
