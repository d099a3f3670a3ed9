// Conversions of FP64 values by integer instructions.
//
// The FP64 pipe of this GPU issues at 1/64 of the FP32 rate, so a kernel that streams particles and
// spends a handful of FP64 instructions on each one (a range check, a quantisation, a rounding to
// single precision) is bound by that pipe rather than by memory.  The functions below give the same
// results bit for bit from the IEEE-754 encodings, with integer and FP32 instructions only, and fall
// back to the FP64 instruction for the rare operands outside their fast range (zero, subnormal or
// tiny values, infinities, NaN).  Host builds use the same code, so it can be checked on the CPU
// against the compiler's own conversions.
#pragma once

#include <stdint.h>
#include <string.h>

__host__ __device__ __forceinline__ unsigned long long fmm_dbits(double x)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

__host__ __device__ __forceinline__ float fmm_fbits(unsigned int b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
#endif
}

__host__ __device__ __forceinline__ float fmm_d2f_slow(double x)
{
#ifdef __CUDA_ARCH__
    return __double2float_rn(x);
#else
    return (float)x;  // round to nearest even, the host default
#endif
}

// x in [0, 1), with -0.0 counted as 0 (the comparison 0 <= x < 1 of the FP64 value).
__host__ __device__ __forceinline__ bool fmm_in_unit(double x)
{
    const unsigned long long u = fmm_dbits(x);
    return (u >> 63) ? (u << 1) == 0ull : (u >> 52) < 1023ull;
}

// floor(x * 2^21) clamped to [0, 2^21 - 1]; 0 for negative values and NaN, 2^21 - 1 for x >= 1.
// x = m 2^(e - 1075) with m the 53-bit significand, so x 2^21 = m 2^(e - 1054) and the floor is a
// right shift by 1054 - e, which lies in [32, 52] for 2^-21 <= x < 1.
__host__ __device__ __forceinline__ unsigned int fmm_quantise21(double x)
{
    const unsigned long long u = fmm_dbits(x);
    if (u >> 63) return 0u;
    const unsigned int e = (unsigned int)(u >> 52);
    if (e >= 1023u) return (e == 2047u && (u << 12) != 0ull) ? 0u : 2097151u;
    if (e < 1002u) return 0u;
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    return (unsigned int)(m >> (1054u - e));
}

// Round to nearest even of a double to single precision (__double2float_rn).  For a biased exponent
// e in [897, 1150] the result is a normal float: keep the top 23 of the 52 fraction bits, round on
// the 29 dropped ones, and let a carry out of the fraction raise the exponent (to infinity past the
// largest float, as rounding does).
__host__ __device__ __forceinline__ float fmm_d2f_rn(double x)
{
    const unsigned long long u = fmm_dbits(x);
    const unsigned int e = (unsigned int)(u >> 52) & 0x7ffu;
    if (e - 897u > 253u) return (u << 1) == 0ull ? fmm_fbits((unsigned int)(u >> 32)) : fmm_d2f_slow(x);  // +-0 exactly
    const unsigned int t = (unsigned int)((u >> 29) & 0x7FFFFFull);
    const unsigned int r = (unsigned int)u & 0x1FFFFFFFu;
    const unsigned int up = (r > 0x10000000u) | ((r == 0x10000000u) & t);
    const unsigned int b = ((e - 896u) << 23) + t + up;
    return fmm_fbits(b | ((unsigned int)(u >> 32) & 0x80000000u));
}

// The float pair of a double: h = fl(x) and l = fl(x - h), as __double2float_rn(x) and
// __double2float_rn(x - (double)h) give them (x - h is exact in FP64).  With x = m 2^(e - 1075),
// x - h = D 2^(e - 1075) where D is the 29 dropped fraction bits, less 2^29 when h rounded up, so
// |D| <= 2^28; D is rounded to 24 bits in integers and placed at its exponent.  For e >= 949 that
// exponent stays in the normal range whatever D is; smaller or non-finite values take the FP64 path.
__host__ __device__ __forceinline__ void fmm_split_f32(double x, float& h, float& l)
{
    const unsigned long long u = fmm_dbits(x);
    const unsigned int e = (unsigned int)(u >> 52) & 0x7ffu;
    if (e - 949u > 201u) {
        h = fmm_d2f_slow(x);
        l = fmm_d2f_slow(x - (double)h);
        return;
    }
    const unsigned int sx = (unsigned int)(u >> 32) & 0x80000000u;
    const unsigned int t = (unsigned int)((u >> 29) & 0x7FFFFFull);
    const unsigned int r = (unsigned int)u & 0x1FFFFFFFu;
    const unsigned int up = (r > 0x10000000u) | ((r == 0x10000000u) & t);
    h = fmm_fbits((((e - 896u) << 23) + t + up) | sx);
    // D = r - up 2^29: magnitude a, negative (opposite to x) when h rounded away from zero
    const unsigned int a = up ? 0x20000000u - r : r;
    if (a == 0u) {
        l = 0.0f;  // x - h is an exact +0 in round to nearest
        return;
    }
    const unsigned int sl = up ? (sx ^ 0x80000000u) : sx;
#ifdef __CUDA_ARCH__
    const int nb = 32 - __clz(a);
#else
    const int nb = 32 - __builtin_clz(a);
#endif
    unsigned int tt;
    if (nb <= 24) {
        tt = a << (24 - nb);
    } else {
        const int sh = nb - 24;
        tt = a >> sh;
        const unsigned int rr = a & ((1u << sh) - 1u), half = 1u << (sh - 1);
        tt += (rr > half) | ((rr == half) & tt);
    }
    // value tt 2^(E - 23) with E = nb - 1 + e - 1075; the hidden bit of tt adds one to the exponent
    // field, a rounding carry to 2^24 one more
    const unsigned int ef = (unsigned int)(nb - 1 + (int)e - 1075 + 126);
    l = fmm_fbits(((ef << 23) + tt) | sl);
}

__host__ __device__ __forceinline__ double fmm_dfrom(unsigned long long u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, sizeof d);
    return d;
#endif
}

// The exact widening of a float to double ((double)f): a normal float's exponent is re-biased by
// 1023 - 127 = 896 and its 23 fraction bits move up by 29; zeros, subnormals, infinities and NaN take
// the conversion instruction.
__host__ __device__ __forceinline__ double fmm_f2d(float f)
{
#ifdef __CUDA_ARCH__
    const unsigned int u = __float_as_uint(f);
#else
    unsigned int u;
    memcpy(&u, &f, sizeof u);
#endif
    const unsigned int e = (u >> 23) & 0xffu;
    if (e - 1u > 253u) return (u << 1) == 0u ? fmm_dfrom((unsigned long long)u << 32) : (double)f;  // +-0 exactly
    return fmm_dfrom(((unsigned long long)(u & 0x80000000u) << 32) | ((unsigned long long)(e + 896u) << 52) |
                     ((unsigned long long)(u & 0x7FFFFFu) << 29));
}

// Order key of a double in [0, inf) for integer minimum and maximum: its bits, with -0.0 taken as
// +0.0 (numerically equal).  fmm_dfrom of the key gives the value back.
__host__ __device__ __forceinline__ unsigned long long fmm_nonneg_key(double x)
{
    const unsigned long long u = fmm_dbits(x);
    return (u << 1) == 0ull ? 0ull : u;
}
