// dfloat.cuh -- double-float arithmetic: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2 (a 48-bit significand).
// Built from the error-free transformations of Knuth (TwoSum), Dekker
// (FastTwoSum) and the FMA product split (TwoProd), so every operation runs
// on the FP32 pipes; GB300's FP64 rate is 1/64 of its FP32 rate.
#pragma once

#include <cuda_runtime.h>

namespace recon {

struct df {
    float hi, lo;
};

__host__ __device__ __forceinline__ df df_make(float hi, float lo) { return {hi, lo}; }

// a + b = s + e exactly (any magnitudes).
__host__ __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// a + b = s + e exactly when |a| >= |b| (or a == 0).
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

__host__ __device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    df r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__host__ __device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__host__ __device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__host__ __device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    df r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a * b = p + e exactly (the FMA product split)
__host__ __device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = a * b;
    e = fmaf(a, b, -p);
}
// a * 2^k for a power-of-two float factor (exact)
__host__ __device__ __forceinline__ df df_scale2(df a, float f) { return {a.hi * f, a.lo * f}; }

// double -> double-float (one FP64 subtraction)
__host__ __device__ __forceinline__ df df_from_double(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}


// The same split as df_from_double, from the bit pattern with integer
// operations only (FP64 instructions, conversions included, issue at 1/64 of
// the FP32 rate; a split kernel spent its time waiting on them).  For
// 2^-40 <= |x| < 2^126: hi rounds the 52-bit fraction to 23 bits (nearest,
// ties to even; a carry into the exponent falls out of the integer addition),
// and x - hi = (r - inc 2^29) 2^(e - 1075) exactly, r the 29 dropped bits and
// inc the rounding increment, so lo is that integer rounded to a float once
// and scaled by a power of two (exact).  Bit-identical to df_from_double in
// that range; other x (zero, tiny, huge, non-finite) take df_from_double.
__host__ __device__ __forceinline__ unsigned long long df_dbits(double x)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long u;
    __builtin_memcpy(&u, &x, sizeof u);
    return u;
#endif
}
__host__ __device__ __forceinline__ float df_fbits(unsigned u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    __builtin_memcpy(&f, &u, sizeof f);
    return f;
#endif
}
// RN(d) for |d| <= 2^29 on the FP32 pipes (no integer-to-float conversion
// instruction): d = dh 2^14 + dl with 0 <= dl < 2^14; both parts are exact
// floats by the 1.5 * 2^23 bias trick, and one fma rounds their exact sum.
__host__ __device__ __forceinline__ float df_i2f(int d)
{
    const int dh = d >> 14, dl = d - dh * 16384;
    const float fh = df_fbits(0x4B400000u + (unsigned)dh) - 12582912.0f;
    const float fl = df_fbits(0x4B400000u + (unsigned)dl) - 12582912.0f;
    return fmaf(fh, 16384.0f, fl);
}

__host__ __device__ __forceinline__ double df_dfrombits(unsigned long long u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    __builtin_memcpy(&d, &u, sizeof d);
    return d;
#endif
}
#ifdef __CUDA_ARCH__
__device__ __noinline__ double df_f2d_ool(float x) { return (double)x; }
#else
inline double df_f2d_ool(float x) { return (double)x; }
#endif
// float -> double from the bit pattern (exact) with integer operations only:
// for a normal float the exponent is rebiased (127 -> 1023) and the 23-bit
// fraction widened to 52 bits; zeros keep their sign; subnormal, infinite and
// NaN floats take the conversion instruction, out of line.
__host__ __device__ __forceinline__ double df_f2d_bits(float x)
{
    unsigned u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(x);
#else
    __builtin_memcpy(&u, &x, sizeof u);
#endif
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (e - 1u >= 254u) {   // e == 0 or e == 255
        if ((u & 0x7FFFFFFFu) == 0u) return df_dfrombits(sign);
        return df_f2d_ool(x);
    }
    return df_dfrombits(sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29));
}
// hi + lo in FP64: both parts widened exactly, one FP64 addition
__host__ __device__ __forceinline__ double df_to_double_bits(df a) { return df_f2d_bits(a.hi) + df_f2d_bits(a.lo); }
// the FP64 split, out of line on the device so that the rare inputs outside
// the integer path's range take a real branch (an inlined copy was evaluated
// for every element and kept the FP64 pipe busy)
#ifdef __CUDA_ARCH__
__device__ __noinline__ df df_from_double_ool(double x) { return df_from_double(x); }
#else
inline df df_from_double_ool(double x) { return df_from_double(x); }
#endif
__host__ __device__ __forceinline__ df df_from_double_bits(double x)
{
    const unsigned long long u = df_dbits(x);
    const unsigned e = (unsigned)(u >> 52) & 0x7FFu;
    if (e < 1023u - 40u || e > 1023u + 125u) return df_from_double_ool(x);
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    const unsigned r = (unsigned)(m & 0x1FFFFFFFull);      // the 29 dropped bits
    const unsigned keep = (unsigned)(m >> 29);              // the 23 kept bits
    const unsigned inc = (r > 0x10000000u || (r == 0x10000000u && (keep & 1u))) ? 1u : 0u;
    const unsigned hbits = (((e - 1023u + 127u) << 23) | keep) + inc;
    const int d = (int)r - (int)(inc << 29);                 // |d| <= 2^28
    const float scale = df_fbits((e - 1075u + 127u) << 23);  // 2^(e - 1075), a normal float here
    // signed remainder (a zero remainder gives +0, as x - hi does in FP64)
    return {df_fbits(sign | hbits), df_i2f(sign ? -d : d) * scale};
}

}  // namespace recon
