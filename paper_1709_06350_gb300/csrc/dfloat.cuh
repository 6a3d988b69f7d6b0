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

__device__ __forceinline__ df df_make(float hi, float lo) { return {hi, lo}; }

// a + b = s + e exactly (any magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// a + b = s + e exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    df r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    df r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a * 2^k for a power-of-two float factor (exact)
__device__ __forceinline__ df df_scale2(df a, float f) { return {a.hi * f, a.lo * f}; }

// double -> double-float (one FP64 subtraction)
__host__ __device__ __forceinline__ df df_from_double(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace recon
