// Double-float numbers: a value hi + lo held as two floats with |lo| at most
// half an ulp of hi, about 48 significant bits, computed on the FP32 pipes.
// GB300 runs FP32 arithmetic at 64 times its FP64 rate, so a recurrence step
// that FP64 arithmetic bounds becomes bound by its gathers again.
//
// The operations are the classical error-free transformations: Knuth's
// two-sum (the exact rounding error of a float sum), Dekker's fast two-sum
// for |a| >= |b|, and the two-product through a fused multiply-add, combined
// as in the double-float arithmetic of Dekker (1971).  Addition is the short
// form (the low parts added without their own error term): its error is about
// 2^-47 of the larger operand, an absolute error far below what the moment
// tolerances allow.
#pragma once

#include <cuda_runtime.h>

namespace mlt {

struct __align__(8) df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit constexpr df64(int v) : hi((float)v), lo(0.0f) {}
    // The nearest double-float to v (host or device; on the device it costs
    // FP64 conversions, so kernels convert their constants once).
    __host__ __device__ explicit df64(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ df64 df_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return df64(s, (a - (s - bb)) + (b - bb));
}

// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 operator+(df64 x, df64 y)
{
    const df64 s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ df64& operator+=(df64& x, df64 y)
{
    x = x + y;
    return x;
}

__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }

__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

// hi * hi exactly by the fused two-product, plus the cross terms.
__device__ __forceinline__ df64 operator*(df64 x, df64 y)
{
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}

// Running-sum addition with a deferred renormalisation: x.hi + y.hi is formed
// with its exact rounding error (Knuth's two-sum), the error and y.lo go into
// the low part, and the pair is left unnormalised (8 FP32 operations against
// 11 for the full sum).  After k such additions the low part carries k
// roundings of at most 2^-24 of itself, so a caller renormalises (df_norm)
// every few dozen terms; over 32 terms the deferred error stays below
// 2^-38 of the sum's magnitude.
__device__ __forceinline__ df64 df_add_lazy(df64 x, df64 y)
{
    const df64 s = df_two_sum(x.hi, y.hi);
    return df64(s.hi, x.lo + (s.lo + y.lo));
}

__device__ __forceinline__ df64 df_norm(df64 x) { return df_fast_two_sum(x.hi, x.lo); }

using ::fma;   // the float and double overloads stay visible beside this one
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }

__device__ __forceinline__ double df_to_double(df64 x) { return (double)x.hi + (double)x.lo; }

}  // namespace mlt
