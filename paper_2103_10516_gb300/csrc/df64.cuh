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

#include <cstdint>

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

// Packed FP32 pairs: two FP32 values in one 64-bit register (the first in the
// low half), operated on by one f32x2 instruction, round to nearest.  GB300
// issues each of these once for both values.
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t neg2(uint64_t a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ uint64_t pack2(float a, float b)
{
    return (uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32);
}
__device__ __forceinline__ float lo_half(uint64_t x) { return __uint_as_float((unsigned)x); }
__device__ __forceinline__ float hi_half(uint64_t x) { return __uint_as_float((unsigned)(x >> 32)); }

// Two double-float numbers side by side: h holds their high parts, l their
// low parts.  Each operation below is the df64 operation of the same name
// applied to both numbers, step for step with the same roundings, so its
// results are those of two scalar calls bit for bit.
struct df2 {
    uint64_t h, l;
};

__device__ __forceinline__ df2 df2_of(df64 x0, df64 x1) { return df2{pack2(x0.hi, x1.hi), pack2(x0.lo, x1.lo)}; }
__device__ __forceinline__ df64 df2_first(df2 x) { return df64(lo_half(x.h), lo_half(x.l)); }
__device__ __forceinline__ df64 df2_second(df2 x) { return df64(hi_half(x.h), hi_half(x.l)); }

__device__ __forceinline__ df2 df2_fast_two_sum(uint64_t a, uint64_t b)
{
    const uint64_t s = add2(a, b);
    return df2{s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ df2 operator+(df2 x, df2 y)
{
    const uint64_t s = add2(x.h, y.h);
    const uint64_t bb = sub2(s, x.h);
    const uint64_t e = add2(sub2(x.h, sub2(s, bb)), sub2(y.h, bb));
    return df2_fast_two_sum(s, add2(e, add2(x.l, y.l)));
}

__device__ __forceinline__ df2 operator-(df2 x) { return df2{neg2(x.h), neg2(x.l)}; }

__device__ __forceinline__ df2 operator*(df2 x, df2 y)
{
    const uint64_t p = mul2(x.h, y.h);
    uint64_t e = fma2(x.h, y.h, neg2(p));
    e = fma2(x.h, y.l, e);
    e = fma2(x.l, y.h, e);
    return df2_fast_two_sum(p, e);
}

// 2x, exactly (both parts doubled).
__device__ __forceinline__ df2 df2_twice(df2 x) { return df2{add2(x.h, x.h), add2(x.l, x.l)}; }

}  // namespace mlt
