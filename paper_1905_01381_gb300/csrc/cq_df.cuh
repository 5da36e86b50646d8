// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits, computed
// with FP32 instructions only.  On this GPU FP32 runs at 62x the FP64 rate,
// so a double-float operation (7-20 FP32 instructions) costs a fraction of
// an FP64 one.  The building blocks are the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum; Dekker, Numer. Math. 18, 224 (1971))
// and the FMA-based exact product; the compositions follow the "sloppy"
// double-word addition and the double-word products analysed by Joldes,
// Muller and Popescu (ACM TOMS 44, 2017).  The exponent range is FP32's.
#pragma once
#include <cuda_runtime.h>

namespace cq {

// the df overloads below must not hide the FP32/FP64 ones for code in cq
using ::fma;
using ::fmaf;

// The arithmetic compiles for the host too (a host program checks it
// against exact rational arithmetic); the shuffles and 1/sqrt are device
// code.

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.f) {}
    // nearest double-float of an FP64 value (two conversions and one FP64
    // subtraction; constant-folded for literal arguments)
    __host__ __device__ constexpr explicit df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__host__ __device__ __forceinline__ df df_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return df(s, (a - (s - bb)) + (b - bb));
}

__host__ __device__ __forceinline__ df df_fast_two_sum(float a, float b)   // |a| >= |b| or a == 0
{
    const float s = a + b;
    return df(s, b - (s - a));
}

__host__ __device__ __forceinline__ df operator+(df a, df b)
{
    const df s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__host__ __device__ __forceinline__ df operator*(df a, df b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return df_fast_two_sum(p, e);
}

// a * b + c with one renormalisation
__host__ __device__ __forceinline__ df fma(df a, df b, df c)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const df s = df_two_sum(p, c.hi);
    return df_fast_two_sum(s.hi, s.lo + (e + c.lo));
}

__host__ __device__ __forceinline__ df& operator+=(df& a, df b) { a = a + b; return a; }
__host__ __device__ __forceinline__ df& operator*=(df& a, df b) { a = a * b; return a; }
__host__ __device__ __forceinline__ bool operator<(df a, float b) { return a.hi < b || (a.hi == b && a.lo < 0.f); }

// warp shuffles of a double-float (both words)
__device__ __forceinline__ df shfl_down_r(df v, int o)
{
    return df(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ df shfl_xor_r(df v, int o)
{
    return df(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ float shfl_down_r(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down_r(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_xor_r(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor_r(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }

// 1/sqrt(x), x > 0: FP32 estimate and one Newton step in double-float,
// r <- r + r (1 - x r^2) / 2
__device__ __forceinline__ df rsqrt_r(df x)
{
    const float r0 = rsqrtf(x.hi);
    const df r(r0, 0.f);
    const df t = fma(-x, r * r, df(1.f, 0.f));     // 1 - x r0^2 (small)
    return fma(r * df(0.5f, 0.f), t, r);
}

// 1/x: FP32 estimate and one Newton step, r <- r + r (1 - x r)
__host__ __device__ __forceinline__ df recip(df x)
{
    const float r0 = 1.0f / x.hi;
    const df r(r0, 0.f);
    const df t = fma(-x, r, df(1.f, 0.f));
    return fma(r, t, r);
}

// sqrt(x), x > 0: s <- s + (x - s^2) / (2 s)
__host__ __device__ __forceinline__ df sqrt_df(df x)
{
    const float s0 = sqrtf(x.hi);
    const df s(s0, 0.f);
    const df t = fma(-s, s, x);
    return fma(t, df(0.5f / s0, 0.f), s);
}

}  // namespace cq
