// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2),
// about 48 significant bits.  Sums use the error-free two-sum transformation (Knuth), products the
// FMA-based two-product (p = a*b, e = fma(a, b, -p) exactly), followed by renormalisation
// (Dekker's fast two-sum).  Everything runs on the FP32 units, which on this GPU have 64 times the
// FP64 throughput; the J/K kernels use it for the quartets that need FP64-class accuracy.
#pragma once
#include <cuda_runtime.h>

struct df32 {
    float hi, lo;
    __device__ __forceinline__ df32() {}
    __device__ __forceinline__ constexpr df32(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit df32(int v) : hi((float)v), lo(0.f) {}
    __device__ __forceinline__ explicit df32(float v) : hi(v), lo(0.f) {}
    __device__ __forceinline__ explicit df32(double v);   // after d2f_alu / f2d_alu
};

__device__ __forceinline__ df32 df_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return df32(s, b - (s - a));
}

__device__ __forceinline__ df32 df_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return df32(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ df32 operator+(df32 a, df32 b)
{
    df32 s = df_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df32 operator-(df32 a) { return df32(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }

__device__ __forceinline__ df32 operator*(df32 a, df32 b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df32 operator/(df32 a, df32 b)
{
    const float q1 = __fdividef(a.hi, b.hi);
    const df32 r = a - b * df32(q1, 0.f);
    const float q2 = __fdividef(r.hi, b.hi);
    return df_fast_two_sum(q1, q2);
}

__device__ __forceinline__ df32& operator+=(df32& a, df32 b) { a = a + b; return a; }
__device__ __forceinline__ df32& operator-=(df32& a, df32 b) { a = a - b; return a; }
__device__ __forceinline__ df32& operator*=(df32& a, df32 b) { a = a * b; return a; }
__device__ __forceinline__ bool operator!=(df32 a, df32 b) { return a.hi != b.hi || a.lo != b.lo; }
__device__ __forceinline__ bool operator<(df32 a, double b) { return a.hi < (float)b; }

// sqrt by one Newton correction of the FP32 root: s + (a - s^2) / (2 s)
__device__ __forceinline__ df32 df_sqrt(df32 a)
{
    if (a.hi <= 0.f) return df32(0.f, 0.f);
    const float s = sqrtf(a.hi);
    const df32 r = a - df32(s, 0.f) * df32(s, 0.f);
    return df_fast_two_sum(s, __fdividef(r.hi, 2.f * s));
}

__device__ __forceinline__ df32 df_shfl_xor(df32 v, int o)
{
    return df32(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

// element type of the density copy a J/K kernel of arithmetic type R reads (D itself for FP64,
// FP32-rounded for FP32, hi / lo pairs for double-float)
template <typename R> struct DElem { typedef double T; };
template <> struct DElem<float> { typedef float T; };
template <> struct DElem<df32> { typedef float2 T; };
