// Double-float ("float-float") arithmetic: a value is carried as an
// unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2 when
// normalised, about 48 significant bits).  Sums and products use the
// error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the
// FMA form of TwoProd, so every operation runs on the FP32 pipes.  On this
// part the FP64 pipe is a small fraction of the FP32 rate, and the solver
// needs far more than FP32 accuracy in its vectors (a fixed number of CG
// steps amplifies their rounding by orders of magnitude).
//
// Every operation uses the explicit round-to-nearest intrinsics so the
// compiler can neither contract nor reassociate them; that would break the
// error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace ct {

// ---- error-free transformations ------------------------------------------
// s + e == a + b exactly (any magnitudes).
__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return make_float2(s, e);
}

// s + e == a + b exactly, valid when |a| >= |b| (or a == 0).
__device__ __forceinline__ float2 fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return make_float2(s, e);
}

// p + e == a * b exactly (barring underflow).
__device__ __forceinline__ float2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return make_float2(p, e);
}

// ---- double-float arithmetic on float2 (x = hi, y = lo) ---------------------
__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    float2 s = two_sum(a.x, b.x);
    const float2 t = two_sum(a.y, b.y);
    s.y = __fadd_rn(s.y, t.x);
    s = fast_two_sum(s.x, s.y);
    s.y = __fadd_rn(s.y, t.y);
    return fast_two_sum(s.x, s.y);
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    float2 p = two_prod(a.x, b.x);
    p.y = __fmaf_rn(a.x, b.y, p.y);
    p.y = __fmaf_rn(a.y, b.x, p.y);
    return fast_two_sum(p.x, p.y);
}

// a * b for an FP32 b.
__device__ __forceinline__ float2 df_mul_f(float2 a, float b)
{
    float2 p = two_prod(a.x, b);
    p.y = __fmaf_rn(a.y, b, p.y);
    return fast_two_sum(p.x, p.y);
}

__device__ __forceinline__ float2 df_abs(float2 a) { return a.x < 0.0f ? df_neg(a) : a; }

// a > b for normalised values.
__device__ __forceinline__ bool df_gt(float2 a, float2 b)
{
    return a.x > b.x || (a.x == b.x && a.y > b.y);
}

__device__ __forceinline__ float2 df_zero() { return make_float2(0.0f, 0.0f); }

// ---- conversions -----------------------------------------------------------
__host__ __device__ inline float2 df_from_double(double v)
{
    const float hi = (float)v;
    const float lo = (float)(v - (double)hi);
    return make_float2(hi, lo);
}

__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// Nearest FP32 value of hi + lo.
__device__ __forceinline__ float df_to_float(float2 a) { return __fadd_rn(a.x, a.y); }

// ---- accumulation of FP32 products ------------------------------------------
// (s, c) is an unnormalised accumulator: s carries the running sum, c the
// collected rounding errors.  Adds a * (xh + xl) with a * xh exact.
__device__ __forceinline__ void acc_fma(float& s, float& c, float a, float2 x)
{
    const float2 p = two_prod(a, x.x);
    const float2 t = two_sum(s, p.x);
    s = t.x;
    c = __fadd_rn(c, __fadd_rn(t.y, __fmaf_rn(a, x.y, p.y)));
}

// Adds a double-float value to an accumulator.
__device__ __forceinline__ void acc_add(float& s, float& c, float2 v)
{
    const float2 t = two_sum(s, v.x);
    s = t.x;
    c = __fadd_rn(c, __fadd_rn(t.y, v.y));
}

__device__ __forceinline__ float2 acc_value(float s, float c) { return two_sum(s, c); }

// Warp-wide sum of double-float values (every lane gets the total).
__device__ __forceinline__ float2 warp_sum_df(float2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float2 w;
        w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = df_add(v, w);
    }
    return v;
}

}  // namespace ct
