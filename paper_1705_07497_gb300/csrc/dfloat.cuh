// Double-float ("float-float") helpers: a value is carried as an unevaluated
// sum hi + lo of two FP32 numbers (about 48 significant bits), and products
// of FP32 matrix entries with such values are accumulated with error-free
// transformations (Dekker/Knuth TwoProd via FMA and TwoSum).  This keeps the
// per-entry work of the solver's sparse products on the FP32 pipes while the
// result carries close to FP64 accuracy.
//
// Every operation below uses the explicit round-to-nearest intrinsics so the
// compiler cannot contract or reassociate them (that would break the
// error-free transformations).
#pragma once

#include <cuda_runtime.h>

namespace ct {

// (hi, lo) with hi = fp32(v), lo = fp32(v - hi).
__device__ __forceinline__ float2 split_f2(double v)
{
    const float hi = __double2float_rn(v);
    const float lo = __double2float_rn(__dsub_rn(v, (double)hi));
    return make_float2(hi, lo);
}

// s + c += a * (xh + xl), where a*xh is added exactly and a*xl in FP32.
__device__ __forceinline__ void df_fma(float& s, float& c, float a, float xh, float xl)
{
    const float ph = __fmul_rn(a, xh);
    const float pe = __fmaf_rn(a, xh, -ph);          // a*xh = ph + pe exactly
    const float t = __fadd_rn(s, ph);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(ph, bp));  // s + ph = t + e
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, __fmaf_rn(a, xl, pe)));
}

// s + c += (wh + wl) * (xh + xl): the product of two double-float values,
// with wh*xh exact and the cross terms in FP32.
__device__ __forceinline__ void df_fma2(float& s, float& c, float wh, float wl, float xh, float xl)
{
    const float ph = __fmul_rn(wh, xh);
    const float pe = __fmaf_rn(wh, xh, -ph);
    const float t = __fadd_rn(s, ph);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(ph, bp));
    s = t;
    const float cross = __fmaf_rn(wh, xl, __fmul_rn(wl, xh));
    c = __fadd_rn(c, __fadd_rn(e, __fadd_rn(pe, cross)));
}

__device__ __forceinline__ double df_value(float s, float c) { return (double)s + (double)c; }

}  // namespace ct
