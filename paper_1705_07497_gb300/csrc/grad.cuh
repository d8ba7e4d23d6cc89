// The adjoint of the forward-difference gradient on the tiled image layout
// (layout.cuh), in double-float arithmetic.  grad u = (u(i, j+1) - u(i, j),
// u(i+1, j) - u(i, j)) with the last difference zero (Neumann); grad^T below
// is its exact adjoint.
#pragma once

#include "dfloat.cuh"
#include "layout.cuh"

namespace ct {

// (grad^T (vx, vy)) at pixel (i, j), internal index t.
__device__ __forceinline__ float2 grad_adj_df(const float2* __restrict__ vx, const float2* __restrict__ vy,
                                              int64_t t, int i, int j, int n, int tn)
{
    float2 acc = df_zero();
    if (j >= 1) acc = df_add(acc, vx[tiled_index(i, j - 1, tn)]);
    if (j <= n - 2) acc = df_sub(acc, vx[t]);
    if (i >= 1) acc = df_add(acc, vy[tiled_index(i - 1, j, tn)]);
    if (i <= n - 2) acc = df_sub(acc, vy[t]);
    return acc;
}

}  // namespace ct
