// Epilogue shared by the kernels that end a CG operator product
// Op(p) = c_id p + c_ata N(p) + c_grad grad^T grad p (Eqs. KKT, PD_resolve,
// SB_solve): given N(p) at one pixel it forms Op(p), writes the CG vector of
// the epilogue's mode and accumulates the grid-wide dot products, which the
// last block finishes into the slice's CG scalars.
#pragma once

#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "grad.cuh"
#include "layout.cuh"
#include "reduce.cuh"

namespace ct {

// (grad^T grad u) at pixel (i, j), Neumann forward differences, tiled layout.
__device__ __forceinline__ float2 lap_df(const float2* __restrict__ u, int64_t t, int i, int j, int n, int tn)
{
    const float2 c = u[t];
    float2 acc = df_zero();
    if (j > 0) acc = df_add(acc, df_sub(c, u[tiled_index(i, j - 1, tn)]));
    if (j < n - 1) acc = df_add(acc, df_sub(c, u[tiled_index(i, j + 1, tn)]));
    if (i > 0) acc = df_add(acc, df_sub(c, u[tiled_index(i - 1, j, tn)]));
    if (i < n - 1) acc = df_add(acc, df_sub(c, u[tiled_index(i + 1, j, tn)]));
    return acc;
}

// Per-pixel epilogue.  MODE 1: q = Op(p), accumulate p.q.  MODE 2: r = rhs -
// Op(u), p = r, accumulate r.r and rhs.rhs.  MODE 3: r = rhs - Op(u), r.r.
template <int MODE>
__device__ __forceinline__ void op_epilogue(const OpEpilogue& a, int n, int tn, int64_t t, int i, int j,
                                            float2 nacc, float& s0, float& c0, float& s1, float& c1)
{
    const float2 in = a.in[t];
    float2 op = df_mul(a.c_ata, nacc);
    op = df_add(op, df_mul(a.c_grad, lap_df(a.in, t, i, j, n, tn)));
    op = df_add(op, df_mul(a.c_id, in));
    if (MODE == 1) {
        a.out[t] = op;
        acc_add(s0, c0, df_mul(in, op));
    } else {
        const float2 rhs =
            a.rhs ? a.rhs[t] : df_add(a.atf[t], df_mul(a.lam, grad_adj_df(a.vx, a.vy, t, i, j, n, tn)));
        const float2 r = df_sub(rhs, op);
        a.out[t] = r;
        if (MODE == 2) a.p_out[t] = r;
        acc_add(s0, c0, df_mul(r, r));
        acc_add(s1, c1, df_mul(rhs, rhs));
    }
}

template <int MODE>
__device__ __forceinline__ void op_finish(const OpEpilogue& a, float s0, float c0, float s1, float c1)
{
    float2 v[2] = {acc_value(s0, c0), acc_value(s1, c1)};
    double tot[2];
    if (grid_reduce_last<2>(v, a.partials, a.counter, tot)) {
        if (MODE == 1) cg_after_pq(*a.cg, tot[0]);
        if (MODE == 2) cg_after_residual(*a.cg, tot[0], tot[1], a.tol);
        if (MODE == 3) a.cg->rr = tot[0];
    }
}

}  // namespace ct
