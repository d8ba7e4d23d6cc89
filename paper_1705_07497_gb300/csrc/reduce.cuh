// Deterministic grid reductions and the conjugate-gradient scalar updates
// that follow them.  Per-thread and per-block sums are double-float (FP32
// pipes); only the grid totals and the CG scalars are FP64, computed by one
// thread and handed back to the kernels as double-float pairs.
#pragma once

#include "ct_internal.cuh"
#include "dfloat.cuh"

namespace ct {

// Reduces NQ per-thread double-float values over the block (fixed order),
// writes the block's partials, and lets the last block to finish sum all
// partials (fixed order).  Returns true in thread 0 of the last block, with
// the grid totals in tot[].  The counter is reset by the last block.
template <int NQ>
__device__ bool grid_reduce_last(const float2 (&v)[NQ], float2* partials, unsigned* counter,
                                 double (&tot)[NQ])
{
    __shared__ float2 sh[NQ][32];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float2 s = warp_sum_df(v[q]);
        if (lane == 0) sh[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float2 s = sh[q][0];
            for (int w = 1; w < nwarp; ++w) s = df_add(s, sh[q][w]);
            partials[(size_t)q * gridDim.x + blockIdx.x] = s;
        }
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float2 s = df_zero();
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            s = df_add(s, __ldcg(partials + (size_t)q * gridDim.x + b));
        s = warp_sum_df(s);
        if (lane == 0) sh[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float2 s = sh[q][0];
            for (int w = 1; w < nwarp; ++w) s = df_add(s, sh[q][w]);
            tot[q] = df_to_double(s);
        }
        *counter = 0u;
    }
    return threadIdx.x == 0;
}

// grid_reduce_last for a block of 128 threads in which every thread carries
// the values of two pixels of a 256-pixel tile: va of pixel slice 2w and vb of
// slice 2w + 1 (w its warp).  Every sum is grouped exactly as grid_reduce_last
// groups it in a block of 256 threads with one pixel per thread (warp sums
// per slice, slices in order, and the last block's partials summed by 256
// virtual threads t and t + 128), so both give the same bits.
template <int NQ>
__device__ bool grid_reduce_last_pair(const float2 (&va)[NQ], const float2 (&vb)[NQ], float2* partials,
                                      unsigned* counter, double (&tot)[NQ])
{
    __shared__ float2 sh[NQ][8];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float2 sa = warp_sum_df(va[q]);
        const float2 sb = warp_sum_df(vb[q]);
        if (lane == 0) {
            sh[q][2 * warp] = sa;
            sh[q][2 * warp + 1] = sb;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float2 s = sh[q][0];
            for (int w = 1; w < 8; ++w) s = df_add(s, sh[q][w]);
            partials[(size_t)q * gridDim.x + blockIdx.x] = s;
        }
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float2 s1 = df_zero(), s2 = df_zero();
        for (unsigned b = threadIdx.x; b < gridDim.x; b += 256)
            s1 = df_add(s1, __ldcg(partials + (size_t)q * gridDim.x + b));
        for (unsigned b = threadIdx.x + 128; b < gridDim.x; b += 256)
            s2 = df_add(s2, __ldcg(partials + (size_t)q * gridDim.x + b));
        s1 = warp_sum_df(s1);
        s2 = warp_sum_df(s2);
        if (lane == 0) {
            sh[q][warp] = s1;
            sh[q][warp + 4] = s2;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float2 s = sh[q][0];
            for (int w = 1; w < 8; ++w) s = df_add(s, sh[q][w]);
            tot[q] = df_to_double(s);
        }
        *counter = 0u;
    }
    return threadIdx.x == 0;
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// r0 = rhs - Op(u0) has been formed: start the iteration.
__device__ __forceinline__ void cg_after_residual(CgSlice& st, double rr, double rhs2, double tol)
{
    st.rr = rr;
    st.rhs2 = rhs2;
    st.iters = 0;
    st.alpha = 0.0;
    st.beta = 0.0;
    st.alpha_df = df_zero();
    st.beta_df = df_zero();
    st.status = CT_OK;
    if (!finite_d(rr) || !finite_d(rhs2)) {
        st.status = CT_ERR_NONFINITE;
        st.active = 0;
        return;
    }
    st.active = (rr > 0.0) && !(tol > 0.0 && sqrt(rr) <= tol * sqrt(rhs2));
}

// q = Op(p) and p.q are known: the step length.
__device__ __forceinline__ void cg_after_pq(CgSlice& st, double pq)
{
    if (!st.active) {
        st.alpha = 0.0;
        st.alpha_df = df_zero();
        return;
    }
    if (!finite_d(pq)) {
        st.status = CT_ERR_NONFINITE;
        st.active = 0;
        st.alpha = 0.0;
    } else if (!(pq > 0.0)) {
        st.status = CT_ERR_BREAKDOWN;
        st.active = 0;
        st.alpha = 0.0;
    } else {
        st.alpha = st.rr / pq;
    }
    st.alpha_df = df_from_double(st.alpha);
}

// u += alpha p, r -= alpha q done and r.r known: the new direction's beta.
__device__ __forceinline__ void cg_after_update(CgSlice& st, double rr_new, double tol)
{
    if (!st.active) {
        st.beta = 0.0;
        st.beta_df = df_zero();
        return;
    }
    st.iters += 1;
    st.beta = rr_new / st.rr;
    st.beta_df = df_from_double(st.beta);
    st.rr = rr_new;
    if (!finite_d(rr_new)) {
        st.status = CT_ERR_NONFINITE;
        st.active = 0;
    } else if (rr_new == 0.0 || (tol > 0.0 && sqrt(rr_new) <= tol * sqrt(st.rhs2))) {
        st.active = 0;
    }
}

// One Bregman update finished with ||u^{k+1} - u^k||_1 = upd.
__device__ __forceinline__ void sb_after_update(SbSlice& sb, double upd, double tol)
{
    if (sb.stopped) return;
    if (!finite_d(upd)) {
        sb.status = CT_ERR_NONFINITE;
        sb.stopped = 1;
        return;
    }
    if (sb.outer_done == 0) sb.first_upd = upd;
    sb.last_upd = upd;
    sb.outer_done += 1;
    if (tol > 0.0 && upd < tol * sb.first_upd) sb.stopped = 1;
}

}  // namespace ct
