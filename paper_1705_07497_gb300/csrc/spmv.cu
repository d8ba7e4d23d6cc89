// Stand-alone sparse products y = A x and x = A^T y in FP32 (ct_forward and
// ct_adjoint).  Sec. 2: the normal operator R* M* M R is the bottleneck of
// every iterative solver; Sec. 3 replaces it by precomputed sparse matrix
// products.  The solvers use the extended-precision variants of
// solver_ops.cu.
//
// Single-slice products (batch = 1) use one warp per CSR row: each lane
// streams 8 consecutive entries per step with two 16-byte column loads and
// one or two 16-byte value loads (evict-first, the matrix is read once per
// product), gathers x through the read-only path (x stays in L1/L2), and the
// warp finishes with a shuffle reduction.  Rows are padded to multiples of 8
// entries, so every vector load is aligned and no lane needs a bounds mask.
//
// Batched products (slices innermost, [len][B]) use one warp per row with
// each lane owning columns lane + 32 t of the row's output; the row's entries
// are read once and broadcast through shuffles.
#include "ct_internal.cuh"
#include "reduce.cuh"
#include "sparse_common.cuh"

namespace ct {
namespace {

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Dot product of one CSR row with a gathered vector (result in every lane).
template <typename VT, bool GS>
__device__ __forceinline__ float row_dot(const CsrView& m, const VT* __restrict__ val, int64_t row,
                                         const float* __restrict__ x, const float* __restrict__ gs,
                                         int lane)
{
    const int64_t s = m.rp[row], e = m.rp[row + 1];
    float acc = 0.0f;
    for (int64_t k = s + lane * 8; k < e; k += 256) {
        const int4 c0 = __ldcs(reinterpret_cast<const int4*>(m.col + k));
        const int4 c1 = __ldcs(reinterpret_cast<const int4*>(m.col + k + 4));
        float v[8];
        Vals<VT>::load8(val, k, v);
        const int c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            float xv = __ldg(x + c[t]);
            if (GS) xv *= __ldg(gs + c[t]);
            acc = fmaf(v[t], xv, acc);
        }
    }
    return warp_sum_f(acc);
}

struct StoreArgs {
    float* y;
    float scale;
    const float* row_scale;  // optional per-row output scale
    int rpow;                // 1: scale by s, 2: by s^2
    const int32_t* gate;     // skip when *gate != 0
    const CgSlice* cg;       // skip when !cg->active (batch 1 only)
};

template <typename VT, bool GS>
__global__ void __launch_bounds__(256) spmv_store_kernel(CsrView m, const VT* __restrict__ val,
                                                         const float* __restrict__ x,
                                                         const float* __restrict__ gs, StoreArgs a)
{
    if (a.gate && *a.gate) return;
    if (a.cg && !a.cg->active) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = warp; row < m.rows; row += nw) {
        const float acc = row_dot<VT, GS>(m, val, row, x, gs, lane);
        if (lane == 0) {
            float o = a.scale * acc;
            if (a.row_scale) {
                const float s = a.row_scale[row];
                o *= (a.rpow == 2 ? s * s : s);
            }
            a.y[row] = o;
        }
    }
}

// Batched product Y[row][b] = sum_k val_k X[col_k][b] (slices innermost).
template <typename VT, bool GS, int NB>
__global__ void __launch_bounds__(256) spmm_store_kernel(CsrView m, const VT* __restrict__ val,
                                                         const float* __restrict__ x,
                                                         const float* __restrict__ gs, int B,
                                                         StoreArgs a)
{
    if (a.gate && *a.gate) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int b0 = blockIdx.y * (32 * NB);
    for (int64_t row = warp; row < m.rows; row += nw) {
        float acc[NB];
#pragma unroll
        for (int t = 0; t < NB; ++t) acc[t] = 0.0f;
        const int64_t s = m.rp[row], e = m.rp[row + 1];
        for (int64_t k0 = s; k0 < e; k0 += 32) {
            const int64_t k = k0 + lane;
            int c = 0;
            float v = 0.0f;
            if (k < e) {
                c = __ldcs(m.col + k);
                v = Vals<VT>::one(val, k);
                if (GS) v *= __ldg(gs + c);
            }
            const int cnt = (e - k0) < 32 ? (int)(e - k0) : 32;
            for (int u = 0; u < cnt; ++u) {
                const int cu = __shfl_sync(0xffffffffu, c, u);
                const float vu = __shfl_sync(0xffffffffu, v, u);
                const float* xr = x + (int64_t)cu * B;
#pragma unroll
                for (int t = 0; t < NB; ++t) {
                    const int b = b0 + lane + 32 * t;
                    if (b < B) acc[t] = fmaf(vu, __ldg(xr + b), acc[t]);
                }
            }
        }
        float rs = a.scale;
        if (a.row_scale) {
            const float s2 = a.row_scale[row];
            rs *= (a.rpow == 2 ? s2 * s2 : s2);
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            const int b = b0 + lane + 32 * t;
            if (b < B) a.y[row * B + b] = rs * acc[t];
        }
    }
}

template <typename VT, bool GS>
int launch_store(const ct_matrix* M, const Csr& C, const VT* val, const float* x, float* y,
                 int32_t batch, const float* gs, StoreArgs a, cudaStream_t st)
{
    CsrView m{C.row_ptr, C.col, C.rows};
    a.y = y;
    if (batch == 1) {
        const int grid = grid_for(M, C.rows, 8, 8);
        spmv_store_kernel<VT, GS><<<grid, 256, 0, st>>>(m, val, x, gs, a);
    } else {
        const int nb = batch <= 32 ? 1 : batch <= 64 ? 2 : batch <= 128 ? 4 : 8;
        const int ycols = (batch + 32 * nb - 1) / (32 * nb);
        dim3 grid(grid_for(M, C.rows, 8, 8), ycols);
        switch (nb) {
        case 1: spmm_store_kernel<VT, GS, 1><<<grid, 256, 0, st>>>(m, val, x, gs, batch, a); break;
        case 2: spmm_store_kernel<VT, GS, 2><<<grid, 256, 0, st>>>(m, val, x, gs, batch, a); break;
        case 4: spmm_store_kernel<VT, GS, 4><<<grid, 256, 0, st>>>(m, val, x, gs, batch, a); break;
        default: spmm_store_kernel<VT, GS, 8><<<grid, 256, 0, st>>>(m, val, x, gs, batch, a); break;
        }
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

int grid_for(const ct_matrix* M, int64_t work_items, int items_per_block, int max_per_sm)
{
    int64_t g = (work_items + items_per_block - 1) / items_per_block;
    const int64_t cap = (int64_t)(M->sm_count > 0 ? M->sm_count : 148) * max_per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

int launch_forward(const ct_matrix* M, ValKind vk, const float* x, float* y, int32_t batch,
                   float out_scale, bool scale_sq, cudaStream_t st)
{
    if (batch == 1 && out_scale == 1.0f && !scale_sq) return launch_forward_f32(M, vk, x, y, st);
    StoreArgs a{};
    a.scale = out_scale;
    if (vk == ValKind::F16) {
        a.row_scale = M->row_scale;
        a.rpow = scale_sq ? 2 : 1;
        return launch_store<__half, false>(M, M->A, M->A.qval, x, y, batch, nullptr, a, st);
    }
    return launch_store<float, false>(M, M->A, M->A.val, x, y, batch, nullptr, a, st);
}

int launch_adjoint(const ct_matrix* M, ValKind vk, const float* y, float* x, int32_t batch,
                   float out_scale, bool scale_y, cudaStream_t st)
{
    if (batch == 1 && out_scale == 1.0f) {
        if (vk != ValKind::F16) return launch_adjoint_f32(M, vk, y, nullptr, x, st);
        // A^T y = Q^T (s .* y): form s .* y once in double-float, then the product
        ct_matrix* Mm = const_cast<ct_matrix*>(M);
        Workspace& w = Mm->ws;
        if (w.pub_y2_len < M->rows) {
            cudaFree(w.pub_y2);
            w.pub_y2 = nullptr;
            w.pub_y2_len = 0;
            CT_CUDA(cudaMalloc((void**)&w.pub_y2, (size_t)M->rows * sizeof(float2)));
            w.pub_y2_len = M->rows;
        }
        CT_CHECK(launch_to_df(M, y, M->row_scale, w.pub_y2, M->rows, st));
        return launch_adjoint_f32(M, vk, y, w.pub_y2, x, st);
    }
    StoreArgs a{};
    a.scale = out_scale;
    if (vk == ValKind::F16) {
        if (scale_y)
            return launch_store<__half, true>(M, M->At, M->At.qval, y, x, batch, M->row_scale, a, st);
        return launch_store<__half, false>(M, M->At, M->At.qval, y, x, batch, nullptr, a, st);
    }
    return launch_store<float, false>(M, M->At, M->At.val, y, x, batch, nullptr, a, st);
}

}  // namespace ct
