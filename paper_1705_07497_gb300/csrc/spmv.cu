// Stand-alone products y = A x and x = A^T y with FP32 vectors (ct_forward and
// ct_adjoint).  Sec. 2: the normal operator R* M* M R is the bottleneck of
// every iterative solver; Sec. 3 replaces it by precomputed sparse matrix
// products.  Both forms accumulate in double-float with the same kernels the
// solvers use: one warp per row for a single slice (solver_ops.cu), one warp
// per row and 32-slice chunk for a batch (batch.cu).
#include "ct_internal.cuh"
#include "dfloat.cuh"

namespace ct {
namespace {

// FP64 -> double-float, optionally times a per-row FP32 scale (index i / B).
__global__ void d2df_kernel(const double* __restrict__ in, const float* __restrict__ scale, float2* __restrict__ out,
                            int64_t len, int B)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double v = in[i];
        if (scale) v *= (double)scale[i / B];
        out[i] = df_from_double(v);
    }
}

__global__ void df2d_kernel(const float2* __restrict__ in, double* __restrict__ out, int64_t len)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = df_to_double(in[i]);
}

int ensure_buf(float2** buf, int64_t* len, int64_t need)
{
    if (*len >= need) return CT_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *len = 0;
    CT_CUDA(cudaMalloc((void**)buf, (size_t)need * sizeof(float2)));
    *len = need;
    return CT_OK;
}

// in (FP64, len_in) -> product -> out (FP64, len_out), through double-float buffers.
int product_f64(const ct_matrix* M, int which, const double* in, double* out, int32_t B, cudaStream_t st)
{
    ct_matrix* Mm = const_cast<ct_matrix*>(M);
    Workspace& w = Mm->ws;
    const int64_t nx = M->cols * B, ny = M->rows * B;
    CT_CHECK(ensure_buf(&w.pub_x2, &w.pub_x2_len, nx));
    CT_CHECK(ensure_buf(&w.pub_y2, &w.pub_y2_len, ny));
    float2* src = which == 0 ? w.pub_x2 : w.pub_y2;
    float2* dst = which == 0 ? w.pub_y2 : w.pub_x2;
    const int64_t lin = which == 0 ? nx : ny, lout = which == 0 ? ny : nx;
    const bool f16 = (M->flags & CT_VAL_FP16_ROWSCALE) != 0;
    d2df_kernel<<<grid_for(M, lin, 256, 8), 256, 0, st>>>(in, (which == 1 && f16) ? M->row_scale : nullptr, src,
                                                          lin, B);
    CT_CUDA(cudaGetLastError());
    if (B == 1) {
        if (which == 0)
            CT_CHECK(launch_forward_df(M, f16 ? ValKind::F16 : ValKind::F32, src, dst, 1, nullptr, nullptr, st));
        else
            CT_CHECK(launch_adjoint_df(M, f16 ? ValKind::F16 : ValKind::F32, src, dst, 1.0, st));
    } else {
        CT_CHECK(batched_product_df(M, which, src, dst, B, st));
    }
    df2d_kernel<<<grid_for(M, lout, 256, 8), 256, 0, st>>>(dst, out, lout);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

int launch_forward_f64(const ct_matrix* M, ValKind, const double* x, double* y, int32_t batch, cudaStream_t st)
{
    return product_f64(M, 0, x, y, batch, st);
}

int launch_adjoint_f64(const ct_matrix* M, ValKind, const double* y, double* x, int32_t batch, cudaStream_t st)
{
    return product_f64(M, 1, y, x, batch, st);
}

int grid_for(const ct_matrix* M, int64_t work_items, int items_per_block, int max_per_sm)
{
    int64_t g = (work_items + items_per_block - 1) / items_per_block;
    const int64_t cap = (int64_t)(M->sm_count > 0 ? M->sm_count : 148) * max_per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

int launch_forward(const ct_matrix* M, ValKind vk, const float* x, float* y, int32_t batch, cudaStream_t st)
{
    if (batch == 1) return launch_forward_f32(M, vk, x, y, st);
    return batched_forward_adjoint(M, 0, x, y, batch, st);
}

int launch_adjoint(const ct_matrix* M, ValKind vk, const float* y, float* x, int32_t batch, cudaStream_t st)
{
    if (batch != 1) return batched_forward_adjoint(M, 1, y, x, batch, st);
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

}  // namespace ct
