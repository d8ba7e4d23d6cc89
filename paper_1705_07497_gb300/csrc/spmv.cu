// Stand-alone products y = A x and x = A^T y with FP32 vectors (ct_forward and
// ct_adjoint).  Sec. 2: the normal operator R* M* M R is the bottleneck of
// every iterative solver; Sec. 3 replaces it by precomputed sparse matrix
// products.  Both forms accumulate in double-float with the same kernels the
// solvers use: one warp per row for a single slice (solver_ops.cu), one warp
// per row and 32-slice chunk for a batch (batch.cu).
#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "sparse_common.cuh"

namespace ct {
namespace {

// FP64-vector products for the differentiable path: FP64 gathers and FP64
// accumulation (one FMA per entry on the FP64 pipe).  The derivative of the
// unrolled reconstruction amplifies rounding far more than the reconstruction
// itself, so this path trades speed for FP64 accuracy; the solvers use the
// double-float kernels.
template <typename VT>
__device__ __forceinline__ double val64(const VT* v, int64_t k);
template <>
__device__ __forceinline__ double val64<float>(const float* v, int64_t k) { return (double)__ldg(v + k); }
template <>
__device__ __forceinline__ double val64<__half>(const __half* v, int64_t k)
{
    return (double)__half2float(v[k]);
}

// B == 1: one warp per row, lanes interleaved over the entries.
template <typename VT>
__global__ void __launch_bounds__(256) csr_f64_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      const VT* __restrict__ val, int64_t rows,
                                                      const double* __restrict__ x, double* __restrict__ y,
                                                      const float* __restrict__ row_scale,
                                                      const float* __restrict__ in_scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = warp; row < rows; row += nw) {
        double acc = 0.0;
        for (int64_t k = rp[row] + lane; k < rp[row + 1]; k += 32) {
            const int c = __ldg(col + k);
            double xv = __ldg(x + c);
            if (in_scale) xv *= (double)__ldg(in_scale + c);
            acc = fma(val64<VT>(val, k), xv, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[row] = row_scale ? acc * (double)row_scale[row] : acc;
    }
}

// B > 1: one warp per (row, 32-slice chunk), lane = slice.
template <typename VT>
__global__ void __launch_bounds__(256) spmm_f64_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                       const VT* __restrict__ val, int64_t rows,
                                                       const double* __restrict__ x, double* __restrict__ y, int B,
                                                       const float* __restrict__ row_scale,
                                                       const float* __restrict__ in_scale)
{
    const int lane = threadIdx.x & 31;
    const int chunks = (B + 31) / 32;
    const int64_t task0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t ntask = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t task = task0; task < rows * chunks; task += ntask) {
        const int64_t row = task / chunks;
        const int b = (int)(task % chunks) * 32 + lane;
        if (b >= B) continue;
        double acc = 0.0;
        for (int64_t k = rp[row]; k < rp[row + 1]; ++k) {
            const int c = __ldg(col + k);
            double xv = __ldg(x + (int64_t)c * B + b);
            if (in_scale) xv *= (double)__ldg(in_scale + c);
            acc = fma(val64<VT>(val, k), xv, acc);
        }
        y[row * B + b] = row_scale ? acc * (double)row_scale[row] : acc;
    }
}

int product_f64(const ct_matrix* M, int which, const double* in, double* out, int32_t B, cudaStream_t st)
{
    const Csr& C = which == 0 ? M->A : M->At;
    const bool f16 = (M->flags & CT_VAL_FP16_ROWSCALE) != 0;
    // FP16 storage: A = diag(s) Q, A^T y = Q^T (s .* y)
    const float* row_scale = (f16 && which == 0) ? M->row_scale : nullptr;
    const float* in_scale = (f16 && which == 1) ? M->row_scale : nullptr;
    if (B == 1) {
        const int grid = grid_for(M, C.rows, 8, 8);
        if (f16)
            csr_f64_kernel<__half><<<grid, 256, 0, st>>>(C.row_ptr, C.col, C.qval, C.rows, in, out, row_scale, in_scale);
        else
            csr_f64_kernel<float><<<grid, 256, 0, st>>>(C.row_ptr, C.col, C.val, C.rows, in, out, row_scale, in_scale);
    } else {
        const int64_t tasks = C.rows * ((B + 31) / 32);
        const int grid = grid_for(M, tasks, 8, 8);
        if (f16)
            spmm_f64_kernel<__half><<<grid, 256, 0, st>>>(C.row_ptr, C.col, C.qval, C.rows, in, out, B, row_scale,
                                                          in_scale);
        else
            spmm_f64_kernel<float><<<grid, 256, 0, st>>>(C.row_ptr, C.col, C.val, C.rows, in, out, B, row_scale,
                                                         in_scale);
    }
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
