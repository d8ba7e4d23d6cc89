// Stand-alone products y = A x and x = A^T y (ct_forward, ct_adjoint and their
// FP64-vector forms).  Sec. 2: the normal operator R* M* M R is the
// bottleneck of every iterative solver; Sec. 3 replaces it by precomputed
// sparse matrix products.  The FP32 forms accumulate in double-float with the
// kernels the solvers use (solver_ops.cu for one slice, batch.cu for a
// batch); the caller's row-major image is moved to and from the internal tile
// order on the way.
#include <algorithm>

#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "layout.cuh"
#include "sparse_common.cuh"

namespace ct {
namespace {

// Caller's row-major image -> internal tile order (FP32, padding zero).
__global__ void to_tiles_kernel(const float* __restrict__ in, float* __restrict__ out, int n, int tn)
{
    const int64_t npad = padded_pixels(n);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npad; t += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(t, tn, i, j);
        out[t] = (i < n && j < n) ? in[(int64_t)i * n + j] : 0.0f;
    }
}

// FP64-vector products on the FP64 pipe (handles built with
// CT_F64_FP64_PIPE): FP64 gathers and FP64 accumulation, one FMA per entry.
// The default path (below) splits the FP64 vectors into double-float pairs
// and runs the solvers' kernels on the FP32 pipes, with the same accuracy in
// the derivatives of the unrolled reconstruction and several times the speed.
template <typename VT>
__device__ __forceinline__ double val64(const VT* v, int64_t k);
template <>
__device__ __forceinline__ double val64<float>(const float* v, int64_t k) { return (double)__ldg(v + k); }
template <>
__device__ __forceinline__ double val64<__half>(const __half* v, int64_t k)
{
    return (double)__half2float(v[k]);
}

struct F64Map {
    int which;  // 0: A (rows = rays, columns = internal pixels); 1: A^T (rows = internal pixels)
    const int32_t* col;
    const uint16_t* col16;
    const int32_t* band_lo;
    const int32_t* band_off;
    const uint16_t* band_angle;
    int n, tn, nb, nk;
};

// Index into the caller's vector for an entry (pixel: row-major; ray: q).
__device__ __forceinline__ int64_t f64_col(const F64Map& fm, int64_t row, int64_t k)
{
    if (fm.which == 0) {
        int i, j;
        tiled_coords(__ldg(fm.col + k), fm.tn, i, j);
        return (int64_t)i * fm.n + j;
    }
    const int c = (int)__ldg(fm.col16 + k);
    const int a = __ldg(fm.band_angle + c);
    return (int64_t)a * fm.nb + fm.band_lo[(row >> 8) * fm.nk + a] + (c - __ldg(fm.band_off + a));
}

// Output position of a row in the caller's vector (-1: padding pixel).
__device__ __forceinline__ int64_t f64_row(const F64Map& fm, int64_t row)
{
    if (fm.which == 0) return row;
    int i, j;
    tiled_coords(row, fm.tn, i, j);
    return (i < fm.n && j < fm.n) ? (int64_t)i * fm.n + j : -1;
}

// B = 1: one lane per row (a warp per SELL slice, the lane's row entries in
// order).  B > 1: see below.
template <typename VT>
__global__ void __launch_bounds__(256) f64_kernel(SellView m, F64Map fm, const VT* __restrict__ val,
                                                  const double* __restrict__ x, double* __restrict__ y,
                                                  int B, const float* __restrict__ row_scale,
                                                  const float* __restrict__ in_scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (B == 1) {
        const int64_t nslices = (m.rows + kSliceRows - 1) / kSliceRows;
        for (int64_t s = warp; s < nslices; s += nw) {
            const int64_t row = s * kSliceRows + lane;
            if (row >= m.rows) continue;
            const int64_t pos = f64_row(fm, row);
            if (pos < 0) continue;
            const int64_t base = row_base(m, row);
            const int len = m.len[row];
            double acc = 0.0;
            for (int e = 0; e < len; ++e) {
                const int64_t k = chunk_pos(base, e);
                const int64_t c = f64_col(fm, row, k);
                double xv = __ldg(x + c);
                if (in_scale) xv *= (double)__ldg(in_scale + c);
                acc = fma(val64<VT>(val, k), xv, acc);
            }
            y[pos] = row_scale ? acc * (double)row_scale[row] : acc;
        }
        return;
    }
    // B > 1: sub-groups of W lanes (W = the power of two >= B, at most 32),
    // one row per sub-group and one slice per lane; the sub-group stages W
    // entries at a time (the input index and the value in FP64, converted
    // once) and every lane then does one gather and one FP64 FMA per entry.
    __shared__ double sval[8][32];
    __shared__ int64_t scol[8][32];
    int W = 1;
    while (W < B && W < 32) W <<= 1;
    const int rpw = 32 / W, g = lane / W, t_in = lane % W, wib = threadIdx.x >> 5;
    const int chunks = (B + W - 1) / W;
    const int64_t groups = (m.rows + rpw - 1) / rpw;
    for (int64_t task = warp; task < groups * chunks; task += nw) {
        const int64_t row = (task / chunks) * rpw + g;
        const int b = (int)(task % chunks) * W + t_in;
        const bool rv = row < m.rows;
        const int64_t pos = rv ? f64_row(fm, row) : -1;
        const int len = (rv && pos >= 0) ? m.len[row] : 0;
        const int64_t base = rv ? row_base(m, row) : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        double acc = 0.0;
        for (int j0 = 0; j0 < maxlen; j0 += W) {
            if (j0 + t_in < len) {
                const int64_t k = chunk_pos(base, j0 + t_in);
                const int64_t c = f64_col(fm, row, k);
                double v = val64<VT>(val, k);
                if (in_scale) v *= (double)__ldg(in_scale + c);
                scol[wib][lane] = c;
                sval[wib][lane] = v;
            }
            __syncwarp();
            const int cnt = min(W, len - j0);
            if (b < B)
                for (int t = 0; t < cnt; ++t)
                    acc = fma(sval[wib][g * W + t], __ldg(x + scol[wib][g * W + t] * B + b), acc);
            __syncwarp();
        }
        if (len > 0 && b < B) y[pos * B + b] = row_scale ? acc * (double)row_scale[row] : acc;
        else if (rv && pos >= 0 && b < B) y[pos * B + b] = 0.0;
    }
}

int product_f64(const ct_matrix* M, int which, const double* in, double* out, int32_t B, cudaStream_t st)
{
    const Sell& C = which == 0 ? M->A : M->At;
    const bool f16 = (M->flags & CT_VAL_FP16_ROWSCALE) != 0;
    // FP16 storage: A = diag(s) Q, A^T y = Q^T (s .* y)
    const float* row_scale = (f16 && which == 0) ? M->row_scale : nullptr;
    const float* in_scale = (f16 && which == 1) ? M->row_scale : nullptr;
    const F64Map fm{which, M->A.col, M->At.col16, M->band_lo, M->band_off, M->band_angle,
                    M->g.n, M->tn, M->g.n_bins, M->n_kept};
    const SellView m{C.slice_ptr, C.row_len, C.rows};
    int W = 1;
    while (W < B && W < 32) W <<= 1;
    const int64_t tasks = B == 1 ? (C.rows + kSliceRows - 1) / kSliceRows
                                 : (C.rows + 32 / W - 1) / (32 / W) * ((B + W - 1) / W);
    const int grid = grid_for(M, tasks, 8, 8);
    if (f16)
        f64_kernel<__half><<<grid, 256, 0, st>>>(m, fm, C.qval, in, out, B, row_scale, in_scale);
    else
        f64_kernel<float><<<grid, 256, 0, st>>>(m, fm, C.val, in, out, B, row_scale, in_scale);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// out = alpha * out + lambda * (grad^T grad x), FP64 vectors [N*N][B] in the
// caller's row-major order; forward differences with a zero last difference.
__global__ void normal_epilogue_f64_kernel(const double* __restrict__ x, double* __restrict__ out, int n, int B,
                                           double alpha, double lam)
{
    const int64_t total = (int64_t)n * n * B;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = k / B;
        const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
        const double c = x[k];
        double lap = 0.0;
        if (j > 0) lap += c - x[k - B];
        if (j < n - 1) lap += c - x[k + B];
        if (i > 0) lap += c - x[k - (int64_t)n * B];
        if (i < n - 1) lap += c - x[k + (int64_t)n * B];
        out[k] = alpha * out[k] + lam * lap;
    }
}

// ---- FP64 vectors through the double-float kernels (the default) ----
//
// An FP64 value v becomes the pair (hi, lo) = (fl32(v), fl32(v - hi)), which
// holds v to 2^-48 relative; the products then run on the FP32 pipes exactly
// as the solvers' (error-free products of the FP32 matrix values with both
// parts, compensated sums), and an output pair goes back as hi + lo in FP64.
__device__ __forceinline__ float2 split_f64(double v)
{
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ double join_f64(float2 p) { return (double)p.x + (double)p.y; }

// Caller's row-major FP64 image [n*n][B] -> double-float pairs in tile order [npad][B].
__global__ void f64_image_to_df_kernel(const double* __restrict__ in, float2* __restrict__ out, int n, int tn, int B)
{
    const int64_t len = padded_pixels(n) * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / B;
        const int b = (int)(e - t * B);
        int i, j;
        tiled_coords(t, tn, i, j);
        out[e] = (i < n && j < n) ? split_f64(in[((int64_t)i * n + j) * B + b]) : make_float2(0.0f, 0.0f);
    }
}

// FP64 sinogram [rows][B] -> double-float pairs, times the row scale s when
// given (FP16 storage: A^T y = Q^T (s .* y); the product s y is formed in FP64).
__global__ void f64_rows_to_df_kernel(const double* __restrict__ in, const float* __restrict__ scale,
                                      float2* __restrict__ out, int64_t rows, int B)
{
    const int64_t len = rows * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = in[e];
        out[e] = split_f64(scale ? v * (double)scale[e / B] : v);
    }
}

__global__ void df_rows_to_f64_kernel(const float2* __restrict__ in, double* __restrict__ out, int64_t len)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = join_f64(in[e]);
}

// Double-float image in tile order [npad][B] -> FP64 row-major [n*n][B];
// with x given, out = alpha * in + lambda * grad^T grad x instead (the
// operator epilogue of ct_normal_f64, on the caller's FP64 x).
__global__ void df_image_to_f64_kernel(const float2* __restrict__ in, double* __restrict__ out, int n, int tn, int B,
                                       const double* __restrict__ x, double alpha, double lam)
{
    const int64_t total = (int64_t)n * n * B;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = k / B;
        const int b = (int)(k - p * B);
        const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
        const double v = join_f64(in[tiled_index(i, j, tn) * B + b]);
        if (!x) {
            out[k] = v;
            continue;
        }
        const double c = x[k];
        double lap = 0.0;
        if (j > 0) lap += c - x[k - B];
        if (j < n - 1) lap += c - x[k + B];
        if (i > 0) lap += c - x[k - (int64_t)n * B];
        if (i < n - 1) lap += c - x[k + (int64_t)n * B];
        out[k] = alpha * v + lam * lap;
    }
}

int ensure_f64_buffer(float2*& buf, int64_t& have, int64_t need)
{
    if (have >= need) return CT_OK;
    cudaFree(buf);
    buf = nullptr;
    have = 0;
    const cudaError_t e = cudaMalloc((void**)&buf, (size_t)need * sizeof(float2));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(double-float FP64-product buffer)", __FILE__, __LINE__);
    have = need;
    return CT_OK;
}

// Double-float product on internal layouts: which = 0: out = s^rpow .* (A in)
// ([npad][B] -> [rows][B]); which = 1: out = A^T in ([rows][B] -> [npad][B];
// with FP16 storage Q^T in).
int product_df_internal(const ct_matrix* M, int which, const float2* in, float2* out, int32_t B, int rpow,
                        cudaStream_t st)
{
    const ValKind vk = (M->flags & CT_VAL_FP16_ROWSCALE) ? ValKind::F16 : ValKind::F32;
    if (B > 1) return batched_product_df(M, which, in, out, B, which == 0 ? rpow : 0, st);
    if (which == 0) return launch_forward_df(M, vk, in, out, vk == ValKind::F16 ? rpow : 0, nullptr, nullptr, st);
    return launch_adjoint_df(M, vk, in, out, 1.0, st);
}

int product_f64_df(const ct_matrix* M, int which, const double* in, double* out, int32_t B, cudaStream_t st)
{
    Workspace& w = const_cast<ct_matrix*>(M)->ws;
    const bool f16 = (M->flags & CT_VAL_FP16_ROWSCALE) != 0;
    CT_CHECK(ensure_f64_buffer(w.f64_a, w.f64_a_len, std::max<int64_t>(M->npad, M->rows) * B));
    CT_CHECK(ensure_f64_buffer(w.f64_b, w.f64_b_len, std::max<int64_t>(M->npad, M->rows) * B));
    if (which == 0) {
        f64_image_to_df_kernel<<<grid_for(M, M->npad * B, 256, 8), 256, 0, st>>>(in, w.f64_a, M->g.n, M->tn, B);
        CT_CUDA(cudaGetLastError());
        CT_CHECK(product_df_internal(M, 0, w.f64_a, w.f64_b, B, 1, st));
        df_rows_to_f64_kernel<<<grid_for(M, M->rows * B, 256, 8), 256, 0, st>>>(w.f64_b, out, M->rows * B);
    } else {
        f64_rows_to_df_kernel<<<grid_for(M, M->rows * B, 256, 8), 256, 0, st>>>(in, f16 ? M->row_scale : nullptr,
                                                                              w.f64_a, M->rows, B);
        CT_CUDA(cudaGetLastError());
        CT_CHECK(product_df_internal(M, 1, w.f64_a, w.f64_b, B, 0, st));
        df_image_to_f64_kernel<<<grid_for(M, (int64_t)M->g.n * M->g.n * B, 256, 8), 256, 0, st>>>(
            w.f64_b, out, M->g.n, M->tn, B, nullptr, 0.0, 0.0);
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// ct_normal_f64 in double-float: x split once, A x with s^2 (FP16 storage:
// A^T A = Q^T diag(s^2) Q), A^T of that, then the epilogue back in FP64.
int normal_f64_df(const ct_matrix* M, double alpha, double lam, const double* x, double* out, int32_t B,
                  cudaStream_t st)
{
    Workspace& w = const_cast<ct_matrix*>(M)->ws;
    CT_CHECK(ensure_f64_buffer(w.f64_a, w.f64_a_len, std::max<int64_t>(M->npad, M->rows) * B));
    CT_CHECK(ensure_f64_buffer(w.f64_b, w.f64_b_len, std::max<int64_t>(M->npad, M->rows) * B));
    CT_CHECK(ensure_f64_buffer(w.f64_c, w.f64_c_len, M->npad * (int64_t)B));
    f64_image_to_df_kernel<<<grid_for(M, M->npad * B, 256, 8), 256, 0, st>>>(x, w.f64_a, M->g.n, M->tn, B);
    CT_CUDA(cudaGetLastError());
    CT_CHECK(product_df_internal(M, 0, w.f64_a, w.f64_b, B, 2, st));
    CT_CHECK(product_df_internal(M, 1, w.f64_b, w.f64_c, B, 0, st));
    df_image_to_f64_kernel<<<grid_for(M, (int64_t)M->g.n * M->g.n * B, 256, 8), 256, 0, st>>>(
        w.f64_c, out, M->g.n, M->tn, B, x, alpha, lam);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

int normal_f64(const ct_matrix* M, double alpha, double lam, const double* x, double* out, int32_t B,
               cudaStream_t st)
{
    if (!(M->flags & CT_F64_FP64_PIPE)) return normal_f64_df(M, alpha, lam, x, out, B, st);
    ct_matrix* Mm = const_cast<ct_matrix*>(M);
    Workspace& w = Mm->ws;
    const int64_t need = M->rows * (int64_t)B;
    if (w.f64_y_len < need) {
        cudaFree(w.f64_y);
        w.f64_y = nullptr;
        w.f64_y_len = 0;
        const cudaError_t e = cudaMalloc((void**)&w.f64_y, (size_t)need * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(FP64 sinogram temp)", __FILE__, __LINE__);
        w.f64_y_len = need;
    }
    CT_CHECK(product_f64(M, 0, x, w.f64_y, B, st));
    CT_CHECK(product_f64(M, 1, w.f64_y, out, B, st));
    const int64_t total = (int64_t)M->g.n * M->g.n * B;
    normal_epilogue_f64_kernel<<<grid_for(M, total, 256, 8), 256, 0, st>>>(x, out, M->g.n, B, alpha, lam);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
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
    if (batch != 1) return batched_forward_adjoint(M, 0, x, y, batch, st);
    ct_matrix* Mm = const_cast<ct_matrix*>(M);
    Workspace& w = Mm->ws;
    if (w.pub_x_len < M->npad) {
        cudaFree(w.pub_x);
        w.pub_x = nullptr;
        w.pub_x_len = 0;
        CT_CUDA(cudaMalloc((void**)&w.pub_x, (size_t)M->npad * sizeof(float)));
        w.pub_x_len = M->npad;
    }
    to_tiles_kernel<<<grid_for(M, M->npad, 256, 8), 256, 0, st>>>(x, w.pub_x, M->g.n, M->tn);
    CT_CUDA(cudaGetLastError());
    return launch_forward_f32(M, vk, w.pub_x, y, st);
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

int launch_forward_f64(const ct_matrix* M, ValKind, const double* x, double* y, int32_t batch, cudaStream_t st)
{
    if (!(M->flags & CT_F64_FP64_PIPE)) return product_f64_df(M, 0, x, y, batch, st);
    return product_f64(M, 0, x, y, batch, st);
}

int launch_adjoint_f64(const ct_matrix* M, ValKind, const double* y, double* x, int32_t batch, cudaStream_t st)
{
    if (!(M->flags & CT_F64_FP64_PIPE)) return product_f64_df(M, 1, y, x, batch, st);
    return product_f64(M, 1, y, x, batch, st);
}

}  // namespace ct
