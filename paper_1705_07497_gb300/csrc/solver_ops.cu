// Sparse products inside the solvers, fused with the CG operator:
//     Op(p) = c_id p + c_ata A^T A p + c_grad grad^T grad p
// (Eqs. KKT, PD_resolve, SB_solve), or with the surrogate stencil T in place
// of A^T A (Sec. 3.2, Eq. surr_SBupd).
//
// Precision.  A fixed number of CG steps on these systems amplifies rounding
// of the iteration vectors by several orders of magnitude, so the solver
// vectors are FP64 and the products accumulate in double-float: the matrix
// stays FP32 (or FP16 with a row scale) and streams from HBM exactly as in
// the FP32 product, each gathered vector element is an FP32 pair (hi, lo),
// and every entry's contribution is added with error-free transformations on
// the FP32 pipes (no FP64 arithmetic per entry).  Only per-row and per-pixel
// work (the row total, the epilogue, the dot products) runs in FP64.
//
// Layout of the work: one warp per CSR row, each lane streaming 8 consecutive
// entries per step (two 16-byte column loads, one or two 16-byte value
// loads, evict-first), a shuffle reduction per row, and the epilogue in lane
// 0.  Grid-wide dot products finish in the last block (reduce.cuh).
#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "reduce.cuh"
#include "sparse_common.cuh"

namespace ct {
namespace {

// Gathered vector element as (hi, lo): FP32 vectors have lo = 0.
__device__ __forceinline__ float2 gather_x(const float* __restrict__ x, int c)
{
    return make_float2(__ldg(x + c), 0.0f);
}
__device__ __forceinline__ float2 gather_x(const float2* __restrict__ x, int c) { return __ldg(x + c); }

__device__ __forceinline__ void store_y(float* y, int64_t i, double v) { y[i] = __double2float_rn(v); }
__device__ __forceinline__ void store_y(float2* y, int64_t i, double v) { y[i] = split_f2(v); }
__device__ __forceinline__ void store_y(double* y, int64_t i, double v) { y[i] = v; }

// Double-float dot product of one CSR row with a gathered vector (all lanes).
template <typename VT, typename XT>
__device__ __forceinline__ double row_dot_df(const CsrView& m, const VT* __restrict__ val, int64_t row,
                                             const XT* __restrict__ x, int lane)
{
    const int64_t s = m.rp[row], e = m.rp[row + 1];
    float hs = 0.0f, hc = 0.0f;
    for (int64_t k = s + lane * 8; k < e; k += 256) {
        const int4 c0 = __ldcs(reinterpret_cast<const int4*>(m.col + k));
        const int4 c1 = __ldcs(reinterpret_cast<const int4*>(m.col + k + 4));
        float v[8];
        Vals<VT>::load8(val, k, v);
        const int c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const float2 xv = gather_x(x, c[t]);
            df_fma(hs, hc, v[t], xv.x, xv.y);
        }
    }
    return warp_sum_d(df_value(hs, hc));
}

// (grad^T grad u)_p, Neumann forward differences, FP64.
__device__ __forceinline__ double lap64(const double* __restrict__ u, int64_t p, int n)
{
    const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
    const double c = u[p];
    double acc = 0.0;
    if (j > 0) acc += c - u[p - 1];
    if (j < n - 1) acc += c - u[p + 1];
    if (i > 0) acc += c - u[p - n];
    if (i < n - 1) acc += c - u[p + n];
    return acc;
}

// (grad^T (vx, vy))_p, adjoint of the forward differences, FP64.
__device__ __forceinline__ double grad_adj64(const double* __restrict__ vx, const double* __restrict__ vy,
                                             int64_t p, int n)
{
    const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
    double acc = 0.0;
    if (j >= 1) acc += vx[p - 1];
    if (j <= n - 2) acc -= vx[p];
    if (i >= 1) acc += vy[p - n];
    if (i <= n - 2) acc -= vy[p];
    return acc;
}

template <int MODE>
__device__ __forceinline__ void op_epilogue(const OpEpilogue& a, int n, int64_t p, double nacc,
                                            double& d0, double& d1)
{
    const double in = a.in[p];
    const double op = a.c_ata * nacc + a.c_grad * lap64(a.in, p, n) + a.c_id * in;
    if (MODE == 1) {
        a.out[p] = op;
        d0 += in * op;
    } else {
        const double rhs = a.rhs ? a.rhs[p] : a.atf[p] + a.lam * grad_adj64(a.vx, a.vy, p, n);
        const double r = rhs - op;
        a.out[p] = r;
        if (MODE == 2) {
            a.p_out[p] = r;
            a.p2_out[p] = split_f2(r);
        }
        d0 += r * r;
        d1 += rhs * rhs;
    }
}

template <int MODE>
__device__ __forceinline__ void op_finish(const OpEpilogue& a, double d0, double d1)
{
    double v[2] = {d0, d1}, tot[2];
    if (grid_reduce_last<2>(v, a.partials, a.counter, tot)) {
        if (MODE == 1) cg_after_pq(*a.cg, tot[0]);
        if (MODE == 2) cg_after_residual(*a.cg, tot[0], tot[1], a.tol);
        if (MODE == 3) a.cg->rr = tot[0];
    }
}

struct FwdArgs {
    const float* row_scale;  // FP16 storage: multiply rows by s^rpow
    int rpow;
    double scale;
    const CgSlice* cg;
    const int32_t* gate;
};

// y = A x (rows of A) or x = A^T y (rows of A^T): one warp per row.
template <typename VT, typename XT, typename YT>
__global__ void __launch_bounds__(256) csr_df_kernel(CsrView m, const VT* __restrict__ val,
                                                     const XT* __restrict__ x, YT* __restrict__ y,
                                                     FwdArgs a)
{
    if (a.gate && *a.gate) return;
    if (a.cg && !a.cg->active) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = warp; row < m.rows; row += nw) {
        double acc = row_dot_df<VT, XT>(m, val, row, x, lane);
        if (lane == 0) {
            if (a.row_scale) {
                const double s = (double)a.row_scale[row];
                acc *= (a.rpow == 2 ? s * s : s);
            }
            store_y(y, row, a.scale * acc);
        }
    }
}

template <typename VT, int MODE>
__global__ void __launch_bounds__(256) adj_op_df_kernel(CsrView m, const VT* __restrict__ val,
                                                        const float2* __restrict__ y2, OpEpilogue a, int n)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t row = warp; row < m.rows; row += nw) {
        const double acc = row_dot_df<VT, float2>(m, val, row, y2, lane);
        if (lane == 0) op_epilogue<MODE>(a, n, row, acc, d0, d1);
    }
    op_finish<MODE>(a, d0, d1);
}

// Surrogate operator (Sec. 3.2, Eq. def_sparse_surr): (T p)_x = sum_d s(d)
// p_{x+d} over the window, translates outside the image dropped.  One thread
// per pixel; taps (double-float pairs) staged in shared memory.
template <int MODE>
__global__ void __launch_bounds__(256) stencil_op_df_kernel(OpEpilogue a, int n,
                                                            const int32_t* __restrict__ taps_d,
                                                            const float* __restrict__ taps_w, int ntaps)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    extern __shared__ unsigned char smem_raw[];
    int2* sd = reinterpret_cast<int2*>(smem_raw);
    float2* sw = reinterpret_cast<float2*>(smem_raw + sizeof(int2) * ntaps);
    for (int t = threadIdx.x; t < ntaps; t += blockDim.x) {
        sd[t] = make_int2(taps_d[2 * t], taps_d[2 * t + 1]);
        sw[t] = make_float2(taps_w[2 * t], taps_w[2 * t + 1]);
    }
    __syncthreads();
    const int64_t n2 = (int64_t)n * n;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n2;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
        float hs = 0.0f, hc = 0.0f;
        for (int t = 0; t < ntaps; ++t) {
            const int ii = i + sd[t].x, jj = j + sd[t].y;
            if (ii >= 0 && ii < n && jj >= 0 && jj < n) {
                const float2 xv = a.in2[(int64_t)ii * n + jj];
                df_fma2(hs, hc, sw[t].x, sw[t].y, xv.x, xv.y);
            }
        }
        op_epilogue<MODE>(a, n, p, df_value(hs, hc), d0, d1);
    }
    op_finish<MODE>(a, d0, d1);
}

__global__ void to_split_kernel(const float* __restrict__ in, const float* __restrict__ scale,
                                float2* __restrict__ out, int64_t len)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = (double)in[i];
        if (scale) v *= (double)scale[i];
        out[i] = split_f2(v);
    }
}

}  // namespace

template <typename XT, typename YT>
int launch_csr_df(const ct_matrix* M, const Csr& C, ValKind vk, const XT* x, YT* y, FwdArgs a,
                  cudaStream_t st)
{
    CsrView m{C.row_ptr, C.col, C.rows};
    const int grid = grid_for(M, C.rows, 8, 8);
    if (vk == ValKind::F16)
        csr_df_kernel<__half, XT, YT><<<grid, 256, 0, st>>>(m, C.qval, x, y, a);
    else
        csr_df_kernel<float, XT, YT><<<grid, 256, 0, st>>>(m, C.val, x, y, a);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int launch_forward_df(const ct_matrix* M, ValKind vk, const float2* x2, float2* y2, int rpow,
                      const CgSlice* cg, const int32_t* gate, cudaStream_t st)
{
    FwdArgs a{vk == ValKind::F16 ? M->row_scale : nullptr, rpow, 1.0, cg, gate};
    return launch_csr_df(M, M->A, vk, x2, y2, a, st);
}

int launch_adjoint_df(const ct_matrix* M, ValKind vk, const float2* y2, double* out, double scale,
                      cudaStream_t st)
{
    FwdArgs a{nullptr, 0, scale, nullptr, nullptr};
    return launch_csr_df(M, M->At, vk, y2, out, a, st);
}

int launch_forward_f32(const ct_matrix* M, ValKind vk, const float* x, float* y, cudaStream_t st)
{
    FwdArgs a{vk == ValKind::F16 ? M->row_scale : nullptr, 1, 1.0, nullptr, nullptr};
    return launch_csr_df(M, M->A, vk, x, y, a, st);
}

int launch_adjoint_f32(const ct_matrix* M, ValKind vk, const float* y, const float2* y2_scaled, float* x,
                       cudaStream_t st)
{
    FwdArgs a{nullptr, 0, 1.0, nullptr, nullptr};
    if (y2_scaled) return launch_csr_df(M, M->At, vk, y2_scaled, x, a, st);
    return launch_csr_df(M, M->At, vk, y, x, a, st);
}

int launch_adjoint_op_df(const ct_matrix* M, ValKind vk, const float2* y2, const OpEpilogue& ep,
                         cudaStream_t st)
{
    const Csr& C = M->At;
    CsrView m{C.row_ptr, C.col, C.rows};
    const int grid = grid_for(M, C.rows, 8, 8);
    const int n = M->g.n;
#define CT_OP_LAUNCH(VT, VAL)                                                                    \
    switch (ep.mode) {                                                                           \
    case 1: adj_op_df_kernel<VT, 1><<<grid, 256, 0, st>>>(m, VAL, y2, ep, n); break;             \
    case 2: adj_op_df_kernel<VT, 2><<<grid, 256, 0, st>>>(m, VAL, y2, ep, n); break;             \
    default: adj_op_df_kernel<VT, 3><<<grid, 256, 0, st>>>(m, VAL, y2, ep, n); break;            \
    }
    if (vk == ValKind::F16) {
        CT_OP_LAUNCH(__half, C.qval)
    } else {
        CT_OP_LAUNCH(float, C.val)
    }
#undef CT_OP_LAUNCH
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int launch_stencil_op_df(const ct_matrix* M, const Stencil* S, const OpEpilogue& ep, cudaStream_t st)
{
    const int n = M->g.n;
    const int64_t n2 = (int64_t)n * n;
    const int grid = grid_for(M, n2, 256, 8);
    const int ntaps = S ? S->ntaps : 0;
    const size_t smem = (sizeof(int2) + sizeof(float2)) * (size_t)ntaps;
    const int32_t* d = S ? S->d : nullptr;
    const float* w = S ? S->w : nullptr;
    switch (ep.mode) {
    case 1: stencil_op_df_kernel<1><<<grid, 256, smem, st>>>(ep, n, d, w, ntaps); break;
    case 2: stencil_op_df_kernel<2><<<grid, 256, smem, st>>>(ep, n, d, w, ntaps); break;
    default: stencil_op_df_kernel<3><<<grid, 256, smem, st>>>(ep, n, d, w, ntaps); break;
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int launch_to_split(const ct_matrix* M, const float* in, const float* scale, float2* out2, int64_t len,
                    cudaStream_t st)
{
    to_split_kernel<<<grid_for(M, len, 256, 8), 256, 0, st>>>(in, scale, out2, len);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ct
