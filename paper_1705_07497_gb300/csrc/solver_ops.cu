// Sparse products inside the solvers, fused with the CG operator:
//     Op(p) = c_id p + c_ata A^T A p + c_grad grad^T grad p
// (Eqs. KKT, PD_resolve, SB_solve), or with the surrogate stencil T in place
// of A^T A (Sec. 3.2, Eq. surr_SBupd).
//
// Precision.  A fixed number of CG steps on these systems amplifies rounding
// of the iteration vectors by several orders of magnitude, so every solver
// vector is a double-float pair (dfloat.cuh) and every product accumulates
// with error-free transformations on the FP32 pipes; the matrix stays FP32
// (or FP16 with a row scale) and streams from HBM exactly as in an FP32
// product.  No FP64 instruction runs per entry or per row: on this part the
// FP64 pipe is far too narrow for that.
//
// Layout of the work: a warp owns a group of 16 consecutive CSR rows and
// computes their dot products one after the other (the lanes stream the row
// interleaved, 8 independent entries per lane in flight, evict-first; a
// shuffle reduction per row).  Lane r
// keeps row r's total, and the 16 epilogues then run side by side with
// coalesced vector accesses.  Grid-wide dot products finish in the last block
// (reduce.cuh).
#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "reduce.cuh"
#include "sparse_common.cuh"

namespace ct {
namespace {

constexpr int kRowsPerWarp = 16;

// Gathered vector element as a double-float pair: FP32 vectors have lo = 0.
__device__ __forceinline__ float2 gather_x(const float* __restrict__ x, int c)
{
    return make_float2(__ldg(x + c), 0.0f);
}
__device__ __forceinline__ float2 gather_x(const float2* __restrict__ x, int c) { return __ldg(x + c); }

__device__ __forceinline__ void store_y(float* y, int64_t i, float2 v) { y[i] = df_to_float(v); }
__device__ __forceinline__ void store_y(float2* y, int64_t i, float2 v) { y[i] = v; }

// Dot product of one CSR row with a gathered vector; every lane gets it.
// Lane l takes entries s + l, s + l + 32, ...: at each step the warp reads 32
// consecutive entries (coalesced) and gathers 32 consecutive columns, which
// along a ray or across neighbouring bins are mostly adjacent in memory.
template <typename VT, typename XT>
__device__ __forceinline__ float2 row_dot(const CsrView& m, const VT* __restrict__ val, int64_t row,
                                          const XT* __restrict__ x, int lane)
{
    const int64_t s = m.rp[row], e = m.rp[row + 1];
    float hs = 0.0f, hc = 0.0f;
    for (int64_t k0 = s + lane; k0 < e; k0 += 8 * 32) {
        int c[8];
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int64_t k = k0 + 32 * t;
            c[t] = k < e ? __ldcs(m.col + k) : -1;
            v[t] = k < e ? Vals<VT>::one(val, k) : 0.0f;
        }
        float2 xv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) xv[t] = c[t] >= 0 ? gather_x(x, c[t]) : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int t = 0; t < 8; ++t) acc_fma(hs, hc, v[t], xv[t]);
    }
    return warp_sum_df(acc_value(hs, hc));
}

// Runs the dot products of the warp's group of rows; lane r returns row
// (first + r)'s total (lanes >= nrows return zero).
template <typename VT, typename XT>
__device__ __forceinline__ float2 group_dots(const CsrView& m, const VT* __restrict__ val, int64_t first,
                                             int nrows, const XT* __restrict__ x, int lane)
{
    float2 mine = df_zero();
    for (int r = 0; r < nrows; ++r) {
        const float2 d = row_dot<VT, XT>(m, val, first + r, x, lane);
        if (lane == r) mine = d;
    }
    return mine;
}

// (grad^T grad u)_p with the Neumann forward-difference gradient.
__device__ __forceinline__ float2 lap_df(const float2* __restrict__ u, int64_t p, int n)
{
    const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
    const float2 c = u[p];
    float2 acc = df_zero();
    if (j > 0) acc = df_add(acc, df_sub(c, u[p - 1]));
    if (j < n - 1) acc = df_add(acc, df_sub(c, u[p + 1]));
    if (i > 0) acc = df_add(acc, df_sub(c, u[p - n]));
    if (i < n - 1) acc = df_add(acc, df_sub(c, u[p + n]));
    return acc;
}

// (grad^T (vx, vy))_p, the adjoint of the forward differences.
__device__ __forceinline__ float2 grad_adj_df(const float2* __restrict__ vx, const float2* __restrict__ vy,
                                              int64_t p, int n)
{
    const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
    float2 acc = df_zero();
    if (j >= 1) acc = df_add(acc, vx[p - 1]);
    if (j <= n - 2) acc = df_sub(acc, vx[p]);
    if (i >= 1) acc = df_add(acc, vy[p - n]);
    if (i <= n - 2) acc = df_sub(acc, vy[p]);
    return acc;
}

// Per-pixel epilogue.  MODE 1: q = Op(p), accumulate p.q.  MODE 2: r = rhs -
// Op(u), p = r, accumulate r.r and rhs.rhs.  MODE 3: r = rhs - Op(u), r.r.
template <int MODE>
__device__ __forceinline__ void op_epilogue(const OpEpilogue& a, int n, int64_t p, float2 nacc,
                                            float& s0, float& c0, float& s1, float& c1)
{
    const float2 in = a.in[p];
    float2 op = df_mul(a.c_ata, nacc);
    op = df_add(op, df_mul(a.c_grad, lap_df(a.in, p, n)));
    op = df_add(op, df_mul(a.c_id, in));
    if (MODE == 1) {
        a.out[p] = op;
        acc_add(s0, c0, df_mul(in, op));
    } else {
        const float2 rhs = a.rhs ? a.rhs[p] : df_add(a.atf[p], df_mul(a.lam, grad_adj_df(a.vx, a.vy, p, n)));
        const float2 r = df_sub(rhs, op);
        a.out[p] = r;
        if (MODE == 2) a.p_out[p] = r;
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

struct ProdArgs {
    const float* row_scale;  // FP16 storage: multiply rows by s^rpow
    int rpow;
    float2 scale;
    const CgSlice* cg;
    const int32_t* gate;
};

// y = scale * (rows of the matrix) . x, one warp per group of rows.
template <typename VT, typename XT, typename YT>
__global__ void __launch_bounds__(256) csr_df_kernel(CsrView m, const VT* __restrict__ val,
                                                     const XT* __restrict__ x, YT* __restrict__ y,
                                                     ProdArgs a)
{
    if (a.gate && *a.gate) return;
    if (a.cg && !a.cg->active) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t first = warp * kRowsPerWarp; first < m.rows; first += nw * kRowsPerWarp) {
        const int nrows = (m.rows - first) < kRowsPerWarp ? (int)(m.rows - first) : kRowsPerWarp;
        float2 acc = group_dots<VT, XT>(m, val, first, nrows, x, lane);
        if (lane < nrows) {
            const int64_t row = first + lane;
            if (a.row_scale) {
                const float s = a.row_scale[row];
                acc = df_mul_f(acc, s);
                if (a.rpow == 2) acc = df_mul_f(acc, s);
            }
            store_y(y, row, df_mul(a.scale, acc));
        }
    }
}

template <typename VT, int MODE>
__global__ void __launch_bounds__(256) adj_op_df_kernel(CsrView m, const VT* __restrict__ val,
                                                        const float2* __restrict__ y, OpEpilogue a, int n)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    for (int64_t first = warp * kRowsPerWarp; first < m.rows; first += nw * kRowsPerWarp) {
        const int nrows = (m.rows - first) < kRowsPerWarp ? (int)(m.rows - first) : kRowsPerWarp;
        const float2 acc = group_dots<VT, float2>(m, val, first, nrows, y, lane);
        if (lane < nrows) op_epilogue<MODE>(a, n, first + lane, acc, s0, c0, s1, c1);
    }
    op_finish<MODE>(a, s0, c0, s1, c1);
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
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n2;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
        float hs = 0.0f, hc = 0.0f;
        for (int t = 0; t < ntaps; ++t) {
            const int ii = i + sd[t].x, jj = j + sd[t].y;
            if (ii >= 0 && ii < n && jj >= 0 && jj < n) acc_add(hs, hc, df_mul(sw[t], a.in[(int64_t)ii * n + jj]));
        }
        op_epilogue<MODE>(a, n, p, acc_value(hs, hc), s0, c0, s1, c1);
    }
    op_finish<MODE>(a, s0, c0, s1, c1);
}

__global__ void to_df_kernel(const float* __restrict__ in, const float* __restrict__ scale,
                             float2* __restrict__ out, int64_t len)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        out[i] = scale ? two_prod(in[i], scale[i]) : make_float2(in[i], 0.0f);
    }
}

template <typename XT, typename YT>
int launch_csr(const ct_matrix* M, const Csr& C, ValKind vk, const XT* x, YT* y, ProdArgs a, cudaStream_t st)
{
    CsrView m{C.row_ptr, C.col, C.rows};
    const int grid = grid_for(M, C.rows, 8 * kRowsPerWarp, 8);
    if (vk == ValKind::F16)
        csr_df_kernel<__half, XT, YT><<<grid, 256, 0, st>>>(m, C.qval, x, y, a);
    else
        csr_df_kernel<float, XT, YT><<<grid, 256, 0, st>>>(m, C.val, x, y, a);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

int launch_forward_df(const ct_matrix* M, ValKind vk, const float2* x, float2* y, int rpow,
                      const CgSlice* cg, const int32_t* gate, cudaStream_t st)
{
    ProdArgs a{vk == ValKind::F16 ? M->row_scale : nullptr, rpow, make_float2(1.0f, 0.0f), cg, gate};
    return launch_csr(M, M->A, vk, x, y, a, st);
}

int launch_adjoint_df(const ct_matrix* M, ValKind vk, const float2* y, float2* out, double scale,
                      cudaStream_t st)
{
    ProdArgs a{nullptr, 0, df_from_double(scale), nullptr, nullptr};
    return launch_csr(M, M->At, vk, y, out, a, st);
}

int launch_forward_f32(const ct_matrix* M, ValKind vk, const float* x, float* y, cudaStream_t st)
{
    ProdArgs a{vk == ValKind::F16 ? M->row_scale : nullptr, 1, make_float2(1.0f, 0.0f), nullptr, nullptr};
    return launch_csr(M, M->A, vk, x, y, a, st);
}

int launch_adjoint_f32(const ct_matrix* M, ValKind vk, const float* y, const float2* y_scaled, float* x,
                       cudaStream_t st)
{
    ProdArgs a{nullptr, 0, make_float2(1.0f, 0.0f), nullptr, nullptr};
    if (y_scaled) return launch_csr(M, M->At, vk, y_scaled, x, a, st);
    return launch_csr(M, M->At, vk, y, x, a, st);
}

int launch_adjoint_op_df(const ct_matrix* M, ValKind vk, const float2* y, const OpEpilogue& ep,
                         cudaStream_t st)
{
    const Csr& C = M->At;
    CsrView m{C.row_ptr, C.col, C.rows};
    const int grid = grid_for(M, C.rows, 8 * kRowsPerWarp, 8);
    const int n = M->g.n;
#define CT_OP_LAUNCH(VT, VAL)                                                                    \
    switch (ep.mode) {                                                                           \
    case 1: adj_op_df_kernel<VT, 1><<<grid, 256, 0, st>>>(m, VAL, y, ep, n); break;              \
    case 2: adj_op_df_kernel<VT, 2><<<grid, 256, 0, st>>>(m, VAL, y, ep, n); break;              \
    default: adj_op_df_kernel<VT, 3><<<grid, 256, 0, st>>>(m, VAL, y, ep, n); break;             \
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

int launch_to_df(const ct_matrix* M, const float* in, const float* scale, float2* out, int64_t len,
                 cudaStream_t st)
{
    to_df_kernel<<<grid_for(M, len, 256, 8), 256, 0, st>>>(in, scale, out, len);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ct
