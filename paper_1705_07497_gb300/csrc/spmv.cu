// Sparse products with A and A^T (Sec. 2: the normal operator R* M* M R is the
// bottleneck of every iterative solver; Sec. 3 replaces it by precomputed
// sparse matrix products), the surrogate stencil T (Sec. 3.2), and the
// epilogues that fuse the rest of the CG operator into the adjoint product.
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

namespace ct {
namespace {

struct CsrView {
    const int64_t* rp;
    const int32_t* col;
    int64_t rows;
};

template <typename VT>
struct Vals;

template <>
struct Vals<float> {
    static __device__ __forceinline__ void load8(const float* v, int64_t k, float (&o)[8])
    {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(v + k));
        const float4 b = __ldcs(reinterpret_cast<const float4*>(v + k + 4));
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
        o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    }
    static __device__ __forceinline__ float one(const float* v, int64_t k) { return __ldcs(v + k); }
};

template <>
struct Vals<__half> {
    static __device__ __forceinline__ void load8(const __half* v, int64_t k, float (&o)[8])
    {
        const uint4 a = __ldcs(reinterpret_cast<const uint4*>(v + k));
        const __half2* h = reinterpret_cast<const __half2*>(&a);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 f = __half22float2(h[t]);
            o[2 * t] = f.x;
            o[2 * t + 1] = f.y;
        }
    }
    static __device__ __forceinline__ float one(const __half* v, int64_t k)
    {
        return __half2float(v[k]);
    }
};

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

// (grad^T grad u)_p with the Neumann forward-difference gradient.
__device__ __forceinline__ float neumann_lap(const float* __restrict__ u, int64_t p, int n, int64_t B)
{
    const int64_t pix = p / B;
    const int i = (int)(pix / n), j = (int)(pix - (int64_t)i * n);
    const float c = u[p];
    float acc = 0.0f;
    if (j > 0) acc += c - u[p - B];
    if (j < n - 1) acc += c - u[p + B];
    if (i > 0) acc += c - u[p - (int64_t)n * B];
    if (i < n - 1) acc += c - u[p + (int64_t)n * B];
    return acc;
}

// (grad^T (vx, vy))_p, the adjoint of the forward differences.
__device__ __forceinline__ float grad_adj_at(const float* __restrict__ vx, const float* __restrict__ vy,
                                             int64_t p, int n, int64_t B)
{
    const int64_t pix = p / B;
    const int i = (int)(pix / n), j = (int)(pix - (int64_t)i * n);
    float acc = 0.0f;
    if (j >= 1) acc += vx[p - B];
    if (j <= n - 2) acc -= vx[p];
    if (i >= 1) acc += vy[p - (int64_t)n * B];
    if (i <= n - 2) acc -= vy[p];
    return acc;
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

// Per-pixel operator epilogue shared by the sparse and stencil kernels.
// MODE 1: q = Op(p), accumulate p.q.
// MODE 2: r = rhs - Op(u), p = r, accumulate r.r and rhs.rhs (CG start).
// MODE 3: r = rhs - Op(u) only, accumulate r.r (residual replacement).
template <int MODE>
__device__ __forceinline__ void op_epilogue(const OpEpilogue& a, int n, int64_t p, float nacc,
                                            double& d0, double& d1)
{
    const float in = a.in[p];
    const float op = a.c_ata * nacc + a.c_grad * neumann_lap(a.in, p, n, 1) + a.c_id * in;
    if (MODE == 1) {
        a.out[p] = op;
        d0 += (double)in * (double)op;
    } else {
        const float rhs = a.rhs ? a.rhs[p] : a.atf[p] + a.lam * grad_adj_at(a.vx, a.vy, p, n, 1);
        const float r = rhs - op;
        a.out[p] = r;
        if (MODE == 2) a.p_out[p] = r;
        d0 += (double)r * (double)r;
        d1 += (double)rhs * (double)rhs;
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

template <typename VT, bool GS, int MODE>
__global__ void __launch_bounds__(256) spmv_op_kernel(CsrView m, const VT* __restrict__ val,
                                                      const float* __restrict__ y,
                                                      const float* __restrict__ gs, OpEpilogue a,
                                                      int n)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t row = warp; row < m.rows; row += nw) {
        const float acc = row_dot<VT, GS>(m, val, row, y, gs, lane);
        if (lane == 0) op_epilogue<MODE>(a, n, row, acc, d0, d1);
    }
    op_finish<MODE>(a, d0, d1);
}

// Surrogate operator (Sec. 3.2, Eq. def_sparse_surr): (T p)_x = sum_d s(d)
// p_{x+d} over the window, translates outside the image dropped; fused with
// the same epilogue.  One thread per pixel; taps staged in shared memory.
template <int MODE>
__global__ void __launch_bounds__(256) stencil_op_kernel(OpEpilogue a, int n,
                                                         const int32_t* __restrict__ taps_d,
                                                         const float* __restrict__ taps_w, int ntaps)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    extern __shared__ unsigned char smem_raw[];
    int2* sd = reinterpret_cast<int2*>(smem_raw);
    float* sw = reinterpret_cast<float*>(smem_raw + sizeof(int2) * ntaps);
    for (int t = threadIdx.x; t < ntaps; t += blockDim.x) {
        sd[t] = make_int2(taps_d[2 * t], taps_d[2 * t + 1]);
        sw[t] = taps_w[t];
    }
    __syncthreads();
    const int64_t n2 = (int64_t)n * n;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n2;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p / n), j = (int)(p - (int64_t)i * n);
        float acc = 0.0f;
        for (int t = 0; t < ntaps; ++t) {
            const int ii = i + sd[t].x, jj = j + sd[t].y;
            if (ii >= 0 && ii < n && jj >= 0 && jj < n) acc = fmaf(sw[t], a.in[(int64_t)ii * n + jj], acc);
        }
        op_epilogue<MODE>(a, n, p, acc, d0, d1);
    }
    op_finish<MODE>(a, d0, d1);
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
    StoreArgs a{};
    a.scale = out_scale;
    if (vk == ValKind::F16) {
        a.row_scale = M->row_scale;
        a.rpow = scale_sq ? 2 : 1;
        return launch_store<__half, false>(M, M->A, M->A.qval, x, y, batch, nullptr, a, st);
    }
    return launch_store<float, false>(M, M->A, M->A.val, x, y, batch, nullptr, a, st);
}

int launch_forward_gated(const ct_matrix* M, ValKind vk, const float* x, float* y, int32_t batch,
                         bool normal_scale, const CgSlice* cg, const int32_t* gate, cudaStream_t st)
{
    StoreArgs a{};
    a.scale = 1.0f;
    a.gate = gate;
    a.cg = batch == 1 ? cg : nullptr;
    if (vk == ValKind::F16) {
        a.row_scale = M->row_scale;
        a.rpow = normal_scale ? 2 : 1;
        return launch_store<__half, false>(M, M->A, M->A.qval, x, y, batch, nullptr, a, st);
    }
    return launch_store<float, false>(M, M->A, M->A.val, x, y, batch, nullptr, a, st);
}

int launch_adjoint(const ct_matrix* M, ValKind vk, const float* y, float* x, int32_t batch,
                   float out_scale, bool scale_y, cudaStream_t st)
{
    StoreArgs a{};
    a.scale = out_scale;
    if (vk == ValKind::F16) {
        if (scale_y)
            return launch_store<__half, true>(M, M->At, M->At.qval, y, x, batch, M->row_scale, a, st);
        return launch_store<__half, false>(M, M->At, M->At.qval, y, x, batch, nullptr, a, st);
    }
    return launch_store<float, false>(M, M->At, M->At.val, y, x, batch, nullptr, a, st);
}

int launch_adjoint_op(const ct_matrix* M, ValKind vk, const float* y, int32_t batch,
                      const OpEpilogue& ep, cudaStream_t st)
{
    if (batch != 1) return fail(CT_ERR_UNSUPPORTED, "fused operator epilogue needs batch 1");
    const Csr& C = M->At;
    CsrView m{C.row_ptr, C.col, C.rows};
    const int grid = grid_for(M, C.rows, 8, 8);
    const int n = M->g.n;
#define CT_OP_LAUNCH(VT, VAL)                                                                   \
    switch (ep.mode) {                                                                          \
    case 1: spmv_op_kernel<VT, false, 1><<<grid, 256, 0, st>>>(m, VAL, y, nullptr, ep, n); break; \
    case 2: spmv_op_kernel<VT, false, 2><<<grid, 256, 0, st>>>(m, VAL, y, nullptr, ep, n); break; \
    default: spmv_op_kernel<VT, false, 3><<<grid, 256, 0, st>>>(m, VAL, y, nullptr, ep, n); break; \
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

int launch_stencil_op(const ct_matrix* M, const Stencil* S, int32_t batch, const OpEpilogue& ep,
                      cudaStream_t st)
{
    if (batch != 1) return fail(CT_ERR_UNSUPPORTED, "stencil operator epilogue needs batch 1");
    const int n = M->g.n;
    const int64_t n2 = (int64_t)n * n;
    const int grid = grid_for(M, n2, 256, 8);
    const int ntaps = S ? S->ntaps : 0;
    const size_t smem = (sizeof(int2) + sizeof(float)) * (size_t)ntaps;
    const int32_t* d = S ? S->d : nullptr;
    const float* w = S ? S->w : nullptr;
    switch (ep.mode) {
    case 1: stencil_op_kernel<1><<<grid, 256, smem, st>>>(ep, n, d, w, ntaps); break;
    case 2: stencil_op_kernel<2><<<grid, 256, smem, st>>>(ep, n, d, w, ntaps); break;
    default: stencil_op_kernel<3><<<grid, 256, smem, st>>>(ep, n, d, w, ntaps); break;
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ct
