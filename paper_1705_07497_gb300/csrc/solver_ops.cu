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
// y = A x: a warp owns a group of 16 consecutive rays and computes their dot
// products one after the other; lanes stream the row interleaved (8
// independent entries per lane in flight, evict-first) and gather x from the
// tiled image layout (layout.cuh), where a run of pixels along any ray stays
// within a few cache lines; a shuffle reduction per row, and lane r keeps
// row r's total so the 16 stores run side by side.
//
// x = A^T y: one CTA per 16 x 16 image tile.  The CTA first copies the tile's
// sinogram band (kBandW bins per kept angle) into shared memory with
// coalesced loads; every entry of the tile's rows then reads its operand from
// shared memory through its 16-bit band index.  Each warp computes 32 pixels
// (two groups of 16), and the operator epilogue for a group runs lane-parallel.
// Grid-wide dot products finish in the last block (reduce.cuh).
#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "layout.cuh"
#include "reduce.cuh"
#include "sparse_common.cuh"

namespace ct {
namespace {

constexpr int kRowsPerWarp = 16;

struct BandView {
    const int64_t* rp;
    const uint16_t* col16;
    const int32_t* band_lo;
    int n, tn, nb, nk;
};

// Gathered vector element as a double-float pair: FP32 vectors have lo = 0.
__device__ __forceinline__ float2 gather_x(const float* __restrict__ x, int64_t c)
{
    return make_float2(__ldg(x + c), 0.0f);
}
__device__ __forceinline__ float2 gather_x(const float2* __restrict__ x, int64_t c) { return __ldg(x + c); }

__device__ __forceinline__ void store_y(float* y, int64_t i, float2 v) { y[i] = df_to_float(v); }
__device__ __forceinline__ void store_y(float2* y, int64_t i, float2 v) { y[i] = v; }

// Dot product of one CSR row with a gathered vector; every lane gets it.
// Lane l takes entries s + l, s + l + 32, ...: at each step the warp reads 32
// consecutive entries (coalesced) and gathers 32 consecutive columns.
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

// Dot product of one A^T row with the tile's staged sinogram band, computed by
// a half-warp: each of its 16 lanes takes 8 consecutive entries per step with
// 16-byte loads (rows are padded to multiples of 8 entries); the operands come
// from shared memory, so consecutive entries per lane cost nothing in
// coalescing.  Every lane of the half-warp gets the total.
__device__ __forceinline__ void load8_col16(const uint16_t* p, int64_t k, int (&c)[8])
{
    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p + k));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        c[2 * t] = (int)(w[t] & 0xffffu);
        c[2 * t + 1] = (int)(w[t] >> 16);
    }
}

template <typename VT>
__device__ __forceinline__ float2 band_row_dot_half(const int64_t* __restrict__ rp, const uint16_t* __restrict__ col16,
                                                    const VT* __restrict__ val, int64_t row,
                                                    const float2* __restrict__ band, int hl)
{
    const int64_t s = rp[row], e = rp[row + 1];
    float hs = 0.0f, hc = 0.0f;
    for (int64_t k = s + hl * 8; k < e; k += 128) {
        int c[8];
        float v[8];
        load8_col16(col16, k, c);
        Vals<VT>::load8(val, k, v);
#pragma unroll
        for (int t = 0; t < 8; ++t) acc_fma(hs, hc, v[t], band[c[t]]);
    }
    float2 r = acc_value(hs, hc);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        float2 w;
        w.x = __shfl_xor_sync(0xffffffffu, r.x, o);
        w.y = __shfl_xor_sync(0xffffffffu, r.y, o);
        r = df_add(r, w);
    }
    return r;
}

// The 16 dot products of rows first .. first + 15 of the tile, two rows at a
// time (one per half-warp); lane r (< 16) returns row first + r's total.
template <typename VT>
__device__ __forceinline__ float2 band_group_dots(const BandView& bv, const VT* __restrict__ val, int64_t first,
                                                  const float2* __restrict__ band, int lane)
{
    const int half = lane >> 4, hl = lane & 15;
    float2 mine = df_zero();
#pragma unroll 2
    for (int r = 0; r < kRowsPerWarp; r += 2) {
        const float2 d = band_row_dot_half<VT>(bv.rp, bv.col16, val, first + r + half, band, hl);
        const float2 d0 = make_float2(__shfl_sync(0xffffffffu, d.x, 0), __shfl_sync(0xffffffffu, d.y, 0));
        const float2 d1 = make_float2(__shfl_sync(0xffffffffu, d.x, 16), __shfl_sync(0xffffffffu, d.y, 16));
        if (lane == r) mine = d0;
        if (lane == r + 1) mine = d1;
    }
    return mine;
}

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

// (grad^T (vx, vy)) at pixel (i, j), the adjoint of the forward differences.
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

struct ProdArgs {
    const float* row_scale;  // FP16 storage: multiply rows by s^rpow
    int rpow;
    float2 scale;
    const CgSlice* cg;
    const int32_t* gate;
};

// y = scale * A x, one warp per group of rays (x in the tiled layout).
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
        float2 mine = df_zero();
        for (int r = 0; r < nrows; ++r) {
            const float2 d = row_dot<VT, XT>(m, val, first + r, x, lane);
            if (lane == r) mine = d;
        }
        if (lane < nrows) {
            const int64_t row = first + lane;
            if (a.row_scale) {
                const float s = a.row_scale[row];
                mine = df_mul_f(mine, s);
                if (a.rpow == 2) mine = df_mul_f(mine, s);
            }
            store_y(y, row, df_mul(a.scale, mine));
        }
    }
}

// Copies the tile's sinogram band into shared memory.
template <typename YT>
__device__ __forceinline__ void stage_band(const BandView& bv, int tile, const YT* __restrict__ y, float2* band)
{
    const int32_t* blo = bv.band_lo + (int64_t)tile * bv.nk;
    const int total = bv.nk * kBandW;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int k = idx / kBandW;
        const int b = blo[k] + (idx - k * kBandW);
        band[idx] = b < bv.nb ? gather_x(y, (int64_t)k * bv.nb + b) : make_float2(0.0f, 0.0f);
    }
}

// Plain store of an A^T row total: OT = float2 writes the internal layout;
// OT = float writes the caller's row-major image.
__device__ __forceinline__ void store_pix(float2* out, int64_t t, int i, int j, int n, float2 v) { out[t] = v; }
__device__ __forceinline__ void store_pix(float* out, int64_t t, int i, int j, int n, float2 v)
{
    out[(int64_t)i * n + j] = df_to_float(v);
}

template <typename VT, typename YT, typename OT>
__global__ void __launch_bounds__(256) band_adj_kernel(BandView bv, const VT* __restrict__ val,
                                                       const YT* __restrict__ y, OT* __restrict__ out,
                                                       float2 scale)
{
    extern __shared__ float2 band[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ntiles = bv.tn * bv.tn;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        stage_band(bv, tile, y, band);
        __syncthreads();
        for (int g = 0; g < 2; ++g) {
            const int64_t first = (int64_t)tile * kTilePix + w * 32 + g * kRowsPerWarp;
            const float2 mine = band_group_dots<VT>(bv, val, first, band, lane);
            if (lane < kRowsPerWarp) {
                const int64_t t = first + lane;
                int i, j;
                tiled_coords(t, bv.tn, i, j);
                if (i < bv.n && j < bv.n) store_pix(out, t, i, j, bv.n, df_mul(scale, mine));
            }
        }
        __syncthreads();
    }
}

template <typename VT, int MODE>
__global__ void __launch_bounds__(256) band_op_kernel(BandView bv, const VT* __restrict__ val,
                                                      const float2* __restrict__ y, OpEpilogue a)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    extern __shared__ float2 band[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ntiles = bv.tn * bv.tn;
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        stage_band(bv, tile, y, band);
        __syncthreads();
        for (int g = 0; g < 2; ++g) {
            const int64_t first = (int64_t)tile * kTilePix + w * 32 + g * kRowsPerWarp;
            const float2 mine = band_group_dots<VT>(bv, val, first, band, lane);
            if (lane < kRowsPerWarp) {
                const int64_t t = first + lane;
                int i, j;
                tiled_coords(t, bv.tn, i, j);
                if (i < bv.n && j < bv.n) {
                    op_epilogue<MODE>(a, bv.n, bv.tn, t, i, j, mine, s0, c0, s1, c1);
                } else {
                    a.out[t] = df_zero();  // padding stays zero
                    if (MODE == 2) a.p_out[t] = df_zero();
                }
            }
        }
        __syncthreads();
    }
    op_finish<MODE>(a, s0, c0, s1, c1);
}

// Surrogate operator (Sec. 3.2, Eq. def_sparse_surr): (T p)_x = sum_d s(d)
// p_{x+d} over the window, translates outside the image dropped.  One thread
// per pixel; taps (double-float pairs) staged in shared memory.
template <int MODE>
__global__ void __launch_bounds__(256) stencil_op_df_kernel(OpEpilogue a, int n, int tn, int64_t npad,
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
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npad;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(p, tn, i, j);
        if (i >= n || j >= n) {
            a.out[p] = df_zero();  // padding stays zero
            if (MODE == 2) a.p_out[p] = df_zero();
            continue;
        }
        float hs = 0.0f, hc = 0.0f;
        for (int t = 0; t < ntaps; ++t) {
            const int ii = i + sd[t].x, jj = j + sd[t].y;
            if (ii >= 0 && ii < n && jj >= 0 && jj < n) acc_add(hs, hc, df_mul(sw[t], a.in[tiled_index(ii, jj, tn)]));
        }
        op_epilogue<MODE>(a, n, tn, p, i, j, acc_value(hs, hc), s0, c0, s1, c1);
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
int launch_csr(const ct_matrix* M, ValKind vk, const XT* x, YT* y, ProdArgs a, cudaStream_t st)
{
    const Csr& C = M->A;
    CsrView m{C.row_ptr, C.col, C.rows};
    const int grid = grid_for(M, C.rows, 8 * kRowsPerWarp, 8);
    if (vk == ValKind::F16)
        csr_df_kernel<__half, XT, YT><<<grid, 256, 0, st>>>(m, C.qval, x, y, a);
    else
        csr_df_kernel<float, XT, YT><<<grid, 256, 0, st>>>(m, C.val, x, y, a);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

BandView band_view(const ct_matrix* M)
{
    return BandView{M->At.row_ptr, M->At.col16, M->band_lo, M->g.n, M->tn, M->g.n_bins, M->n_kept};
}

size_t band_smem(const ct_matrix* M) { return (size_t)M->n_kept * kBandW * sizeof(float2); }

int band_grid(const ct_matrix* M) { return M->tn * M->tn; }

template <typename K>
int allow_smem(K kernel, size_t smem)
{
    if (smem > 48 * 1024)
        CT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return CT_OK;
}

template <typename VT, typename YT, typename OT>
int launch_band_adj(const ct_matrix* M, const VT* val, const YT* y, OT* out, float2 scale, cudaStream_t st)
{
    const size_t smem = band_smem(M);
    CT_CHECK(allow_smem(band_adj_kernel<VT, YT, OT>, smem));
    band_adj_kernel<VT, YT, OT><<<band_grid(M), 256, smem, st>>>(band_view(M), val, y, out, scale);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

template <typename VT, int MODE>
int launch_band_op(const ct_matrix* M, const VT* val, const float2* y, const OpEpilogue& ep, cudaStream_t st)
{
    const size_t smem = band_smem(M);
    CT_CHECK(allow_smem(band_op_kernel<VT, MODE>, smem));
    band_op_kernel<VT, MODE><<<band_grid(M), 256, smem, st>>>(band_view(M), val, y, ep);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

int launch_forward_df(const ct_matrix* M, ValKind vk, const float2* x, float2* y, int rpow,
                      const CgSlice* cg, const int32_t* gate, cudaStream_t st)
{
    ProdArgs a{vk == ValKind::F16 ? M->row_scale : nullptr, rpow, make_float2(1.0f, 0.0f), cg, gate};
    return launch_csr(M, vk, x, y, a, st);
}

int launch_adjoint_df(const ct_matrix* M, ValKind vk, const float2* y, float2* out, double scale,
                      cudaStream_t st)
{
    const float2 sc = df_from_double(scale);
    if (vk == ValKind::F16) return launch_band_adj(M, M->At.qval, y, out, sc, st);
    return launch_band_adj(M, M->At.val, y, out, sc, st);
}

int launch_forward_f32(const ct_matrix* M, ValKind vk, const float* x_tiled, float* y, cudaStream_t st)
{
    ProdArgs a{vk == ValKind::F16 ? M->row_scale : nullptr, 1, make_float2(1.0f, 0.0f), nullptr, nullptr};
    return launch_csr(M, vk, x_tiled, y, a, st);
}

int launch_adjoint_f32(const ct_matrix* M, ValKind vk, const float* y, const float2* y_scaled, float* x,
                       cudaStream_t st)
{
    const float2 one = make_float2(1.0f, 0.0f);
    if (vk == ValKind::F16) return launch_band_adj(M, M->At.qval, y_scaled, x, one, st);
    return launch_band_adj(M, M->At.val, y, x, one, st);
}

int launch_adjoint_op_df(const ct_matrix* M, ValKind vk, const float2* y, const OpEpilogue& ep,
                         cudaStream_t st)
{
    if (vk == ValKind::F16) {
        switch (ep.mode) {
        case 1: return launch_band_op<__half, 1>(M, M->At.qval, y, ep, st);
        case 2: return launch_band_op<__half, 2>(M, M->At.qval, y, ep, st);
        default: return launch_band_op<__half, 3>(M, M->At.qval, y, ep, st);
        }
    }
    switch (ep.mode) {
    case 1: return launch_band_op<float, 1>(M, M->At.val, y, ep, st);
    case 2: return launch_band_op<float, 2>(M, M->At.val, y, ep, st);
    default: return launch_band_op<float, 3>(M, M->At.val, y, ep, st);
    }
}

int launch_stencil_op_df(const ct_matrix* M, const Stencil* S, const OpEpilogue& ep, cudaStream_t st)
{
    const int n = M->g.n;
    const int grid = grid_for(M, M->npad, 256, 8);
    const int ntaps = S ? S->ntaps : 0;
    const size_t smem = (sizeof(int2) + sizeof(float2)) * (size_t)ntaps;
    const int32_t* d = S ? S->d : nullptr;
    const float* w = S ? S->w : nullptr;
    switch (ep.mode) {
    case 1: stencil_op_df_kernel<1><<<grid, 256, smem, st>>>(ep, n, M->tn, M->npad, d, w, ntaps); break;
    case 2: stencil_op_df_kernel<2><<<grid, 256, smem, st>>>(ep, n, M->tn, M->npad, d, w, ntaps); break;
    default: stencil_op_df_kernel<3><<<grid, 256, smem, st>>>(ep, n, M->tn, M->npad, d, w, ntaps); break;
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
