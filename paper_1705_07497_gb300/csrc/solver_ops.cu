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
// Both matrices are stored in SELL-32 (ct_internal.cuh): a warp takes one
// slice of 32 rows, one row per lane, and each lane walks its own row in
// 8-entry chunks with vector loads (the warp's loads for one chunk are 32
// contiguous chunks), two chunks in flight, accumulating in a double-float
// pair.  No shuffles or per-row reductions; lanes past their row's length
// stop loading.
//
// y = A x: slices of 32 consecutive rays; x is gathered from the tiled image
// layout (layout.cuh), where a run of pixels along any ray stays within a few
// cache lines.
//
// x = A^T y: one CTA of 8 warps per 16 x 16 image tile, one warp per slice
// of 32 pixels.  The CTA first copies the tile's sinogram band (W_k bins per
// kept angle, layout.cuh) into shared memory; every entry then reads its
// operand there through its 16-bit band index.  The operator epilogue runs
// with one pixel per lane.  Grid-wide dot products finish in the last block
// (reduce.cuh).  At 180 kept angles the double-float band is 30.75 KB, so
// seven CTAs fit an SM and a 512 x 512 image (1024 tiles) runs in one wave
// on 152 SMs.
#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "grad.cuh"
#include "layout.cuh"
#include "op_epilogue.cuh"
#include "reduce.cuh"
#include "slice_kernels.cuh"
#include "sparse_common.cuh"

namespace ct {
namespace {

constexpr int kAdjMinBlocks = 7;                    // CTAs per SM the register budget allows
constexpr int kAdjMinBlocksChunked = 5;             // the same when the band is staged in angle chunks
constexpr int kAdjFewBlocks = 4;                    // the fused kernel's alternative budgets (more registers)
constexpr int kAdjFewBlocksChunked = 3;
constexpr int kAdjAsyncBlocks = 3;                  // single-chunk band with the asynchronous-copy ring
constexpr int kOp2Threads = 128;                    // two pixel rows per lane: four warps per tile
constexpr int kOp2Blocks = 7;

// Offset of the asynchronous-copy ring after a band of `slots` double-float values.
__host__ __device__ inline size_t ring_offset(int slots) { return ((size_t)slots * sizeof(float2) + 15) & ~(size_t)15; }

// y = scale * A x: one block per slice of 32 rays (see fwd_slice).
template <typename VT, typename XT, typename YT, int U>
__global__ void __launch_bounds__(kFwdWarps * 32) sell_fwd_kernel(SellView m, const int32_t* __restrict__ col,
                                                                  const VT* __restrict__ val,
                                                                  const XT* __restrict__ x, YT* __restrict__ y,
                                                                  ProdArgs a)
{
    if (a.gate && *a.gate) return;
    if (a.cg && !a.cg->active) return;
    const int64_t nslices = (m.rows + kSliceRows - 1) / kSliceRows;
    for (int64_t s = blockIdx.x; s < nslices; s += gridDim.x) fwd_slice<VT, XT, YT, U>(m, col, val, x, y, a, s);
}

template <typename VT, typename YT, typename OT, bool CHUNKED>
__global__ void __launch_bounds__(kAdjWarps * 32, CHUNKED ? kAdjMinBlocksChunked : kAdjMinBlocks)
    band_adj_kernel(BandView bv, const VT* __restrict__ val, const YT* __restrict__ y, OT* __restrict__ out,
                    float2 scale)
{
    extern __shared__ __align__(16) unsigned char smem[];
    YT* band = reinterpret_cast<YT*>(smem);
    const int ntiles = bv.tn * bv.tn;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int64_t t;
        float2 d;
        if (CHUNKED) {
            t = (int64_t)tile * kTilePix + threadIdx.x;
            d = band_dot_chunked<VT>(bv, val, tile, y, band, t);
        } else {
            stage_band(bv, tile, y, band);
            d = band_dot<VT>(bv, val, tile, band, t);
        }
        int i, j;
        tiled_coords(t, bv.tn, i, j);
        if (i < bv.n && j < bv.n) store_pix(out, t, i, j, bv.n, df_mul(scale, d));
        __syncthreads();
    }
}

template <typename VT, int MODE, bool CHUNKED, int MINB>
__global__ void __launch_bounds__(kAdjWarps * 32, MINB)
    band_op_kernel(BandView bv, const VT* __restrict__ val, const float2* __restrict__ y, OpEpilogue a)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* band = reinterpret_cast<float2*>(smem);
    const int ntiles = bv.tn * bv.tn;
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int64_t t;
        float2 d;
        if (CHUNKED) {
            t = (int64_t)tile * kTilePix + threadIdx.x;
            d = band_dot_chunked<VT>(bv, val, tile, y, band, t);
        } else {
            stage_band(bv, tile, y, band);
            constexpr int PF = MINB == kAdjAsyncBlocks ? 2 : (MINB < kAdjMinBlocks ? 1 : 0);
            uint4* ring = PF == 2 ? reinterpret_cast<uint4*>(smem + ring_offset(bv.slots)) : nullptr;
            d = band_dot<VT, float2, PF>(bv, val, tile, band, t, ring);
        }
        int i, j;
        tiled_coords(t, bv.tn, i, j);
        if (i < bv.n && j < bv.n) {
            op_epilogue<MODE>(a, bv.n, bv.tn, t, i, j, d, s0, c0, s1, c1);
        } else {
            a.out[t] = df_zero();  // padding stays zero
            if (MODE == 2) a.p_out[t] = df_zero();
        }
        __syncthreads();
    }
    op_finish<MODE>(a, s0, c0, s1, c1);
}

// The same product and epilogue with two pixel rows per lane: a CTA of four
// warps per tile, warp w taking pixel slices 2w and 2w + 1, so that at seven
// CTAs per SM (72 registers per thread) a 512 x 512 image's 1024 tiles run in
// one wave with two rows in flight per lane.  Every row sum, epilogue and
// reduction is grouped as in band_op_kernel (grid_reduce_last_pair), so both
// give the same bits.  Single-chunk bands only.
template <typename VT, int MODE>
__global__ void __launch_bounds__(kOp2Threads, kOp2Blocks)
    band_op2_kernel(BandView bv, const VT* __restrict__ val, const float2* __restrict__ y, OpEpilogue a)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* band = reinterpret_cast<float2*>(smem);
    const int ntiles = bv.tn * bv.tn;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float s0a = 0.0f, c0a = 0.0f, s1a = 0.0f, c1a = 0.0f, s0b = 0.0f, c0b = 0.0f, s1b = 0.0f, c1b = 0.0f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        stage_band(bv, tile, y, band);
        const int64_t ta = (int64_t)tile * kTilePix + (2 * w) * kSliceRows + lane, tb = ta + kSliceRows;
        float2 da, db;
        row_pair_walk<VT>(bv.col16, val, bv.sp[ta >> 5] + lane * kChunk, (bv.len[ta] + kChunk - 1) / kChunk,
                          bv.sp[tb >> 5] + lane * kChunk, (bv.len[tb] + kChunk - 1) / kChunk,
                          BandGather<float2>{band}, da, db);
        int i, j;
        tiled_coords(ta, bv.tn, i, j);
        if (i < bv.n && j < bv.n) {
            op_epilogue<MODE>(a, bv.n, bv.tn, ta, i, j, da, s0a, c0a, s1a, c1a);
        } else {
            a.out[ta] = df_zero();
            if (MODE == 2) a.p_out[ta] = df_zero();
        }
        tiled_coords(tb, bv.tn, i, j);
        if (i < bv.n && j < bv.n) {
            op_epilogue<MODE>(a, bv.n, bv.tn, tb, i, j, db, s0b, c0b, s1b, c1b);
        } else {
            a.out[tb] = df_zero();
            if (MODE == 2) a.p_out[tb] = df_zero();
        }
        __syncthreads();
    }
    float2 va[2] = {acc_value(s0a, c0a), acc_value(s1a, c1a)};
    float2 vb[2] = {acc_value(s0b, c0b), acc_value(s1b, c1b)};
    double tot[2];
    if (grid_reduce_last_pair<2>(va, vb, a.partials, a.counter, tot)) {
        if (MODE == 1) cg_after_pq(*a.cg, tot[0]);
        if (MODE == 2) cg_after_residual(*a.cg, tot[0], tot[1], a.tol);
        if (MODE == 3) a.cg->rr = tot[0];
    }
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
int launch_fwd(const ct_matrix* M, ValKind vk, const XT* x, YT* y, ProdArgs a, cudaStream_t st)
{
    const Sell& C = M->A;
    const SellView m{C.slice_ptr, C.row_len, C.rows};
    // one block per slice: the block scheduler evens out slices of unequal
    // length across SMs
    const int64_t nslices = (C.rows + kSliceRows - 1) / kSliceRows;
    const int grid = (int)(nslices < (1 << 30) ? nslices : (1 << 30));
    const int warps = M->fwd_warps > 0 ? M->fwd_warps : kFwdWarps;
    const int unroll = M->fwd_unroll > 0 ? M->fwd_unroll : kFwdUnroll;
#define CT_FWD(VT, VAL, U) sell_fwd_kernel<VT, XT, YT, U><<<grid, warps * 32, 0, st>>>(m, C.col, VAL, x, y, a)
    if (vk == ValKind::F16) {
        switch (unroll) {
        case 2: CT_FWD(__half, C.qval, 2); break;
        case 4: CT_FWD(__half, C.qval, 4); break;
        case 16: CT_FWD(__half, C.qval, 16); break;
        default: CT_FWD(__half, C.qval, 8); break;
        }
    } else {
        switch (unroll) {
        case 2: CT_FWD(float, C.val, 2); break;
        case 4: CT_FWD(float, C.val, 4); break;
        case 16: CT_FWD(float, C.val, 16); break;
        default: CT_FWD(float, C.val, 8); break;
        }
    }
#undef CT_FWD
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

BandView band_view(const ct_matrix* M)
{
    return BandView{M->At.slice_ptr, M->At.row_len, M->At.col16, M->band_lo, M->band_off, M->band_chunk,
                    (int)M->h_band_chunk.size() - 1, M->band_total, M->g.n, M->tn, M->g.n_bins, M->n_kept};
}

size_t band_smem(const ct_matrix* M, size_t elem) { return band_bytes(M->band_chunk_slots, elem); }

bool band_chunked(const ct_matrix* M) { return M->h_band_chunk.size() > 2; }

int band_grid(const ct_matrix* M) { return M->tn * M->tn; }

template <typename K>
int allow_smem(K kernel, size_t smem)
{
    if (smem > 48 * 1024)
        CT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return CT_OK;
}

template <typename VT, typename YT, typename OT, bool CHUNKED>
int launch_band_adj_t(const ct_matrix* M, const VT* val, const YT* y, OT* out, float2 scale, cudaStream_t st)
{
    const size_t smem = band_smem(M, sizeof(YT));
    CT_CHECK(allow_smem(band_adj_kernel<VT, YT, OT, CHUNKED>, smem));
    band_adj_kernel<VT, YT, OT, CHUNKED><<<band_grid(M), kAdjWarps * 32, smem, st>>>(band_view(M), val, y, out, scale);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

template <typename VT, typename YT, typename OT>
int launch_band_adj(const ct_matrix* M, const VT* val, const YT* y, OT* out, float2 scale, cudaStream_t st)
{
    if (band_chunked(M)) return launch_band_adj_t<VT, YT, OT, true>(M, val, y, out, scale, st);
    return launch_band_adj_t<VT, YT, OT, false>(M, val, y, out, scale, st);
}

template <typename VT, int MODE, bool CHUNKED, int MINB>
int launch_band_op_t(const ct_matrix* M, const VT* val, const float2* y, const OpEpilogue& ep, cudaStream_t st)
{
    size_t smem = band_smem(M, sizeof(float2));
    if (!CHUNKED && MINB == kAdjAsyncBlocks) smem = ring_offset(M->band_chunk_slots) + async_ring_bytes(kAdjWarps * 32);
    CT_CHECK(allow_smem(band_op_kernel<VT, MODE, CHUNKED, MINB>, smem));
    band_op_kernel<VT, MODE, CHUNKED, MINB><<<band_grid(M), kAdjWarps * 32, smem, st>>>(band_view(M), val, y, ep);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// The fused kernel comes in several budgets per band form: sized for
// kAdjMinBlocks (kAdjMinBlocksChunked) CTAs per SM; for fewer CTAs with more
// registers per thread (the next chunk's loads issued before this chunk's
// gathers); and, for a single-chunk band, kAdjAsyncBlocks CTAs whose lanes
// copy two chunks ahead into shared memory.  Every form accumulates each row
// in the same order, so every result bit is the same.
template <typename VT, int MODE>
int launch_band_op2(const ct_matrix* M, const VT* val, const float2* y, const OpEpilogue& ep, cudaStream_t st)
{
    const size_t smem = band_smem(M, sizeof(float2));
    CT_CHECK(allow_smem(band_op2_kernel<VT, MODE>, smem));
    band_op2_kernel<VT, MODE><<<band_grid(M), kOp2Threads, smem, st>>>(band_view(M), val, y, ep);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

template <typename VT, int MODE>
int launch_band_op(const ct_matrix* M, const VT* val, const float2* y, const OpEpilogue& ep, cudaStream_t st)
{
    const int ctas = M->op_ctas;
    if (M->op_pixels == 2 && !band_chunked(M)) return launch_band_op2<VT, MODE>(M, val, y, ep, st);
    if (band_chunked(M)) {
        if (ctas == kAdjFewBlocksChunked) return launch_band_op_t<VT, MODE, true, kAdjFewBlocksChunked>(M, val, y, ep, st);
        return launch_band_op_t<VT, MODE, true, kAdjMinBlocksChunked>(M, val, y, ep, st);
    }
    if (ctas == kAdjFewBlocks) return launch_band_op_t<VT, MODE, false, kAdjFewBlocks>(M, val, y, ep, st);
    if (ctas == kAdjAsyncBlocks) return launch_band_op_t<VT, MODE, false, kAdjAsyncBlocks>(M, val, y, ep, st);
    return launch_band_op_t<VT, MODE, false, kAdjMinBlocks>(M, val, y, ep, st);
}

}  // namespace

int launch_forward_df(const ct_matrix* M, ValKind vk, const float2* x, float2* y, int rpow,
                      const CgSlice* cg, const int32_t* gate, cudaStream_t st)
{
    ProdArgs a{vk == ValKind::F16 ? M->row_scale : nullptr, rpow, make_float2(1.0f, 0.0f), cg, gate};
    return launch_fwd(M, vk, x, y, a, st);
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
    return launch_fwd(M, vk, x_tiled, y, a, st);
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
