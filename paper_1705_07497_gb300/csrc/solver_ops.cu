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
#include "sparse_common.cuh"

namespace ct {
namespace {

constexpr int kFwdWarps = 8;   // warps per block (= per slice of rays) of y = A x
constexpr int kFwdUnroll = 8;  // chunks each lane of y = A x keeps in flight (untuned default)
constexpr int kAdjWarps = kTilePix / kSliceRows;  // warps per CTA of x = A^T y (one per pixel slice)
constexpr int kAdjMinBlocks = 7;                    // CTAs per SM the register budget allows
constexpr int kAdjMinBlocksChunked = 5;             // the same when the band is staged in angle chunks
constexpr int kAdjFewBlocks = 4;                    // the fused kernel's alternative budgets (more registers)
constexpr int kAdjFewBlocksChunked = 3;
constexpr int64_t kStep = kSliceRows * kChunk;      // entries between a lane's consecutive chunks

// Bytes of a staged band of `slots` values.
__host__ __device__ inline size_t band_bytes(int slots, size_t elem) { return (size_t)slots * elem; }

struct BandView {
    const int64_t* sp;    // slice offsets of A^T
    const int32_t* len;   // row lengths of A^T
    const uint16_t* col16;
    const int32_t* band_lo;   // [tiles][nk] first bin of each band
    const int32_t* band_off;  // [nk+1] slot offsets of the angles
    const int32_t* chunk_k;   // [nchunks+1] first kept angle of each staged band chunk
    int nchunks;
    int slots;                // band_off[nk]
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

__device__ __forceinline__ void load8_col(const int32_t* p, int64_t k, int (&c)[8])
{
    const int4 a = __ldcs(reinterpret_cast<const int4*>(p + k));
    const int4 b = __ldcs(reinterpret_cast<const int4*>(p + k + 4));
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
}

__device__ __forceinline__ void load8_col(const uint16_t* p, int64_t k, int (&c)[8])
{
    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p + k));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        c[2 * t] = (int)(w[t] & 0xffffu);
        c[2 * t + 1] = (int)(w[t] >> 16);
    }
}

// Operand of an entry: a gathered vector element (A) or a staged band value (A^T).
template <typename XT>
struct Gather {
    const XT* x;
    __device__ __forceinline__ float2 operator()(int c) const { return gather_x(x, c); }
};
// (shared memory: plain loads)
__device__ __forceinline__ float2 band_value(const float* band, int c) { return make_float2(band[c], 0.0f); }
__device__ __forceinline__ float2 band_value(const float2* band, int c) { return band[c]; }
template <typename BT>
struct BandGather {
    const BT* band;
    __device__ __forceinline__ float2 operator()(int c) const { return band_value(band, c); }
};

// Part of the dot product of the lane's row (entry 0 at `base`, nch chunks)
// with the operands `g` gives: chunk pairs (c, c+1) for c = c_first,
// c_first + c_step, ...; both chunks' loads are issued before either's
// arithmetic.  Accumulates into the double-float pair (hs, hc).
template <typename VT, typename CT, typename G>
__device__ __forceinline__ void row_part(const CT* __restrict__ col, const VT* __restrict__ val, int64_t base,
                                         int nch, int c_first, int c_step, const G& g, float& hs, float& hc)
{
    for (int c = c_first; c < nch; c += c_step) {
        const int64_t p = base + c * kStep;
        if (c + 1 < nch) {
            int c0[8], c1[8];
            float v0[8], v1[8];
            load8_col(col, p, c0);
            load8_col(col, p + kStep, c1);
            Vals<VT>::load8(val, p, v0);
            Vals<VT>::load8(val, p + kStep, v1);
            float2 x0[8], x1[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) x0[t] = g(c0[t]);
#pragma unroll
            for (int t = 0; t < 8; ++t) x1[t] = g(c1[t]);
#pragma unroll
            for (int t = 0; t < 8; ++t) acc_fma(hs, hc, v0[t], x0[t]);
#pragma unroll
            for (int t = 0; t < 8; ++t) acc_fma(hs, hc, v1[t], x1[t]);
        } else {
            int c0[8];
            float v0[8];
            load8_col(col, p, c0);
            Vals<VT>::load8(val, p, v0);
            float2 x0[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) x0[t] = g(c0[t]);
#pragma unroll
            for (int t = 0; t < 8; ++t) acc_fma(hs, hc, v0[t], x0[t]);
        }
    }
}

struct ProdArgs {
    const float* row_scale;  // FP16 storage: multiply rows by s^rpow
    int rpow;
    float2 scale;
    const CgSlice* cg;
    const int32_t* gate;
};

// y = scale * A x (x in the tiled layout).  A block takes a slice of 32 rays
// and each of its warps four adjacent rays of it: the warp's lanes are four
// groups of eight, one group per ray, and at chunk c lane e of a group takes
// entry 8c + e of its ray.  In the SELL-32 layout the four rays' chunk c is
// 32 contiguous entries, so every load of the warp is one 128-byte run, and a
// gather of x touches the pixels of four neighbouring parallel rays over
// eight consecutive entries: a compact patch of the image, about 12 distinct
// 32-byte sectors per gather instead of about 20 when each lane walks its own
// ray (counted on the 512 x 512 matrix).  Each lane sums its entries in order
// (U chunks in flight per step); the eight partial sums of a ray are combined
// by a fixed butterfly.  With fewer warps than 8 a warp takes several groups
// of the slice; results do not depend on the warp count or on U.
template <typename VT, typename XT, typename YT, int U>
__global__ void __launch_bounds__(kFwdWarps * 32) sell_fwd_kernel(SellView m, const int32_t* __restrict__ col,
                                                                  const VT* __restrict__ val,
                                                                  const XT* __restrict__ x, YT* __restrict__ y,
                                                                  ProdArgs a)
{
    if (a.gate && *a.gate) return;
    if (a.cg && !a.cg->active) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int e8 = lane & 7;
    const int64_t nslices = (m.rows + kSliceRows - 1) / kSliceRows;
    for (int64_t s = blockIdx.x; s < nslices; s += gridDim.x) {
        for (int grp = w; grp < kSliceRows / 4; grp += nw) {
            const int64_t row = s * kSliceRows + grp * 4 + (lane >> 3);
            const int len = row < m.rows ? __ldg(m.len + row) : 0;
            const int nch = (len + kChunk - 1) / kChunk;
            int nmax = nch;
#pragma unroll
            for (int o = 8; o < 32; o <<= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
            const int64_t base = __ldg(m.sp + s) + grp * 32 + lane;
            float hs = 0.0f, hc = 0.0f;
            for (int c0 = 0; c0 < nmax; c0 += U) {
                int cc[U];
                float vv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t p = base + (int64_t)(c0 + u) * (kSliceRows * kChunk);
                    cc[u] = c0 + u < nch ? __ldcs(col + p) : -1;
                    vv[u] = c0 + u < nch ? Vals<VT>::one(val, p) : 0.0f;
                }
                float2 xx[U];
#pragma unroll
                for (int u = 0; u < U; ++u) xx[u] = cc[u] >= 0 ? gather_x(x, cc[u]) : df_zero();
#pragma unroll
                for (int u = 0; u < U; ++u) acc_fma(hs, hc, vv[u], xx[u]);
            }
            float2 d = acc_value(hs, hc);
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                float2 t;
                t.x = __shfl_xor_sync(0xffffffffu, d.x, o);
                t.y = __shfl_xor_sync(0xffffffffu, d.y, o);
                d = (e8 & o) ? df_add(t, d) : df_add(d, t);
            }
            if (e8 == 0 && row < m.rows) {
                if (a.row_scale) {
                    const float sc = a.row_scale[row];
                    d = df_mul_f(d, sc);
                    if (a.rpow == 2) d = df_mul_f(d, sc);
                }
                store_y(y, row, df_mul(a.scale, d));
            }
        }
    }
}

// Asynchronous 4- or 8-byte global -> shared copy; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copies the tile's whole sinogram band into shared memory: every angle's W_k
// bins, one warp per angle and one lane per bin, all copies in flight at
// once; bins past the detector read as zero.  Ends with the block
// synchronised.
template <typename YT>
__device__ __forceinline__ void stage_band(const BandView& bv, int tile, const YT* __restrict__ y, YT* band)
{
    const int32_t* blo = bv.band_lo + (int64_t)tile * bv.nk;
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int k = threadIdx.x >> 5; k < bv.nk; k += nwarps) {
        const int off = __ldg(bv.band_off + k);
        if (lane < __ldg(bv.band_off + k + 1) - off) {
            const int b = __ldg(blo + k) + lane;
            const bool in = b < bv.nb;
            cp_async(band + off + lane, y + (in ? (int64_t)k * bv.nb + b : 0), (int)sizeof(YT),
                     in ? (int)sizeof(YT) : 0);
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

// Copies angles [k0, k1) of the tile's sinogram band into shared memory
// (slot off_k0 at band[0]): every angle's W_k bins, one warp per angle and one
// lane per bin, all copies in flight at once; bins past the detector read as
// zero.  Ends with the block synchronised.
template <typename YT>
__device__ __forceinline__ void stage_band_range(const BandView& bv, int tile, const YT* __restrict__ y, YT* band,
                                                 int k0, int k1)
{
    const int32_t* blo = bv.band_lo + (int64_t)tile * bv.nk;
    const int base = __ldg(bv.band_off + k0);
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int k = k0 + (threadIdx.x >> 5); k < k1; k += nwarps) {
        const int off = __ldg(bv.band_off + k);
        if (lane < __ldg(bv.band_off + k + 1) - off) {
            const int b = __ldg(blo + k) + lane;
            const bool in = b < bv.nb;
            cp_async(band + (off - base) + lane, y + (in ? (int64_t)k * bv.nb + b : 0), (int)sizeof(YT),
                     in ? (int)sizeof(YT) : 0);
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

// The lane's row of A^T against a band staged chunk by chunk (many angles):
// for each angle chunk, stage it, then walk the row's 8-entry chunks from the
// lane's position until one reaches past the chunk's slots; a chunk that
// straddles two band chunks is walked in both, each time with the other's
// entries masked.  Every lane of the CTA takes part in every staging.
template <typename VT, typename YT>
__device__ __forceinline__ float2 band_dot_chunked(const BandView& bv, const VT* __restrict__ val, int tile,
                                                   const YT* __restrict__ y, YT* band, int64_t t)
{
    const int lane = threadIdx.x & 31;
    const int len = bv.len[t];
    const int nch = (len + kChunk - 1) / kChunk;
    const int64_t base = bv.sp[t >> 5] + lane * kChunk;
    float hs = 0.0f, hc = 0.0f;
    int c = 0;
    for (int j = 0; j < bv.nchunks; ++j) {
        const int k0 = __ldg(bv.chunk_k + j), k1 = __ldg(bv.chunk_k + j + 1);
        const int lo = __ldg(bv.band_off + k0), hi = __ldg(bv.band_off + k1);
        stage_band_range(bv, tile, y, band, k0, k1);
        // two 8-entry chunks per step, both loads issued first
        while (c < nch) {
            const int64_t p = base + (int64_t)c * kStep;
            const bool two = c + 1 < nch;
            int c0[8], c1[8];
            float v0[8], v1[8];
            load8_col(bv.col16, p, c0);
            Vals<VT>::load8(val, p, v0);
            if (two) {
                load8_col(bv.col16, p + kStep, c1);
                Vals<VT>::load8(val, p + kStep, v1);
            }
            bool beyond = false;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool in = c0[u] >= lo && c0[u] < hi;
                beyond |= c0[u] >= hi;
                acc_fma(hs, hc, in ? v0[u] : 0.0f, band_value(band, in ? c0[u] - lo : 0));
            }
            if (beyond) break;  // the rest of chunk c belongs to a later band chunk
            ++c;
            if (!two) break;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool in = c1[u] >= lo && c1[u] < hi;
                beyond |= c1[u] >= hi;
                acc_fma(hs, hc, in ? v1[u] : 0.0f, band_value(band, in ? c1[u] - lo : 0));
            }
            if (beyond) break;
            ++c;
        }
        __syncthreads();  // every lane done with this band chunk before the next staging
    }
    return acc_value(hs, hc);
}

// Plain store of an A^T row total: OT = float2 writes the internal layout;
// OT = float writes the caller's row-major image.
__device__ __forceinline__ void store_pix(float2* out, int64_t t, int i, int j, int n, float2 v) { out[t] = v; }
__device__ __forceinline__ void store_pix(float* out, int64_t t, int i, int j, int n, float2 v)
{
    out[(int64_t)i * n + j] = df_to_float(v);
}

// Dot product of A^T row t = tile * 256 + warp * 32 + lane with the staged band.
template <typename VT, typename BT>
__device__ __forceinline__ float2 band_dot(const BandView& bv, const VT* __restrict__ val, int tile,
                                           const BT* __restrict__ band, int64_t& t)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    t = (int64_t)tile * kTilePix + w * kSliceRows + lane;
    const int len = bv.len[t];
    float hs = 0.0f, hc = 0.0f;
    row_part<VT>(bv.col16, val, bv.sp[t >> 5] + lane * kChunk, (len + kChunk - 1) / kChunk, 0, 2,
                 BandGather<BT>{band}, hs, hc);
    return acc_value(hs, hc);
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
            d = band_dot<VT>(bv, val, tile, band, t);
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
    const size_t smem = band_smem(M, sizeof(float2));
    CT_CHECK(allow_smem(band_op_kernel<VT, MODE, CHUNKED, MINB>, smem));
    band_op_kernel<VT, MODE, CHUNKED, MINB><<<band_grid(M), kAdjWarps * 32, smem, st>>>(band_view(M), val, y, ep);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// The fused kernel comes in two register budgets per band form: sized for
// kAdjMinBlocks (kAdjMinBlocksChunked) CTAs per SM, or for fewer CTAs with
// more registers per thread; the code, and so every result bit, is the same.
template <typename VT, int MODE>
int launch_band_op(const ct_matrix* M, const VT* val, const float2* y, const OpEpilogue& ep, cudaStream_t st)
{
    const int ctas = M->op_ctas;
    if (band_chunked(M)) {
        if (ctas == kAdjFewBlocksChunked) return launch_band_op_t<VT, MODE, true, kAdjFewBlocksChunked>(M, val, y, ep, st);
        return launch_band_op_t<VT, MODE, true, kAdjMinBlocksChunked>(M, val, y, ep, st);
    }
    if (ctas == kAdjFewBlocks) return launch_band_op_t<VT, MODE, false, kAdjFewBlocks>(M, val, y, ep, st);
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
