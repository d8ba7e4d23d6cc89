// Batched solvers: many slices sharing one geometry (vectors [len][B], the
// slice index innermost).  The sparse products become SpMMs with the slices
// as the dense inner dimension: a warp owns one row for a chunk of 32 slices
// (one slice per lane), reads the row's entries 32 at a time (four 8-entry
// chunks of the SELL layout), stages them in shared memory and broadcasts them, so each lane gathers the
// 32 contiguous slice values of every column it meets.  The blocks of all
// chunks of a row range are adjacent in launch order, so the matrix is read
// from HBM once and reused from L2 by the other chunks.
//
// Arithmetic is double-float throughout (dfloat.cuh), like the single-slice
// path.  Every reduction (per slice) writes deterministic block partials that
// a per-slice finalize kernel sums in a fixed order before applying the CG or
// split-Bregman scalar update (reduce.cuh).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "reduce.cuh"
#include "sparse_common.cuh"

namespace ct {
namespace {

constexpr int kWarps = 8;  // warps per block

__device__ __forceinline__ float2 ld_x(const float* x, int64_t i) { return make_float2(__ldg(x + i), 0.0f); }
__device__ __forceinline__ float2 ld_x(const float2* x, int64_t i) { return __ldg(x + i); }
__device__ __forceinline__ void st_y(float* y, int64_t i, float2 v) { y[i] = df_to_float(v); }
__device__ __forceinline__ void st_y(float2* y, int64_t i, float2 v) { y[i] = v; }

struct Grid2 {
    int rb;      // row blocks per slice chunk
    int chunks;  // ceil(B / (32 * spl))
    int spl;     // slices per lane in the sparse products (1, or 2 for batches >= 64)
};

// Block (rb, chunk) of a 1-D grid of rb * chunks blocks, chunk-major: the
// resident blocks work on one chunk of 32 slices at a time, so the chunk's
// slice vectors stay in L2 while the matrix streams.
__device__ __forceinline__ void block_coords(int chunks, int& rb, int& chunk)
{
    const int G = (int)gridDim.x / chunks;
    rb = (int)blockIdx.x % G;
    chunk = (int)blockIdx.x / G;
}

// Lanes of a warp over (row, slice).  B >= 32: the warp takes one row for 32
// slices (slice chunk * 32 + lane).  B < 32: the warp splits into 32 / W
// sub-groups of W lanes (W = the power of two >= B), one row per sub-group,
// slice = lane % W, so that small batches keep the lanes busy.
struct LaneMap {
    int W;    // lanes per row
    int g;    // this lane's sub-group
    int b;    // this lane's slice
    int rpw;  // rows per warp
};

__host__ __device__ inline int lanes_per_row(int B)
{
    if (B >= 32) return 32;
    int W = 1;
    while (W < B) W <<= 1;
    return W;
}

__device__ __forceinline__ LaneMap lane_map(int B, int chunk, int lane)
{
    LaneMap m;
    m.W = lanes_per_row(B);
    m.g = lane / m.W;
    m.b = B >= 32 ? chunk * 32 + lane : lane % m.W;
    m.rpw = 32 / m.W;
    return m;
}

// Slices per lane of the sparse products: two adjacent slices (one 16-byte
// gather of their double-float values) once a batch fills two warps' lanes.
__host__ __device__ inline int slices_per_lane(int B) { return (B >= 64 && B % 2 == 0) ? 2 : 1; }

// Lane map of the sparse products: SPL slices per lane, chunks of 32 * SPL
// slices; HALF (SPL = 2): half-warps of 16 lanes take one row each for a
// chunk of 32 slices, so that a chunk's gathered vectors (N^2 x 32 slices)
// stay within L2 while the matrix streams past them once per chunk.
template <int SPL, bool HALF = false>
__device__ __forceinline__ LaneMap lane_map_spl(int B, int chunk, int lane)
{
    if (SPL == 1) return lane_map(B, chunk, lane);
    LaneMap m;
    if (HALF) {
        m.W = 16;
        m.g = lane >> 4;
        m.b = chunk * 32 + SPL * (lane & 15);
        m.rpw = 2;
        return m;
    }
    m.W = 32;
    m.g = 0;
    m.b = chunk * 32 * SPL + SPL * lane;
    m.rpw = 1;
    return m;
}

__host__ __device__ inline int chunk_slices(int spl, bool half) { return half ? 32 : 32 * spl; }

// First row of the warp (its sub-group 0) and the stride between a warp's rows.
__device__ __forceinline__ int64_t warp_row0(int rb, int w, const LaneMap& m)
{
    return ((int64_t)rb * kWarps + w) * m.rpw;
}
__device__ __forceinline__ int64_t row_stride(int G, const LaneMap& m) { return (int64_t)G * kWarps * m.rpw; }

__device__ __forceinline__ bool slice_live(int b, int B, const CgSlice* cg, const SbSlice* sb)
{
    if (b >= B) return false;
    if (cg && !cg[b].active) return false;
    if (sb && sb[b].stopped) return false;
    return true;
}

// Sum over the block's warps of each lane's values (fixed order), written as
// the block's partials for slices chunk * 32 * SPL + SPL * lane + s:
// partials[(q*B + b)*G + rb].  With sub-groups (W < 32) the lanes of one
// slice are first combined by a fixed butterfly, and lanes b < B write.
template <int NQ, int SPL = 1>
__device__ __forceinline__ void block_partials(float2 (&v)[NQ][SPL], float2* partials, int B, int G, int rb,
                                               int chunk, int W)
{
    __shared__ float2 red[NQ][kWarps][32 * SPL];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = W; o < 32; o <<= 1) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int e = 0; e < SPL; ++e) {
                float2 t;
                t.x = __shfl_xor_sync(0xffffffffu, v[q][e].x, o);
                t.y = __shfl_xor_sync(0xffffffffu, v[q][e].y, o);
                v[q][e] = df_add(v[q][e], t);
            }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int e = 0; e < SPL; ++e) red[q][w][SPL * lane + e] = v[q][e];
    __syncthreads();
    if (w == 0 && lane < W) {
#pragma unroll
        for (int e = 0; e < SPL; ++e) {
            const int b = chunk * 32 * SPL + SPL * lane + e;
            if (b >= B) continue;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                float2 s = red[q][0][SPL * lane + e];
                for (int k = 1; k < kWarps; ++k) s = df_add(s, red[q][k][SPL * lane + e]);
                partials[((size_t)q * B + b) * G + rb] = s;
            }
        }
    }
}

struct BProd {
    const float* row_scale;
    int rpow;
    float2 scale;
    const CgSlice* cg;
    const SbSlice* sb;
};

// Column of an entry: A stores internal pixel indices; A^T stores band-local
// indices off_k + w that map to sinogram row k * n_bins + band_lo(tile, k) + w.
struct ColMap {
    const int32_t* col;       // A
    const uint16_t* col16;    // A^T (band-local)
    const int32_t* band_lo;
    const int32_t* band_off;
    const uint16_t* band_angle;
    int nb, nk;
};

__device__ __forceinline__ int map_col(const ColMap& cm, int64_t row, int64_t k)
{
    if (cm.col) return __ldcs(cm.col + k);
    const int c = (int)__ldcs(cm.col16 + k);
    const int a = __ldg(cm.band_angle + c);
    return a * cm.nb + __ldg(cm.band_lo + (row >> 8) * cm.nk + a) + (c - __ldg(cm.band_off + a));
}

// Output position of (row, slice): internal layout, or for USER_OUT the
// caller's row-major image (rows are internal pixel indices; padding skipped).
struct OutMap {
    int user;  // 1: rows are pixels written in the caller's layout
    int n, tn;
};

// Stages up to W entries of each sub-group's row (j0 .. j0 + W - 1) in the
// warp's shared buffer: lane (g, t) loads entry j0 + t of its sub-group's row.
template <typename VT>
__device__ __forceinline__ void stage_entries(const ColMap& cm, const VT* __restrict__ val, int64_t row,
                                              int64_t base, int len, int j0, int t, int2* stage)
{
    int2 e = make_int2(0, 0);
    if (j0 + t < len) {
        const int64_t k = chunk_pos(base, j0 + t);
        e = make_int2(map_col(cm, row, k), __float_as_int(Vals<VT>::one(val, k)));
    }
    *stage = e;
}

// Loads of SPL adjacent slices' values of one vector element: double-float
// (16 bytes for two slices) or FP32 (8 bytes for two), as double-float pairs.
template <int SPL>
__device__ __forceinline__ void ld_xs(const float2* x, int64_t i, float2 (&o)[SPL])
{
    if (SPL == 1) {
        o[0] = __ldg(x + i);
    } else {
        const float4 v = __ldg(reinterpret_cast<const float4*>(x + i));
        o[0] = make_float2(v.x, v.y);
        o[SPL - 1] = make_float2(v.z, v.w);
    }
}
template <int SPL>
__device__ __forceinline__ void ld_xs(const float* x, int64_t i, float2 (&o)[SPL])
{
    if (SPL == 1) {
        o[0] = make_float2(__ldg(x + i), 0.0f);
    } else {
        const float2 v = __ldg(reinterpret_cast<const float2*>(x + i));
        o[0] = make_float2(v.x, 0.0f);
        o[SPL - 1] = make_float2(v.y, 0.0f);
    }
}

// acc[e] += sum over the cnt staged entries of val * X[col][b + e], U entries
// per step (U gathers in flight); every U gives the same bits.
template <typename XT, int U, int SPL>
__device__ __forceinline__ void staged_dot(const int2* st, int cnt, const XT* __restrict__ x, int B, int b,
                                           float (&hs)[SPL], float (&hc)[SPL])
{
    int t = 0;
    for (; t + U <= cnt; t += U) {
        int2 e[U];
        float2 xv[U][SPL];
#pragma unroll
        for (int u = 0; u < U; ++u) e[u] = st[t + u];
#pragma unroll
        for (int u = 0; u < U; ++u) ld_xs<SPL>(x, (int64_t)e[u].x * B + b, xv[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < SPL; ++k) acc_fma(hs[k], hc[k], __int_as_float(e[u].y), xv[u][k]);
    }
    for (; t < cnt; ++t) {
        float2 xv[SPL];
        ld_xs<SPL>(x, (int64_t)st[t].x * B + b, xv);
#pragma unroll
        for (int k = 0; k < SPL; ++k) acc_fma(hs[k], hc[k], __int_as_float(st[t].y), xv[k]);
    }
}

// Y[row][b] = scale * sum_k val_k X[col_k][b]; SPL slices per lane (HALF:
// 16 lanes per row, see lane_map_spl).
template <typename VT, typename XT, typename YT, int U, int SPL, bool HALF>
__global__ void __launch_bounds__(256) spmm_df_kernel(SellView m, ColMap cm, const VT* __restrict__ val,
                                                      const XT* __restrict__ x, YT* __restrict__ y, int B,
                                                      BProd a, OutMap om)
{
    __shared__ int2 stage[kWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rb, chunk;
    const int cs = chunk_slices(SPL, HALF);
    const int chunks = (B + cs - 1) / cs;
    block_coords(chunks, rb, chunk);
    const int G = (int)gridDim.x / chunks;
    const LaneMap lm = lane_map_spl<SPL, HALF>(B, chunk, lane);
    const int b = lm.b, t_in = lane % lm.W;
    bool live[SPL];
#pragma unroll
    for (int k = 0; k < SPL; ++k) live[k] = slice_live(b + k, B, a.cg, a.sb);
    const bool any = SPL == 1 ? live[0] : (live[0] || live[SPL - 1]);
    for (int64_t r0 = warp_row0(rb, w, lm); r0 < m.rows; r0 += row_stride(G, lm)) {
        const int64_t row = r0 + lm.g;
        const bool rv = row < m.rows;
        const int len = rv ? m.len[row] : 0;
        const int64_t base = rv ? row_base(m, row) : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        float hs[SPL], hc[SPL];
#pragma unroll
        for (int k = 0; k < SPL; ++k) hs[k] = hc[k] = 0.0f;
        for (int j0 = 0; j0 < maxlen; j0 += lm.W) {
            stage_entries<VT>(cm, val, row, base, len, j0, t_in, &stage[w][lane]);
            __syncwarp();
            const int cnt = min(lm.W, len - j0);
            if (any && cnt > 0) staged_dot<XT, U, SPL>(&stage[w][lm.g * lm.W], cnt, x, B, b, hs, hc);
            __syncwarp();
        }
        if (!rv) continue;
        int64_t pos = row;
        bool keep = true;
        if (om.user) {
            int i, j;
            tiled_coords(row, om.tn, i, j);
            keep = i < om.n && j < om.n;
            pos = (int64_t)i * om.n + j;
        }
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            if (!live[k] || !keep) continue;
            float2 v = acc_value(hs[k], hc[k]);
            if (a.row_scale) {
                const float sc = a.row_scale[row];
                v = df_mul_f(v, sc);
                if (a.rpow == 2) v = df_mul_f(v, sc);
            }
            st_y(y, pos * B + b + k, df_mul(a.scale, v));
        }
    }
}

struct BOp {
    int mode;  // 1: q = Op(p), p.q;  2: r = rhs - Op(u), p = r, r.r, rhs.rhs;  3: r = rhs - Op(u), r.r
    float2 c_id, c_ata, c_grad, lam;
    const float2* in;
    float2* out;
    float2* p_out;
    const float2* rhs;
    const float2* atf;
    const float2* vx;
    const float2* vy;
    const CgSlice* cg;
    const SbSlice* sb;
    float2* partials;
    int n, tn;
};

__device__ __forceinline__ float2 lap_b(const float2* __restrict__ u, int64_t t, int i, int j, int n, int tn, int B,
                                       int b)
{
    const float2 c = u[t * B + b];
    float2 acc = df_zero();
    if (j > 0) acc = df_add(acc, df_sub(c, u[tiled_index(i, j - 1, tn) * B + b]));
    if (j < n - 1) acc = df_add(acc, df_sub(c, u[tiled_index(i, j + 1, tn) * B + b]));
    if (i > 0) acc = df_add(acc, df_sub(c, u[tiled_index(i - 1, j, tn) * B + b]));
    if (i < n - 1) acc = df_add(acc, df_sub(c, u[tiled_index(i + 1, j, tn) * B + b]));
    return acc;
}

__device__ __forceinline__ float2 grad_adj_b(const float2* __restrict__ vx, const float2* __restrict__ vy,
                                             int64_t t, int i, int j, int n, int tn, int B, int b)
{
    float2 acc = df_zero();
    if (j >= 1) acc = df_add(acc, vx[tiled_index(i, j - 1, tn) * B + b]);
    if (j <= n - 2) acc = df_sub(acc, vx[t * B + b]);
    if (i >= 1) acc = df_add(acc, vy[tiled_index(i - 1, j, tn) * B + b]);
    if (i <= n - 2) acc = df_sub(acc, vy[t * B + b]);
    return acc;
}

template <int MODE>
__device__ __forceinline__ void bop_epilogue(const BOp& a, int64_t t, int i, int j, int B, int b, float2 nacc,
                                             float& s0, float& c0, float& s1, float& c1)
{
    const int64_t e = t * B + b;
    const float2 in = a.in[e];
    float2 op = df_mul(a.c_ata, nacc);
    op = df_add(op, df_mul(a.c_grad, lap_b(a.in, t, i, j, a.n, a.tn, B, b)));
    op = df_add(op, df_mul(a.c_id, in));
    if (MODE == 1) {
        a.out[e] = op;
        acc_add(s0, c0, df_mul(in, op));
    } else {
        const float2 rhs =
            a.rhs ? a.rhs[e] : df_add(a.atf[e], df_mul(a.lam, grad_adj_b(a.vx, a.vy, t, i, j, a.n, a.tn, B, b)));
        const float2 r = df_sub(rhs, op);
        a.out[e] = r;
        if (MODE == 2) a.p_out[e] = r;
        acc_add(s0, c0, df_mul(r, r));
        acc_add(s1, c1, df_mul(rhs, rhs));
    }
}

// A^T y for every slice fused with the operator epilogue (rows = pixels);
// SPL slices per lane.
template <typename VT, int MODE, int U, int SPL>
__global__ void __launch_bounds__(256) spmm_op_kernel(SellView m, ColMap cm, const VT* __restrict__ val,
                                                      const float2* __restrict__ y, int B, BOp a)
{
    __shared__ int2 stage[kWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rb, chunk;
    const int chunks = (B + 32 * SPL - 1) / (32 * SPL);
    block_coords(chunks, rb, chunk);
    const int G = (int)gridDim.x / chunks;
    const LaneMap lm = lane_map_spl<SPL>(B, chunk, lane);
    const int b = lm.b, t_in = lane % lm.W;
    bool live[SPL];
#pragma unroll
    for (int k = 0; k < SPL; ++k) live[k] = slice_live(b + k, B, MODE == 2 ? nullptr : a.cg, a.sb);
    const bool any = SPL == 1 ? live[0] : (live[0] || live[SPL - 1]);
    float s0[SPL], c0[SPL], s1[SPL], c1[SPL];
#pragma unroll
    for (int k = 0; k < SPL; ++k) s0[k] = c0[k] = s1[k] = c1[k] = 0.0f;
    for (int64_t r0 = warp_row0(rb, w, lm); r0 < m.rows; r0 += row_stride(G, lm)) {
        const int64_t row = r0 + lm.g;
        const bool rv = row < m.rows;
        const int len = rv ? m.len[row] : 0;
        const int64_t base = rv ? row_base(m, row) : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        float hs[SPL], hc[SPL];
#pragma unroll
        for (int k = 0; k < SPL; ++k) hs[k] = hc[k] = 0.0f;
        for (int j0 = 0; j0 < maxlen; j0 += lm.W) {
            stage_entries<VT>(cm, val, row, base, len, j0, t_in, &stage[w][lane]);
            __syncwarp();
            const int cnt = min(lm.W, len - j0);
            if (any && cnt > 0) staged_dot<float2, U, SPL>(&stage[w][lm.g * lm.W], cnt, y, B, b, hs, hc);
            __syncwarp();
        }
        if (!rv) continue;
        int i, j;
        tiled_coords(row, a.tn, i, j);
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            if (!live[k]) continue;
            if (i < a.n && j < a.n) {
                bop_epilogue<MODE>(a, row, i, j, B, b + k, acc_value(hs[k], hc[k]), s0[k], c0[k], s1[k], c1[k]);
            } else {
                a.out[row * B + b + k] = df_zero();  // padding stays zero
                if (MODE == 2) a.p_out[row * B + b + k] = df_zero();
            }
        }
    }
    float2 v[2][SPL];
#pragma unroll
    for (int k = 0; k < SPL; ++k) {
        v[0][k] = acc_value(s0[k], c0[k]);
        v[1][k] = acc_value(s1[k], c1[k]);
    }
    block_partials<2, SPL>(v, a.partials, B, G, rb, chunk, lm.W);
}

// Surrogate stencil T (Sec. 3.2) for every slice fused with the epilogue.
template <int MODE>
__global__ void __launch_bounds__(256) stencil_b_kernel(int B, BOp a, const int32_t* __restrict__ taps_d,
                                                        const float* __restrict__ taps_w, int ntaps)
{
    extern __shared__ unsigned char smem_raw[];
    int2* sd = reinterpret_cast<int2*>(smem_raw);
    float2* sw = reinterpret_cast<float2*>(smem_raw + sizeof(int2) * ntaps);
    for (int t = threadIdx.x; t < ntaps; t += blockDim.x) {
        sd[t] = make_int2(taps_d[2 * t], taps_d[2 * t + 1]);
        sw[t] = make_float2(taps_w[2 * t], taps_w[2 * t + 1]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rb, chunk;
    const int chunks = (B + 31) / 32;
    block_coords(chunks, rb, chunk);
    const int G = (int)gridDim.x / chunks;
    const LaneMap lm = lane_map(B, chunk, lane);
    const int b = lm.b;
    const int64_t r_first = warp_row0(rb, w, lm) + lm.g, r_step = row_stride(G, lm);
    const bool live = slice_live(b, B, MODE == 2 ? nullptr : a.cg, a.sb);
    const int n = a.n;
    const int64_t npad = padded_pixels(n);
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    if (live) {
        for (int64_t p = r_first; p < npad; p += r_step) {
            int i, j;
            tiled_coords(p, a.tn, i, j);
            if (i >= n || j >= n) {
                a.out[p * B + b] = df_zero();  // padding stays zero
                if (MODE == 2) a.p_out[p * B + b] = df_zero();
                continue;
            }
            float hs = 0.0f, hc = 0.0f;
            for (int t = 0; t < ntaps; ++t) {
                const int ii = i + sd[t].x, jj = j + sd[t].y;
                if (ii >= 0 && ii < n && jj >= 0 && jj < n)
                    acc_add(hs, hc, df_mul(sw[t], a.in[tiled_index(ii, jj, a.tn) * B + b]));
            }
            bop_epilogue<MODE>(a, p, i, j, B, b, acc_value(hs, hc), s0, c0, s1, c1);
        }
    }
    float2 v[2][1] = {{acc_value(s0, c0)}, {acc_value(s1, c1)}};
    block_partials<2>(v, a.partials, B, G, rb, chunk, lm.W);
}

// Element-wise kernels over [n2][B]: thread = (pixel, slice).
__global__ void __launch_bounds__(256) bcg_update_kernel(float2* __restrict__ u, float2* __restrict__ r,
                                                         const float2* __restrict__ p,
                                                         const float2* __restrict__ q, int64_t n2, int B,
                                                         const CgSlice* cg, const SbSlice* sb,
                                                         float2* partials)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rb, chunk;
    const int chunks = (B + 31) / 32;
    block_coords(chunks, rb, chunk);
    const int G = (int)gridDim.x / chunks;
    const LaneMap lm = lane_map(B, chunk, lane);
    const int b = lm.b;
    const int64_t r_first = warp_row0(rb, w, lm) + lm.g, r_step = row_stride(G, lm);
    float s = 0.0f, c = 0.0f;
    if (slice_live(b, B, cg, sb)) {
        const float2 al = cg[b].alpha_df;
        for (int64_t px = r_first; px < n2; px += r_step) {
            const int64_t e = px * B + b;
            u[e] = df_add(u[e], df_mul(al, p[e]));
            const float2 rn = df_sub(r[e], df_mul(al, q[e]));
            r[e] = rn;
            acc_add(s, c, df_mul(rn, rn));
        }
    }
    float2 v[1][1] = {{acc_value(s, c)}};
    block_partials<1>(v, partials, B, G, rb, chunk, lm.W);
}

__global__ void __launch_bounds__(256) bcg_direction_kernel(float2* __restrict__ p, const float2* __restrict__ r,
                                                            int64_t n2, int B, const CgSlice* cg,
                                                            const SbSlice* sb)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rb, chunk;
    const int chunks = (B + 31) / 32;
    block_coords(chunks, rb, chunk);
    const int G = (int)gridDim.x / chunks;
    const LaneMap lm = lane_map(B, chunk, lane);
    const int b = lm.b;
    const int64_t r_first = warp_row0(rb, w, lm) + lm.g, r_step = row_stride(G, lm);
    if (!slice_live(b, B, cg, sb)) return;
    const float2 be = cg[b].beta_df;
    for (int64_t px = r_first; px < n2; px += r_step) {
        const int64_t e = px * B + b;
        p[e] = df_add(r[e], df_mul(be, p[e]));
    }
}

__device__ __forceinline__ float2 shrink_b(float2 x, float2 gamma)
{
    if (!df_gt(df_abs(x), gamma)) return df_zero();
    return x.x < 0.0f ? df_add(x, gamma) : df_sub(x, gamma);
}

__global__ void __launch_bounds__(256) bsb_shrink_kernel(const float2* __restrict__ u, float2* __restrict__ u_old,
                                                         float2* __restrict__ bx, float2* __restrict__ by,
                                                         float2* __restrict__ vx, float2* __restrict__ vy, int n,
                                                         int tn, int B, float2 gamma, const SbSlice* sb,
                                                         float2* partials)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rb, chunk;
    const int chunks = (B + 31) / 32;
    block_coords(chunks, rb, chunk);
    const int G = (int)gridDim.x / chunks;
    const LaneMap lm = lane_map(B, chunk, lane);
    const int b = lm.b;
    const int64_t r_first = warp_row0(rb, w, lm) + lm.g, r_step = row_stride(G, lm);
    const int64_t npad = padded_pixels(n);
    float s = 0.0f, cc = 0.0f;
    if (slice_live(b, B, nullptr, sb)) {
        for (int64_t p = r_first; p < npad; p += r_step) {
            int i, j;
            tiled_coords(p, tn, i, j);
            if (i >= n || j >= n) continue;
            const int64_t e = p * B + b;
            const float2 c = u[e];
            const float2 gx = (j < n - 1) ? df_sub(u[tiled_index(i, j + 1, tn) * B + b], c) : df_zero();
            const float2 gy = (i < n - 1) ? df_sub(u[tiled_index(i + 1, j, tn) * B + b], c) : df_zero();
            const float2 tx = df_add(gx, bx[e]), ty = df_add(gy, by[e]);
            const float2 dx = shrink_b(tx, gamma), dy = shrink_b(ty, gamma);
            const float2 bxn = df_sub(tx, dx), byn = df_sub(ty, dy);
            bx[e] = bxn;
            by[e] = byn;
            vx[e] = df_sub(dx, bxn);
            vy[e] = df_sub(dy, byn);
            acc_add(s, cc, df_abs(df_sub(c, u_old[e])));
            u_old[e] = c;
        }
    }
    float2 v[1][1] = {{acc_value(s, cc)}};
    block_partials<1>(v, partials, B, G, rb, chunk, lm.W);
}

// Per-slice finalisation: sum the G partials of each quantity (fixed order)
// and apply the scalar update.  One block per slice.
enum { FIN_RESIDUAL = 0, FIN_PQ = 1, FIN_UPDATE = 2, FIN_REFRESH = 3, FIN_SB = 4 };

template <int KIND, int NQ>
__global__ void __launch_bounds__(256) finalize_kernel(const float2* __restrict__ partials, int G, int B,
                                                       CgSlice* cg, SbSlice* sb, double tol)
{
    const int b = blockIdx.x;
    __shared__ float2 sh[NQ][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float2 tv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float2 s = df_zero();
        for (int i = threadIdx.x; i < G; i += blockDim.x) s = df_add(s, partials[((size_t)q * B + b) * G + i]);
        s = warp_sum_df(s);
        if (lane == 0) sh[q][w] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float2 s = sh[q][0];
        for (int k = 1; k < (int)(blockDim.x / 32); ++k) s = df_add(s, sh[q][k]);
        tot[q] = df_to_double(s);
    }
    (void)tv;
    if (KIND == FIN_SB) {
        if (sb[b].stopped) return;
        if (cg[b].status != CT_OK) {
            sb[b].status = cg[b].status;
            sb[b].stopped = 1;
        } else {
            sb_after_update(sb[b], tot[0], tol);
        }
        return;
    }
    if (sb && sb[b].stopped) return;
    if (KIND == FIN_RESIDUAL) cg_after_residual(cg[b], tot[0], tot[NQ - 1], tol);
    if (KIND == FIN_PQ) cg_after_pq(cg[b], tot[0]);
    if (KIND == FIN_UPDATE) cg_after_update(cg[b], tot[0], tol);
    if (KIND == FIN_REFRESH && cg[b].active) cg[b].rr = tot[0];
}

// Caller's row-major [n*n][B] (FP32) -> internal tiled [npad][B] double-float.
// The caller's batch [len][B]: one array with the slice innermost, or one
// array per slice (ct_split_bregman_ragged).
struct BatchIn {
    const float* dense;
    const float* const* cols;
    __device__ __forceinline__ float operator()(int64_t i, int B, int b) const
    {
        return dense ? dense[i * B + b] : cols[b][i];
    }
};
struct BatchOut {
    float* dense;
    float* const* cols;
    __device__ __forceinline__ float& operator()(int64_t i, int B, int b) const
    {
        return dense ? dense[i * B + b] : cols[b][i];
    }
};

__global__ void bwiden_kernel(BatchIn in, float2* __restrict__ out, int n, int tn, int B)
{
    const int64_t len = padded_pixels(n) * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / B;
        const int b = (int)(e - t * B);
        int i, j;
        tiled_coords(t, tn, i, j);
        out[e] = (i < n && j < n) ? make_float2(in((int64_t)i * n + j, B, b), 0.0f) : make_float2(0.0f, 0.0f);
    }
}

__global__ void bnarrow_kernel(const float2* __restrict__ in, BatchOut out, int n, int tn, int B)
{
    const int64_t len = padded_pixels(n) * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / B;
        const int b = (int)(e - t * B);
        int i, j;
        tiled_coords(t, tn, i, j);
        if (i < n && j < n) out((int64_t)i * n + j, B, b) = df_to_float(in[e]);
    }
}

// Caller's row-major [n*n][B] (FP32) -> internal tiled [npad][B] FP32.
__global__ void bpermute_in_kernel(const float* __restrict__ in, float* __restrict__ out, int n, int tn, int B)
{
    const int64_t len = padded_pixels(n) * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / B;
        const int b = (int)(e - t * B);
        int i, j;
        tiled_coords(t, tn, i, j);
        out[e] = (i < n && j < n) ? in[((int64_t)i * n + j) * B + b] : 0.0f;
    }
}

// f (FP32, [rows][B]) -> double-float, times the row scale s (FP16 storage).
__global__ void bto_df_kernel(BatchIn in, const float* __restrict__ scale, float2* __restrict__ out, int64_t rows,
                              int B)
{
    const int64_t len = rows * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / B;
        const int b = (int)(e - i * B);
        const float v = in(i, B, b);
        out[e] = scale ? two_prod(v, scale[i]) : make_float2(v, 0.0f);
    }
}

struct BPlan {
    ct_matrix* M;
    Workspace* w;
    ValKind vk;
    bool sparse;
    const Stencil* S;
    BOp base;
    int B;
    int64_t n2;
    int refresh;
    double tol;
    Grid2 g_rows_a, g_rows_t, g_pix;  // decompositions for A, A^T and the image
    const SbSlice* sb;                 // gate (SB) or null
};

Grid2 make_grid(const ct_matrix* M, int64_t rows, int B, int spl = 1, bool half = false)
{
    Grid2 g;
    g.spl = spl;
    const int cs = chunk_slices(spl, half);
    g.chunks = (B + cs - 1) / cs;
    const int64_t rows_per_block = (int64_t)kWarps * (half ? 2 : 32 / lanes_per_row(B));
    const int64_t cap = (int64_t)(M->sm_count > 0 ? M->sm_count : 148) * 8;
    int64_t rb = (rows + rows_per_block - 1) / rows_per_block;
    if (rb > cap) rb = cap;
    if (rb < 1) rb = 1;
    g.rb = (int)rb;
    return g;
}

int launch_fin(const BPlan& P, int kind, const Grid2& g, cudaStream_t st)
{
    Workspace& w = *P.w;
    switch (kind) {
    case FIN_RESIDUAL:
        finalize_kernel<FIN_RESIDUAL, 2><<<P.B, 256, 0, st>>>(w.partials, g.rb, P.B, w.cg, (SbSlice*)P.sb, P.tol);
        break;
    case FIN_PQ: finalize_kernel<FIN_PQ, 1><<<P.B, 256, 0, st>>>(w.partials, g.rb, P.B, w.cg, (SbSlice*)P.sb, P.tol); break;
    case FIN_UPDATE:
        finalize_kernel<FIN_UPDATE, 1><<<P.B, 256, 0, st>>>(w.partials, g.rb, P.B, w.cg, (SbSlice*)P.sb, P.tol);
        break;
    case FIN_REFRESH:
        finalize_kernel<FIN_REFRESH, 1><<<P.B, 256, 0, st>>>(w.partials, g.rb, P.B, w.cg, (SbSlice*)P.sb, P.tol);
        break;
    default: break;
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ColMap colmap_of(const ct_matrix* M, int which)
{
    if (which == 0) return ColMap{M->A.col, nullptr, nullptr, nullptr, nullptr, M->g.n_bins, M->n_kept};
    return ColMap{nullptr, M->At.col16, M->band_lo, M->band_off, M->band_angle, M->g.n_bins, M->n_kept};
}

// Staged-entry unroll of the batched products for batch size B: the tuned or
// pinned choice, else 8.
int spmm_unroll(const ct_matrix* M, int B)
{
    auto it = M->spmm_unroll.find(B);
    return it != M->spmm_unroll.end() && it->second > 0 ? it->second : 8;
}

// Resident blocks per SM of a kernel at 256 threads (queried once per kernel).
template <auto Kernel>
int resident_blocks()
{
    static int occ = 0;
    if (occ == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, Kernel, 256, 0) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 8;
        }
        occ = v;
    }
    return occ;
}

// Blocks of a product launch: the row blocks of g times the slice chunks.
// A batch of one chunk caps its row blocks at what the SMs hold at once, so
// that it runs in one wave with the blocks looping over the rows (measured:
// 16 slices, 0.407 -> 0.319 ms); larger batches keep g's many waves, whose
// chunk-major order measured faster there (256 slices: 9.14 against 9.34 ms
// with the cap).  Every row is summed by the same lanes in the same order
// whatever the count, so results do not depend on it.
template <auto Kernel>
int spmm_blocks(const ct_matrix* M, const Grid2& g)
{
    if (g.chunks > 1) return g.rb * g.chunks;
    const int64_t cap = (int64_t)(M->sm_count > 0 ? M->sm_count : 148) * resident_blocks<Kernel>();
    const int64_t rb = std::max<int64_t>(1, std::min<int64_t>(g.rb, cap));
    return (int)(rb * g.chunks);
}

// which = 0: rows of A (rays); which = 1: rows of A^T (internal pixels).
template <typename XT, typename YT>
int launch_spmm(const ct_matrix* M, int which, ValKind vk, const XT* x, YT* y, int B, BProd a, cudaStream_t st,
                bool user_out = false, int unroll = 0)
{
    const Sell& C = which == 0 ? M->A : M->At;
    const SellView m{C.slice_ptr, C.row_len, C.rows};
    const ColMap cm = colmap_of(M, which);
    const OutMap om{user_out ? 1 : 0, M->g.n, M->tn};
    // paired slices load two adjacent values at once: only from an input
    // aligned for that (a caller's array may be an offset view)
    const int spl = (slices_per_lane(B) == 2 && reinterpret_cast<uintptr_t>(x) % (2 * sizeof(XT)) == 0) ? 2 : 1;
    // y = A x gathers image vectors from all over the image: 32-slice chunks
    // keep them L2-resident (the A^T products gather within a tile's band)
    const bool half = spl == 2 && which == 0;
    const Grid2 g = make_grid(M, C.rows, B, spl, half);
    const int uu = unroll ? unroll : spmm_unroll(M, B);
    const bool u4 = uu == 4, u16 = uu == 16;  // 16: one slice per lane only
#define CT_DF(VT, VAL, U, SPL, H)                                                                   \
    spmm_df_kernel<VT, XT, YT, U, SPL, H><<<spmm_blocks<spmm_df_kernel<VT, XT, YT, U, SPL, H>>(M, g), 256, 0, \
                                            st>>>(m, cm, VAL, x, y, B, a, om)
    if (vk == ValKind::F16) {
        if (half) {
            if (u4) CT_DF(__half, C.qval, 4, 2, true); else CT_DF(__half, C.qval, 8, 2, true);
        } else if (spl == 2) {
            if (u4) CT_DF(__half, C.qval, 4, 2, false); else CT_DF(__half, C.qval, 8, 2, false);
        } else {
            if (u4) CT_DF(__half, C.qval, 4, 1, false);
            else if (u16) CT_DF(__half, C.qval, 16, 1, false);
            else CT_DF(__half, C.qval, 8, 1, false);
        }
    } else {
        if (half) {
            if (u4) CT_DF(float, C.val, 4, 2, true); else CT_DF(float, C.val, 8, 2, true);
        } else if (spl == 2) {
            if (u4) CT_DF(float, C.val, 4, 2, false); else CT_DF(float, C.val, 8, 2, false);
        } else {
            if (u4) CT_DF(float, C.val, 4, 1, false);
            else if (u16) CT_DF(float, C.val, 16, 1, false);
            else CT_DF(float, C.val, 8, 1, false);
        }
    }
#undef CT_DF
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// Chooses the staged-entry unroll for batch size B on this handle by timing
// the forward SpMM (x -> y, both workspace buffers) with each candidate; the
// candidates give identical bits, so only speed depends on the choice.  Runs
// once per (handle, B), never while st is being captured, and keeps a
// pinned choice.
int tune_spmm(ct_matrix* M, ValKind vk, int B, const float2* x, float2* y, cudaStream_t st)
{
    if (M->spmm_unroll.count(B)) return CT_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CT_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return CT_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CT_CUDA(cudaEventCreate(&e0));
    const cudaError_t ec = cudaEventCreate(&e1);
    if (ec != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ec, "cudaEventCreate", __FILE__, __LINE__);
    }
    BProd a{vk == ValKind::F16 ? M->row_scale : nullptr, 1, make_float2(1.0f, 0.0f), nullptr, nullptr};
    // 16 staged entries in flight only where a lane takes one slice
    const int cand[3] = {4, 8, 16};
    const int ncand = slices_per_lane(B) == 1 ? 3 : 2;
    float best_ms = 0.0f;
    int best = 8, rc = CT_OK;
    for (int c = 0; c < ncand && rc == CT_OK; ++c) {
        rc = launch_spmm(M, 0, vk, x, y, B, a, st, false, cand[c]);  // warm-up
        cudaError_t e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && rc == CT_OK && e == cudaSuccess; ++r)
            rc = launch_spmm(M, 0, vk, x, y, B, a, st, false, cand[c]);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess && rc == CT_OK) rc = cuda_fail(e, "timing the batched product", __FILE__, __LINE__);
        if (rc == CT_OK && (c == 0 || ms < best_ms)) {
            best_ms = ms;
            best = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == CT_OK) M->spmm_unroll[B] = best;
    return rc;
}

// Op(in) with the epilogue of `mode`; partials land in w.partials (layout of g).
int bapply(const BPlan& P, BOp ep, const float2* in, cudaStream_t st, Grid2& g_used, bool fp32_refresh = false)
{
    Workspace& w = *P.w;
    ep.in = in;
    if (P.sparse) {
        const ValKind vk = fp32_refresh ? ValKind::F32 : P.vk;
        BProd a{vk == ValKind::F16 ? P.M->row_scale : nullptr, vk == ValKind::F16 ? 2 : 0,
                make_float2(1.0f, 0.0f), ep.mode == 2 ? nullptr : w.cg, P.sb};
        CT_CHECK(launch_spmm(P.M, 0, vk, in, w.y, P.B, a, st));
        const Sell& C = P.M->At;
        const SellView m{C.slice_ptr, C.row_len, C.rows};
        const ColMap cm = colmap_of(P.M, 1);
        g_used = P.g_rows_t;
        const int blocks = g_used.rb * g_used.chunks;
#define CT_BOP(VT, VAL, U, SPL)                                                                       \
    switch (ep.mode) {                                                                                \
    case 1: spmm_op_kernel<VT, 1, U, SPL><<<blocks, 256, 0, st>>>(m, cm, VAL, w.y, P.B, ep); break;  \
    case 2: spmm_op_kernel<VT, 2, U, SPL><<<blocks, 256, 0, st>>>(m, cm, VAL, w.y, P.B, ep); break;  \
    default: spmm_op_kernel<VT, 3, U, SPL><<<blocks, 256, 0, st>>>(m, cm, VAL, w.y, P.B, ep); break; \
    }
        const bool u4 = spmm_unroll(P.M, P.B) == 4;
        const bool pair = g_used.spl == 2;
        if (vk == ValKind::F16) {
            if (pair) {
                if (u4) { CT_BOP(__half, C.qval, 4, 2) } else { CT_BOP(__half, C.qval, 8, 2) }
            } else {
                if (u4) { CT_BOP(__half, C.qval, 4, 1) } else { CT_BOP(__half, C.qval, 8, 1) }
            }
        } else {
            if (pair) {
                if (u4) { CT_BOP(float, C.val, 4, 2) } else { CT_BOP(float, C.val, 8, 2) }
            } else {
                if (u4) { CT_BOP(float, C.val, 4, 1) } else { CT_BOP(float, C.val, 8, 1) }
            }
        }
#undef CT_BOP
    } else {
        g_used = P.g_pix;
        const int blocks = g_used.rb * g_used.chunks;
        const int ntaps = P.S ? P.S->ntaps : 0;
        const size_t smem = (sizeof(int2) + sizeof(float2)) * (size_t)ntaps;
        const int32_t* d = P.S ? P.S->d : nullptr;
        const float* tw = P.S ? P.S->w : nullptr;
        switch (ep.mode) {
        case 1: stencil_b_kernel<1><<<blocks, 256, smem, st>>>(P.B, ep, d, tw, ntaps); break;
        case 2: stencil_b_kernel<2><<<blocks, 256, smem, st>>>(P.B, ep, d, tw, ntaps); break;
        default: stencil_b_kernel<3><<<blocks, 256, smem, st>>>(P.B, ep, d, tw, ntaps); break;
        }
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int benqueue_cg(const BPlan& P, const float2* rhs, int iters, cudaStream_t st)
{
    Workspace& w = *P.w;
    Grid2 g;
    BOp ep = P.base;
    ep.mode = 2;
    ep.out = w.r;
    ep.p_out = w.p;
    ep.rhs = rhs;
    CT_CHECK(bapply(P, ep, w.u, st, g));
    CT_CHECK(launch_fin(P, FIN_RESIDUAL, g, st));
    const int pblocks = P.g_pix.rb * P.g_pix.chunks;
    for (int it = 0; it < iters; ++it) {
        BOp e1 = P.base;
        e1.mode = 1;
        e1.out = w.q;
        CT_CHECK(bapply(P, e1, w.p, st, g));
        CT_CHECK(launch_fin(P, FIN_PQ, g, st));
        bcg_update_kernel<<<pblocks, 256, 0, st>>>(w.u, w.r, w.p, w.q, P.n2, P.B, w.cg, P.sb, w.partials);
        CT_CUDA(cudaGetLastError());
        CT_CHECK(launch_fin(P, FIN_UPDATE, P.g_pix, st));
        bcg_direction_kernel<<<pblocks, 256, 0, st>>>(w.p, w.r, P.n2, P.B, w.cg, P.sb);
        CT_CUDA(cudaGetLastError());
        if (P.refresh > 0 && (it + 1) % P.refresh == 0 && it + 1 < iters) {
            BOp e3 = P.base;
            e3.mode = 3;
            e3.out = w.r;
            e3.rhs = rhs;
            CT_CHECK(bapply(P, e3, w.u, st, g, true));
            CT_CHECK(launch_fin(P, FIN_REFRESH, g, st));
        }
    }
    return CT_OK;
}

int bmake_plan(ct_matrix* M, int B, double c_id, double c_ata, double c_grad, double tol, int surr_r,
               int surr_square, int refresh, BPlan& P)
{
    P.M = M;
    P.w = &M->ws;
    P.B = B;
    P.vk = (M->flags & CT_VAL_FP16_ROWSCALE) ? ValKind::F16 : ValKind::F32;
    P.S = nullptr;
    if (surr_r > 0) {
        Stencil* S = nullptr;
        CT_CHECK(make_stencil(M, surr_r, surr_square, &S));
        P.S = S;
    }
    P.sparse = (c_ata != 0.0) && P.S == nullptr;
    if (c_ata == 0.0) P.S = nullptr;
    P.n2 = M->npad;
    if (refresh > 0) {
        if (P.vk != ValKind::F16 || !M->A.val)
            return fail(CT_ERR_UNSUPPORTED, "refresh_every needs FP16 storage built with CT_KEEP_FP32_COPY");
        if (!P.sparse) refresh = 0;
    }
    P.refresh = refresh;
    P.tol = tol;
    P.sb = nullptr;
    P.g_rows_a = make_grid(M, M->rows, B, slices_per_lane(B));
    P.g_rows_t = make_grid(M, M->At.rows, B, slices_per_lane(B));
    P.g_pix = make_grid(M, P.n2, B);
    BOp& b = P.base;
    std::memset(&b, 0, sizeof(b));
    b.c_id = df_from_double(c_id);
    b.c_ata = df_from_double(c_ata);
    b.c_grad = df_from_double(c_grad);
    b.cg = M->ws.cg;
    b.partials = M->ws.partials;
    b.n = M->g.n;
    b.tn = M->tn;
    return CT_OK;
}

int grid_blocks(const ct_matrix* M, int64_t len)
{
    return grid_for(M, len, 256, 8);
}

}  // namespace

int batched_product_df(const ct_matrix* M, int which, const float2* in, float2* out, int32_t B, int rpow,
                       cudaStream_t st)
{
    const ValKind vk = (M->flags & CT_VAL_FP16_ROWSCALE) ? ValKind::F16 : ValKind::F32;
    // the first forward product of this batch size on the handle picks the
    // staged-entry unroll (timed on these buffers; out is rewritten below)
    if (which == 0) CT_CHECK(tune_spmm(const_cast<ct_matrix*>(M), vk, B, in, out, st));
    BProd a{(vk == ValKind::F16 && which == 0 && rpow > 0) ? M->row_scale : nullptr, rpow, make_float2(1.0f, 0.0f),
            nullptr, nullptr};
    return launch_spmm(M, which, vk, in, out, B, a, st);
}

int batched_forward_adjoint(const ct_matrix* M, int which, const float* in, float* out, int32_t B,
                            cudaStream_t st)
{
    BProd a{nullptr, 0, make_float2(1.0f, 0.0f), nullptr, nullptr};
    const ValKind vk = (M->flags & CT_VAL_FP16_ROWSCALE) ? ValKind::F16 : ValKind::F32;
    ct_matrix* Mm = const_cast<ct_matrix*>(M);
    CT_CHECK(ensure_workspace(Mm, B, true));
    Workspace& w = Mm->ws;
    if (which == 0) {
        if (vk == ValKind::F16) {
            a.row_scale = M->row_scale;
            a.rpow = 1;
        }
        // the caller's image goes to the internal tile order first (FP32 copy in w.u)
        float* xt = reinterpret_cast<float*>(w.u);
        bpermute_in_kernel<<<grid_blocks(M, M->npad * B), 256, 0, st>>>(in, xt, M->g.n, M->tn, B);
        CT_CUDA(cudaGetLastError());
        return launch_spmm(M, 0, vk, (const float*)xt, out, B, a, st);
    }
    if (vk == ValKind::F16) {
        // A^T y = Q^T (s .* y): the scaled copy goes through the workspace sinogram buffer
        bto_df_kernel<<<grid_blocks(M, M->rows * B), 256, 0, st>>>(BatchIn{in, nullptr}, M->row_scale, w.y, M->rows, B);
        CT_CUDA(cudaGetLastError());
        return launch_spmm(M, 1, vk, (const float2*)w.y, out, B, a, st, true);
    }
    return launch_spmm(M, 1, vk, in, out, B, a, st, true);
}

int cg_solve_batched(ct_matrix* M, const ct_cg_params* Pp, const float* rhs, float* u, int32_t B,
                     ct_cg_stats* stats, cudaStream_t st)
{
    if (Pp->max_iters < 0) return fail(CT_ERR_ARG, "max_iters < 0");
    CT_CHECK(ensure_workspace(M, B, true));
    Workspace& w = M->ws;
    BPlan P;
    CT_CHECK(bmake_plan(M, B, Pp->c_id, Pp->c_ata, Pp->c_grad, Pp->rel_tol, Pp->surrogate_r,
                        Pp->surrogate_square, Pp->refresh_every, P));
    const int64_t len = P.n2 * B;
    bwiden_kernel<<<grid_blocks(M, len), 256, 0, st>>>(BatchIn{rhs, nullptr}, w.rhs, M->g.n, M->tn, B);
    bwiden_kernel<<<grid_blocks(M, len), 256, 0, st>>>(BatchIn{u, nullptr}, w.u, M->g.n, M->tn, B);
    CT_CUDA(cudaGetLastError());
    if (P.sparse) CT_CHECK(tune_spmm(M, P.vk, B, w.u, w.y, st));
    CT_CHECK(benqueue_cg(P, w.rhs, Pp->max_iters, st));
    bnarrow_kernel<<<grid_blocks(M, len), 256, 0, st>>>(w.u, BatchOut{u, nullptr}, M->g.n, M->tn, B);
    CT_CUDA(cudaGetLastError());
    if (stats) {
        std::vector<CgSlice> h(B);
        CT_CUDA(cudaMemcpyAsync(h.data(), w.cg, sizeof(CgSlice) * B, cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaStreamSynchronize(st));
        stats->iters = 0;
        stats->final_rel_res = 0.0;
        stats->status = CT_OK;
        for (const CgSlice& c : h) {
            stats->iters = std::max(stats->iters, c.iters);
            const double rel = c.rhs2 > 0 ? std::sqrt(c.rr / c.rhs2) : 0.0;
            stats->final_rel_res = std::max(stats->final_rel_res, rel);
            if (c.status != CT_OK && stats->status == CT_OK) stats->status = c.status;
        }
        if (stats->status != CT_OK)
            return fail(stats->status, stats->status == CT_ERR_BREAKDOWN ? "CG breakdown: p^T Op p <= 0"
                                                                         : "non-finite value in CG");
    }
    return CT_OK;
}

// Up to kMax device pointers, passed by value to the kernel that stores them.
struct PtrChunk {
    static constexpr int kMax = 128;
    float* p[kMax];
    int n, offset;
};

__global__ void set_ptrs_kernel(float** dst, PtrChunk c)
{
    if ((int)threadIdx.x < c.n) dst[c.offset + threadIdx.x] = c.p[threadIdx.x];
}

// One batched split-Bregman run on handle M: set-up, one Bregman update
// (replayed), and read-out, so that several runs can share one graph.
struct SbRun {
    ct_matrix* M = nullptr;
    const ct_sb_params* Sp = nullptr;
    BPlan P;
    int B = 0;
};

int sb_prepare(ct_matrix* M, const ct_sb_params* Sp, BatchIn f, BatchIn u, int32_t B, SbRun& R, cudaStream_t st)
{
    CT_CHECK(ensure_workspace(M, B, true));
    Workspace& w = M->ws;
    R.M = M;
    R.Sp = Sp;
    R.B = B;
    BPlan& P = R.P;
    CT_CHECK(bmake_plan(M, B, 0.0, Sp->alpha, Sp->lambda, Sp->cg_rel_tol, Sp->surrogate_r, Sp->surrogate_square,
                        Sp->refresh_every, P));
    P.sb = w.sb;
    P.base.sb = w.sb;
    P.base.atf = w.atf;
    P.base.vx = w.vx;
    P.base.vy = w.vy;
    P.base.lam = df_from_double(Sp->lambda);
    const int64_t len = P.n2 * B;
    // alpha A^T f once; FP16 storage applies A^T as Q^T (s .* f)
    bto_df_kernel<<<grid_blocks(M, M->rows * B), 256, 0, st>>>(f, P.vk == ValKind::F16 ? M->row_scale : nullptr,
                                                              w.y, M->rows, B);
    CT_CUDA(cudaGetLastError());
    {
        BProd a{nullptr, 0, df_from_double(Sp->alpha), nullptr, nullptr};
        CT_CHECK(launch_spmm(M, 1, P.vk, (const float2*)w.y, w.atf, B, a, st));
    }
    bwiden_kernel<<<grid_blocks(M, len), 256, 0, st>>>(u, w.u, M->g.n, M->tn, B);
    CT_CUDA(cudaGetLastError());
    if (P.sparse) CT_CHECK(tune_spmm(M, P.vk, B, w.u, w.y, st));
    CT_CUDA(cudaMemsetAsync(w.bx, 0, len * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.by, 0, len * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.vx, 0, len * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.vy, 0, len * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.sb, 0, sizeof(SbSlice) * B, st));
    CT_CUDA(cudaMemcpyAsync(w.u_old, w.u, len * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    return CT_OK;
}

// One Bregman update: inner CG, shrink and Bregman step, update size and stop rule.
int sb_update(const SbRun& R, cudaStream_t s)
{
    const BPlan& P = R.P;
    ct_matrix* M = R.M;
    Workspace& w = M->ws;
    const int pblocks = P.g_pix.rb * P.g_pix.chunks;
    CT_CHECK(benqueue_cg(P, nullptr, R.Sp->inner_cg_iters, s));
    bsb_shrink_kernel<<<pblocks, 256, 0, s>>>(w.u, w.u_old, w.bx, w.by, w.vx, w.vy, M->g.n, M->tn, R.B,
                                              df_from_double(1.0 / R.Sp->lambda), w.sb, w.partials);
    CT_CUDA(cudaGetLastError());
    finalize_kernel<FIN_SB, 1><<<R.B, 256, 0, s>>>(w.partials, P.g_pix.rb, R.B, w.cg, w.sb, R.Sp->stop_rel_update);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// Writes the reconstructions and, if stats is given, waits and fills one
// ct_sb_stats per slice (per_slice) or one summary (slice 0, min outer_done).
int sb_finish(const SbRun& R, BatchOut u, ct_sb_stats* stats, bool per_slice, cudaStream_t st)
{
    ct_matrix* M = R.M;
    Workspace& w = M->ws;
    const int B = R.B;
    bnarrow_kernel<<<grid_blocks(M, R.P.n2 * B), 256, 0, st>>>(w.u, u, M->g.n, M->tn, B);
    CT_CUDA(cudaGetLastError());
    if (!stats) return CT_OK;
    std::vector<SbSlice> h(B);
    CT_CUDA(cudaMemcpyAsync(h.data(), w.sb, sizeof(SbSlice) * B, cudaMemcpyDeviceToHost, st));
    CT_CUDA(cudaStreamSynchronize(st));
    int status = CT_OK;
    if (per_slice) {
        for (int b = 0; b < B; ++b) {
            stats[b].outer_done = h[b].outer_done;
            stats[b].first_update_l1 = h[b].first_upd;
            stats[b].last_update_l1 = h[b].last_upd;
            stats[b].status = h[b].status;
            if (h[b].status != CT_OK && status == CT_OK) status = h[b].status;
        }
    } else {
        stats->outer_done = h[0].outer_done;
        stats->first_update_l1 = h[0].first_upd;
        stats->last_update_l1 = h[0].last_upd;
        for (const SbSlice& s : h) {
            stats->outer_done = std::min(stats->outer_done, s.outer_done);
            if (s.status != CT_OK && status == CT_OK) status = s.status;
        }
        stats->status = status;
    }
    if (status != CT_OK) return fail(status, "split Bregman inner solve failed");
    return CT_OK;
}

int split_bregman_batched(ct_matrix* M, const ct_sb_params* Sp, const float* f, float* u, int32_t B,
                          ct_sb_stats* stats, cudaStream_t st)
{
    SbRun R;
    CT_CHECK(sb_prepare(M, Sp, BatchIn{f, nullptr}, BatchIn{u, nullptr}, B, R, st));
    CT_CHECK(run_updates({[&R](cudaStream_t s) { return sb_update(R, s); }}, {M->ws.cap_stream}, Sp->outer_iters,
                         st));
    return sb_finish(R, BatchOut{u, nullptr}, stats, false, st);
}

// Groups the problems by handle.  A group of at most kRaggedSingles problems
// runs as that many single-slice runs (one workspace each: the handle's own
// and extra ones kept with the handle), side by side in the graph: at such
// batch sizes the single-slice kernels, each streaming the matrix at close to
// HBM speed, beat the batched SpMM (measured: 5 problems of 1024 x 1024 with
// 900 angles, 33 ms per CG step as one SpMM against about 16 ms for five
// single-slice products).  Larger groups run the batched kernels through a
// per-slice pointer table.
constexpr int kRaggedSingles = 8;
int split_bregman_ragged(int32_t count, ct_matrix* const* A, const float* const* f, float* const* u,
                         const ct_sb_params* Sp, ct_sb_stats* stats, cudaStream_t st)
{
    std::vector<ct_matrix*> handles;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < count; ++i) {
        size_t g = 0;
        while (g < handles.size() && handles[g] != A[i]) ++g;
        if (g == handles.size()) {
            handles.push_back(A[i]);
            members.emplace_back();
        }
        members[g].push_back(i);
    }
    const size_t G = handles.size();
    std::vector<SbRun> runs(G);
    struct Free1 {
        void operator()(Sb1Run* r) const { sb1_free(r); }
    };
    std::vector<std::vector<std::unique_ptr<Sb1Run, Free1>>> runs1(G);
    std::vector<UpdateFn> fns;
    std::vector<cudaStream_t> caps;
    for (size_t g = 0; g < G; ++g) {
        ct_matrix* M = handles[g];
        const int B = (int)members[g].size();
        if (B <= kRaggedSingles) {
            while ((int)M->ws_pool.size() < B - 1) {
                std::unique_ptr<Workspace> w(new (std::nothrow) Workspace());
                if (!w) return fail(CT_ERR_OOM, "host allocation failed");
                M->ws_pool.push_back(std::move(w));
            }
            for (int b = 0; b < B; ++b) {
                Workspace& w = b == 0 ? M->ws : *M->ws_pool[b - 1];
                Sb1Run* r = nullptr;
                CT_CHECK(sb1_prepare(M, w, Sp, f[members[g][b]], u[members[g][b]], &r, st));
                runs1[g].emplace_back(r);
                fns.push_back([r](cudaStream_t s) { return sb1_update(r, s); });
                caps.push_back(w.cap_stream);
            }
        } else {
            CT_CHECK(ensure_workspace(M, B, true));
            Workspace& w = M->ws;
            if (w.ragged_cap < B) {
                cudaFree(w.ragged_ptrs);
                w.ragged_ptrs = nullptr;
                w.ragged_cap = 0;
                const cudaError_t e = cudaMalloc(&w.ragged_ptrs, sizeof(float*) * 2 * (size_t)B);
                if (e == cudaErrorMemoryAllocation) {
                    (void)cudaGetLastError();
                    return fail(CT_ERR_OOM, "device allocation of the ragged pointer table failed");
                }
                CT_CUDA(e);
                w.ragged_cap = B;
            }
            // the table [f columns | u columns] is written by kernels on st
            // (pointers passed by value), so it is ordered after any earlier
            // call on st that still reads it
            PtrChunk c;
            for (int b0 = 0; b0 < 2 * B; b0 += PtrChunk::kMax) {
                c.n = std::min(PtrChunk::kMax, 2 * B - b0);
                c.offset = b0;
                for (int k = 0; k < c.n; ++k) {
                    const int e = b0 + k;
                    c.p[k] = e < B ? const_cast<float*>(f[members[g][e]]) : u[members[g][e - B]];
                }
                set_ptrs_kernel<<<1, PtrChunk::kMax, 0, st>>>(w.ragged_ptrs, c);
                CT_CUDA(cudaGetLastError());
            }
            CT_CHECK(sb_prepare(M, Sp, BatchIn{nullptr, w.ragged_ptrs}, BatchIn{nullptr, w.ragged_ptrs + B}, B,
                                runs[g], st));
            SbRun* r = &runs[g];
            fns.push_back([r](cudaStream_t s) { return sb_update(*r, s); });
            caps.push_back(M->ws.cap_stream);
        }
    }
    // every group a set of single-slice runs: one persistent launch per
    // update (ragged.cu); else one captured graph of the groups' launches
    bool persistent = false;
    if (std::all_of(members.begin(), members.end(), [](const std::vector<int>& m) { return (int)m.size() <= kRaggedSingles; })) {
        std::vector<Sb1Run*> all;
        for (size_t g = 0; g < G; ++g)
            for (auto& r : runs1[g]) all.push_back(r.get());
        CT_CHECK(ragged_persistent(all, Sp->outer_iters, st, caps[0], &persistent));
    }
    if (!persistent) CT_CHECK(run_updates(fns, caps, Sp->outer_iters, st));
    int status = CT_OK;
    std::vector<ct_sb_stats> gs;
    for (size_t g = 0; g < G; ++g) {
        const int B = (int)members[g].size();
        gs.assign(B, ct_sb_stats{});
        int rc = CT_OK;
        if (B <= kRaggedSingles) {
            for (int b = 0; b < B; ++b) {
                const int rb = sb1_finish(runs1[g][b].get(), u[members[g][b]], stats ? &gs[b] : nullptr, st);
                if (rb != CT_OK && rc == CT_OK) rc = rb;
                if (rb != CT_OK && rb != CT_ERR_BREAKDOWN && rb != CT_ERR_NONFINITE) return rb;
            }
        } else {
            rc = sb_finish(runs[g], BatchOut{nullptr, handles[g]->ws.ragged_ptrs + B}, stats ? gs.data() : nullptr,
                           true, st);
        }
        if (rc != CT_OK && rc != CT_ERR_BREAKDOWN && rc != CT_ERR_NONFINITE) return rc;
        if (rc != CT_OK && status == CT_OK) status = rc;
        if (stats)
            for (int b = 0; b < B; ++b) stats[members[g][b]] = gs[b];
    }
    if (status != CT_OK) return fail(status, "split Bregman inner solve failed");
    return CT_OK;
}

// ct_tune for a batch of B >= 2: the staged-entry unroll of the batched
// products, timed on the handle's workspace (see tune_spmm).
int tune_batched(ct_matrix* M, int32_t B, cudaStream_t st)
{
    CT_CHECK(ensure_workspace(M, B, true));
    const ValKind vk = (M->flags & CT_VAL_FP16_ROWSCALE) ? ValKind::F16 : ValKind::F32;
    CT_CUDA(cudaMemsetAsync(M->ws.u, 0, sizeof(float2) * M->npad * B, st));
    return tune_spmm(M, vk, B, M->ws.u, M->ws.y, st);
}

}  // namespace ct
