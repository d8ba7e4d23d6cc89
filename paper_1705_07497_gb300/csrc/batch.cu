// Batched solvers: many slices sharing one geometry (vectors [len][B], the
// slice index innermost).  The sparse products become SpMMs with the slices
// as the dense inner dimension: a warp owns one row for a chunk of 32 slices
// (one slice per lane), reads the row's entries 32 at a time (coalesced),
// stages them in shared memory and broadcasts them, so each lane gathers the
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
    int rb;      // row blocks
    int chunks;  // ceil(B / 32)
};

// Block (rb, chunk) decomposition of a 1-D grid: consecutive blocks share rows.
__device__ __forceinline__ void block_coords(int chunks, int& rb, int& chunk)
{
    rb = (int)blockIdx.x / chunks;
    chunk = (int)blockIdx.x % chunks;
}

__device__ __forceinline__ bool slice_live(int b, int B, const CgSlice* cg, const SbSlice* sb)
{
    if (b >= B) return false;
    if (cg && !cg[b].active) return false;
    if (sb && sb[b].stopped) return false;
    return true;
}

// Sum over the block's warps of each lane's value (fixed order), written as
// the block's partial for slice chunk*32 + lane:  partials[(q*B + b)*G + rb].
template <int NQ>
__device__ __forceinline__ void block_partials(const float2 (&v)[NQ], float2* partials, int B, int G, int rb,
                                               int chunk)
{
    __shared__ float2 red[NQ][kWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q][w][lane] = v[q];
    __syncthreads();
    if (w == 0) {
        const int b = chunk * 32 + lane;
        if (b < B) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                float2 s = red[q][0][lane];
                for (int k = 1; k < kWarps; ++k) s = df_add(s, red[q][k][lane]);
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
// indices k * W + w that map to sinogram row k * n_bins + band_lo(tile, k) + w.
struct ColMap {
    const int32_t* col;       // A
    const uint16_t* col16;    // A^T (band-local)
    const int32_t* band_lo;
    int nb, nk;
};

__device__ __forceinline__ int map_col(const ColMap& cm, int64_t row, int64_t k)
{
    if (cm.col) return __ldcs(cm.col + k);
    const int c = (int)__ldcs(cm.col16 + k);
    const int a = c / kBandW;
    return a * cm.nb + cm.band_lo[(row >> 8) * cm.nk + a] + (c - a * kBandW);
}

// Output position of (row, slice): internal layout, or for USER_OUT the
// caller's row-major image (rows are internal pixel indices; padding skipped).
struct OutMap {
    int user;  // 1: rows are pixels written in the caller's layout
    int n, tn;
};

// Y[row][b] = scale * sum_k val_k X[col_k][b].
template <typename VT, typename XT, typename YT>
__global__ void __launch_bounds__(256) spmm_df_kernel(CsrView m, ColMap cm, const VT* __restrict__ val,
                                                      const XT* __restrict__ x, YT* __restrict__ y, int B,
                                                      BProd a, OutMap om)
{
    __shared__ int2 stage[kWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rb, chunk;
    const int chunks = (B + 31) / 32;
    block_coords(chunks, rb, chunk);
    const int G = (int)gridDim.x / chunks;
    const int b = chunk * 32 + lane;
    const bool live = slice_live(b, B, a.cg, a.sb);
    for (int64_t row = (int64_t)rb * kWarps + w; row < m.rows; row += (int64_t)G * kWarps) {
        float hs = 0.0f, hc = 0.0f;
        const int64_t rs = m.rp[row], re = m.rp[row + 1];
        for (int64_t k0 = rs; k0 < re; k0 += 32) {
            const int64_t k = k0 + lane;
            int2 e = make_int2(0, 0);
            if (k < re) e = make_int2(map_col(cm, row, k), __float_as_int(Vals<VT>::one(val, k)));
            stage[w][lane] = e;
            __syncwarp();
            const int cnt = (re - k0) < 32 ? (int)(re - k0) : 32;
            if (live) {
                int t = 0;
                for (; t + 4 <= cnt; t += 4) {
                    int2 st[4];
                    float2 xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) st[u] = stage[w][t + u];
#pragma unroll
                    for (int u = 0; u < 4; ++u) xv[u] = ld_x(x, (int64_t)st[u].x * B + b);
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc_fma(hs, hc, __int_as_float(st[u].y), xv[u]);
                }
                for (; t < cnt; ++t) {
                    const int2 st = stage[w][t];
                    acc_fma(hs, hc, __int_as_float(st.y), ld_x(x, (int64_t)st.x * B + b));
                }
            }
            __syncwarp();
        }
        if (live) {
            float2 v = acc_value(hs, hc);
            if (a.row_scale) {
                const float s = a.row_scale[row];
                v = df_mul_f(v, s);
                if (a.rpow == 2) v = df_mul_f(v, s);
            }
            int64_t pos = row;
            if (om.user) {
                int i, j;
                tiled_coords(row, om.tn, i, j);
                if (i >= om.n || j >= om.n) continue;
                pos = (int64_t)i * om.n + j;
            }
            st_y(y, pos * B + b, df_mul(a.scale, v));
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

// A^T y for every slice fused with the operator epilogue (rows = pixels).
template <typename VT, int MODE>
__global__ void __launch_bounds__(256) spmm_op_kernel(CsrView m, ColMap cm, const VT* __restrict__ val,
                                                      const float2* __restrict__ y, int B, BOp a)
{
    __shared__ int2 stage[kWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rb, chunk;
    const int chunks = (B + 31) / 32;
    block_coords(chunks, rb, chunk);
    const int G = (int)gridDim.x / chunks;
    const int b = chunk * 32 + lane;
    const bool live = slice_live(b, B, MODE == 2 ? nullptr : a.cg, a.sb);
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    for (int64_t row = (int64_t)rb * kWarps + w; row < m.rows; row += (int64_t)G * kWarps) {
        float hs = 0.0f, hc = 0.0f;
        const int64_t rs = m.rp[row], re = m.rp[row + 1];
        for (int64_t k0 = rs; k0 < re; k0 += 32) {
            const int64_t k = k0 + lane;
            int2 e = make_int2(0, 0);
            if (k < re) e = make_int2(map_col(cm, row, k), __float_as_int(Vals<VT>::one(val, k)));
            stage[w][lane] = e;
            __syncwarp();
            const int cnt = (re - k0) < 32 ? (int)(re - k0) : 32;
            if (live) {
                int t = 0;
                for (; t + 4 <= cnt; t += 4) {
                    int2 st[4];
                    float2 xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) st[u] = stage[w][t + u];
#pragma unroll
                    for (int u = 0; u < 4; ++u) xv[u] = __ldg(y + (int64_t)st[u].x * B + b);
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc_fma(hs, hc, __int_as_float(st[u].y), xv[u]);
                }
                for (; t < cnt; ++t) {
                    const int2 st = stage[w][t];
                    acc_fma(hs, hc, __int_as_float(st.y), __ldg(y + (int64_t)st.x * B + b));
                }
            }
            __syncwarp();
        }
        if (live) {
            int i, j;
            tiled_coords(row, a.tn, i, j);
            if (i < a.n && j < a.n) {
                bop_epilogue<MODE>(a, row, i, j, B, b, acc_value(hs, hc), s0, c0, s1, c1);
            } else {
                a.out[row * B + b] = df_zero();  // padding stays zero
                if (MODE == 2) a.p_out[row * B + b] = df_zero();
            }
        }
    }
    float2 v[2] = {acc_value(s0, c0), acc_value(s1, c1)};
    block_partials<2>(v, a.partials, B, G, rb, chunk);
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
    const int b = chunk * 32 + lane;
    const bool live = slice_live(b, B, MODE == 2 ? nullptr : a.cg, a.sb);
    const int n = a.n;
    const int64_t npad = padded_pixels(n);
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    if (live) {
        for (int64_t p = (int64_t)rb * kWarps + w; p < npad; p += (int64_t)G * kWarps) {
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
    float2 v[2] = {acc_value(s0, c0), acc_value(s1, c1)};
    block_partials<2>(v, a.partials, B, G, rb, chunk);
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
    const int b = chunk * 32 + lane;
    float s = 0.0f, c = 0.0f;
    if (slice_live(b, B, cg, sb)) {
        const float2 al = cg[b].alpha_df;
        for (int64_t px = (int64_t)rb * kWarps + w; px < n2; px += (int64_t)G * kWarps) {
            const int64_t e = px * B + b;
            u[e] = df_add(u[e], df_mul(al, p[e]));
            const float2 rn = df_sub(r[e], df_mul(al, q[e]));
            r[e] = rn;
            acc_add(s, c, df_mul(rn, rn));
        }
    }
    float2 v[1] = {acc_value(s, c)};
    block_partials<1>(v, partials, B, G, rb, chunk);
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
    const int b = chunk * 32 + lane;
    if (!slice_live(b, B, cg, sb)) return;
    const float2 be = cg[b].beta_df;
    for (int64_t px = (int64_t)rb * kWarps + w; px < n2; px += (int64_t)G * kWarps) {
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
    const int b = chunk * 32 + lane;
    const int64_t npad = padded_pixels(n);
    float s = 0.0f, cc = 0.0f;
    if (slice_live(b, B, nullptr, sb)) {
        for (int64_t p = (int64_t)rb * kWarps + w; p < npad; p += (int64_t)G * kWarps) {
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
    float2 v[1] = {acc_value(s, cc)};
    block_partials<1>(v, partials, B, G, rb, chunk);
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
__global__ void bwiden_kernel(const float* __restrict__ in, float2* __restrict__ out, int n, int tn, int B)
{
    const int64_t len = padded_pixels(n) * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / B;
        const int b = (int)(e - t * B);
        int i, j;
        tiled_coords(t, tn, i, j);
        out[e] = (i < n && j < n) ? make_float2(in[((int64_t)i * n + j) * B + b], 0.0f) : make_float2(0.0f, 0.0f);
    }
}

__global__ void bnarrow_kernel(const float2* __restrict__ in, float* __restrict__ out, int n, int tn, int B)
{
    const int64_t len = padded_pixels(n) * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / B;
        const int b = (int)(e - t * B);
        int i, j;
        tiled_coords(t, tn, i, j);
        if (i < n && j < n) out[((int64_t)i * n + j) * B + b] = df_to_float(in[e]);
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
__global__ void bto_df_kernel(const float* __restrict__ in, const float* __restrict__ scale, float2* __restrict__ out,
                              int64_t rows, int B)
{
    const int64_t len = rows * B;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = scale ? two_prod(in[i], scale[i / B]) : make_float2(in[i], 0.0f);
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

Grid2 make_grid(const ct_matrix* M, int64_t rows, int B)
{
    Grid2 g;
    g.chunks = (B + 31) / 32;
    const int64_t want = (int64_t)(M->sm_count > 0 ? M->sm_count : 148) * 8 / g.chunks;
    int64_t rb = (rows + kWarps - 1) / kWarps;
    if (rb > want) rb = want;
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
    if (which == 0) return ColMap{M->A.col, nullptr, nullptr, M->g.n_bins, M->n_kept};
    return ColMap{nullptr, M->At.col16, M->band_lo, M->g.n_bins, M->n_kept};
}

// which = 0: rows of A (rays); which = 1: rows of A^T (internal pixels).
template <typename XT, typename YT>
int launch_spmm(const ct_matrix* M, int which, ValKind vk, const XT* x, YT* y, int B, BProd a, cudaStream_t st,
                bool user_out = false)
{
    const Csr& C = which == 0 ? M->A : M->At;
    CsrView m{C.row_ptr, nullptr, C.rows};
    const ColMap cm = colmap_of(M, which);
    const OutMap om{user_out ? 1 : 0, M->g.n, M->tn};
    const Grid2 g = make_grid(M, C.rows, B);
    const int blocks = g.rb * g.chunks;
    if (vk == ValKind::F16)
        spmm_df_kernel<__half, XT, YT><<<blocks, 256, 0, st>>>(m, cm, C.qval, x, y, B, a, om);
    else
        spmm_df_kernel<float, XT, YT><<<blocks, 256, 0, st>>>(m, cm, C.val, x, y, B, a, om);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
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
        const Csr& C = P.M->At;
        CsrView m{C.row_ptr, nullptr, C.rows};
        const ColMap cm = colmap_of(P.M, 1);
        g_used = P.g_rows_t;
        const int blocks = g_used.rb * g_used.chunks;
#define CT_BOP(VT, VAL)                                                                              \
    switch (ep.mode) {                                                                               \
    case 1: spmm_op_kernel<VT, 1><<<blocks, 256, 0, st>>>(m, cm, VAL, w.y, P.B, ep); break;         \
    case 2: spmm_op_kernel<VT, 2><<<blocks, 256, 0, st>>>(m, cm, VAL, w.y, P.B, ep); break;         \
    default: spmm_op_kernel<VT, 3><<<blocks, 256, 0, st>>>(m, cm, VAL, w.y, P.B, ep); break;        \
    }
        if (vk == ValKind::F16) {
            CT_BOP(__half, C.qval)
        } else {
            CT_BOP(float, C.val)
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
    P.g_rows_a = make_grid(M, M->rows, B);
    P.g_rows_t = make_grid(M, M->At.rows, B);
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
        bto_df_kernel<<<grid_blocks(M, M->rows * B), 256, 0, st>>>(in, M->row_scale, w.y, M->rows, B);
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
    bwiden_kernel<<<grid_blocks(M, len), 256, 0, st>>>(rhs, w.rhs, M->g.n, M->tn, B);
    bwiden_kernel<<<grid_blocks(M, len), 256, 0, st>>>(u, w.u, M->g.n, M->tn, B);
    CT_CUDA(cudaGetLastError());
    CT_CHECK(benqueue_cg(P, w.rhs, Pp->max_iters, st));
    bnarrow_kernel<<<grid_blocks(M, len), 256, 0, st>>>(w.u, u, M->g.n, M->tn, B);
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

int split_bregman_batched(ct_matrix* M, const ct_sb_params* Sp, const float* f, float* u, int32_t B,
                          ct_sb_stats* stats, cudaStream_t st)
{
    CT_CHECK(ensure_workspace(M, B, true));
    Workspace& w = M->ws;
    BPlan P;
    CT_CHECK(bmake_plan(M, B, 0.0, Sp->alpha, Sp->lambda, 0.0, Sp->surrogate_r, Sp->surrogate_square,
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
    CT_CUDA(cudaMemsetAsync(w.bx, 0, len * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.by, 0, len * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.vx, 0, len * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.vy, 0, len * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.sb, 0, sizeof(SbSlice) * B, st));
    CT_CUDA(cudaMemcpyAsync(w.u_old, w.u, len * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    const int pblocks = P.g_pix.rb * P.g_pix.chunks;
    const float2 gamma = df_from_double(1.0 / Sp->lambda);
    auto outer = [&](cudaStream_t s) -> int {
        CT_CHECK(benqueue_cg(P, nullptr, Sp->inner_cg_iters, s));
        bsb_shrink_kernel<<<pblocks, 256, 0, s>>>(w.u, w.u_old, w.bx, w.by, w.vx, w.vy, M->g.n, M->tn, B, gamma, w.sb,
                                                  w.partials);
        CT_CUDA(cudaGetLastError());
        finalize_kernel<FIN_SB, 1><<<B, 256, 0, s>>>(w.partials, P.g_pix.rb, B, w.cg, w.sb, Sp->stop_rel_update);
        CT_CUDA(cudaGetLastError());
        return CT_OK;
    };
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CT_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone || Sp->outer_iters <= 2) {
        for (int k = 0; k < Sp->outer_iters; ++k) CT_CHECK(outer(st));
    } else {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        CT_CUDA(cudaStreamBeginCapture(w.cap_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = outer(w.cap_stream);
        cudaError_t e = cudaStreamEndCapture(w.cap_stream, &graph);
        if (rc != CT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        CT_CUDA(e);
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CT_CUDA(e);
        for (int k = 0; k < Sp->outer_iters; ++k) {
            e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) break;
        }
        cudaGraphExecDestroy(exec);
        CT_CUDA(e);
    }
    bnarrow_kernel<<<grid_blocks(M, len), 256, 0, st>>>(w.u, u, M->g.n, M->tn, B);
    CT_CUDA(cudaGetLastError());
    if (stats) {
        std::vector<SbSlice> h(B);
        CT_CUDA(cudaMemcpyAsync(h.data(), w.sb, sizeof(SbSlice) * B, cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaStreamSynchronize(st));
        stats->outer_done = h[0].outer_done;
        stats->first_update_l1 = h[0].first_upd;
        stats->last_update_l1 = h[0].last_upd;
        stats->status = CT_OK;
        for (const SbSlice& s : h) {
            stats->outer_done = std::min(stats->outer_done, s.outer_done);
            if (s.status != CT_OK && stats->status == CT_OK) stats->status = s.status;
        }
        if (stats->status != CT_OK) return fail(stats->status, "split Bregman inner solve failed");
    }
    return CT_OK;
}

}  // namespace ct
