// Device parts of the single-slice sparse products, shared by the kernels of
// solver_ops.cu and the persistent ragged-batch kernel (ragged.cu): the SELL
// views and loaders, the per-slice body of y = A x, and the A^T side's
// sinogram-band staging and row walks.
#pragma once

#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "layout.cuh"
#include "sparse_common.cuh"

namespace ct {

constexpr int kFwdWarps = 8;   // warps per block (= per slice of rays) of y = A x
constexpr int kFwdUnroll = 8;  // chunks each lane of y = A x keeps in flight (untuned default)
constexpr int kAdjWarps = kTilePix / kSliceRows;  // warps per CTA of x = A^T y (one per pixel slice)
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
// COH: read through L2 (data written earlier in the same launch).
template <bool COH = false>
__device__ __forceinline__ float2 gather_x(const float* __restrict__ x, int64_t c)
{
    return make_float2(COH ? __ldcg(x + c) : __ldg(x + c), 0.0f);
}
template <bool COH = false>
__device__ __forceinline__ float2 gather_x(const float2* __restrict__ x, int64_t c)
{
    return COH ? __ldcg(x + c) : __ldg(x + c);
}

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
    __device__ __forceinline__ float2 operator()(int c) const { return gather_x<false>(x, c); }
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
// COH: x was written earlier by the same kernel launch (a persistent
// kernel), so it is read through L2 rather than the non-coherent path.
template <typename VT, typename XT, typename YT, int U, bool COH = false>
__device__ __forceinline__ void fwd_slice(const SellView& m, const int32_t* __restrict__ col,
                                          const VT* __restrict__ val, const XT* __restrict__ x,
                                          YT* __restrict__ y, const ProdArgs& a, int64_t s)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int e8 = lane & 7;
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
            for (int u = 0; u < U; ++u) xx[u] = cc[u] >= 0 ? gather_x<COH>(x, cc[u]) : df_zero();
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
// COH: y was written earlier by the same launch (a persistent kernel): plain
// loads through L2 instead of the L1-allocating asynchronous copies.
template <typename YT, bool COH = false>
__device__ __forceinline__ void stage_band(const BandView& bv, int tile, const YT* __restrict__ y, YT* band)
{
    const int32_t* blo = bv.band_lo + (int64_t)tile * bv.nk;
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int k = threadIdx.x >> 5; k < bv.nk; k += nwarps) {
        const int off = __ldg(bv.band_off + k);
        if (lane < __ldg(bv.band_off + k + 1) - off) {
            const int b = __ldg(blo + k) + lane;
            const bool in = b < bv.nb;
            if (COH)
                band[off + lane] = in ? __ldcg(y + (int64_t)k * bv.nb + b) : YT{};
            else
                cp_async(band + off + lane, y + (in ? (int64_t)k * bv.nb + b : 0), (int)sizeof(YT),
                         in ? (int)sizeof(YT) : 0);
        }
    }
    if (!COH) cp_async_wait_all();
    __syncthreads();
}

// Copies angles [k0, k1) of the tile's sinogram band into shared memory
// (slot off_k0 at band[0]): every angle's W_k bins, one warp per angle and one
// lane per bin, all copies in flight at once; bins past the detector read as
// zero.  Ends with the block synchronised.
template <typename YT, bool COH = false>
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
            if (COH)
                band[(off - base) + lane] = in ? __ldcg(y + (int64_t)k * bv.nb + b) : YT{};
            else
                cp_async(band + (off - base) + lane, y + (in ? (int64_t)k * bv.nb + b : 0), (int)sizeof(YT),
                         in ? (int)sizeof(YT) : 0);
        }
    }
    if (!COH) cp_async_wait_all();
    __syncthreads();
}

// The lane's row of A^T against a band staged chunk by chunk (many angles):
// for each angle chunk, stage it, then walk the row's 8-entry chunks from the
// lane's position until one reaches past the chunk's slots; a chunk that
// straddles two band chunks is walked in both, each time with the other's
// entries masked.  Every lane of the CTA takes part in every staging.
// PAIRS = false walks one 8-entry chunk per step (fewer registers; the same
// order of accumulation, so the same bits).
template <typename VT, typename YT, bool COH = false, bool PAIRS = true>
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
        stage_band_range<YT, COH>(bv, tile, y, band, k0, k1);
        // two 8-entry chunks per step, both loads issued first
        while (c < nch) {
            const int64_t p = base + (int64_t)c * kStep;
            const bool two = PAIRS && c + 1 < nch;
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
            if (!PAIRS) continue;
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
// The lane's whole row, one 8-entry chunk per step with the next chunk's
// loads issued before this chunk's gathers and arithmetic (the same order of
// accumulation as row_part, so the same bits); for register budgets that
// hold two chunks in flight.
template <typename VT, typename CT, typename G>
__device__ __forceinline__ void row_walk_prefetch(const CT* __restrict__ col, const VT* __restrict__ val,
                                                  int64_t base, int nch, const G& g, float& hs, float& hc)
{
    if (nch <= 0) return;
    int ca[8];
    float va[8];
    load8_col(col, base, ca);
    Vals<VT>::load8(val, base, va);
#pragma unroll 2
    for (int c = 0; c < nch; ++c) {
        int cb[8];
        float vb[8];
        const bool more = c + 1 < nch;
        if (more) {
            load8_col(col, base + (c + 1) * kStep, cb);
            Vals<VT>::load8(val, base + (c + 1) * kStep, vb);
        }
        float2 x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = g(ca[t]);
#pragma unroll
        for (int t = 0; t < 8; ++t) acc_fma(hs, hc, va[t], x[t]);
        if (more) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                ca[t] = cb[t];
                va[t] = vb[t];
            }
        }
    }
}

// 16-byte asynchronous global -> shared copy through L2, and its groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Slots of the per-lane ring of row_walk_async and its shared-memory bytes
// per thread (a chunk's 16-bit columns and its values, 16 bytes each piece).
constexpr int kAsyncSlots = 3;
constexpr int kAsyncPieces = 3;
__host__ __device__ inline size_t async_ring_bytes(int threads) { return (size_t)threads * kAsyncSlots * kAsyncPieces * 16; }

// The lane's whole row with the matrix chunks copied ahead into a ring of
// kAsyncSlots slots in shared memory by asynchronous copies (each lane copies
// and reads only its own slots, so no barrier is involved): two chunks are in
// flight while one is gathered and accumulated, without holding them in
// registers.  A slot is refilled only after the chunk it held has been
// consumed.  The same order of accumulation as row_part (the same bits).
// ring: this block's ring, [slot][piece][thread] of 16-byte pieces.
template <typename VT, typename G>
__device__ __forceinline__ void row_walk_async(const uint16_t* __restrict__ col, const VT* __restrict__ val,
                                               int64_t base, int nch, const G& g, float& hs, float& hc, uint4* ring)
{
    constexpr int NV = sizeof(VT) == 4 ? 2 : 1;  // 16-byte pieces of a chunk's values
    const int tid = threadIdx.x, nt = blockDim.x;
    auto slot_piece = [&](int slot, int piece) { return ring + ((size_t)slot * kAsyncPieces + piece) * nt + tid; };
    auto issue = [&](int c) {
        const int slot = c % kAsyncSlots;
        const int64_t p = base + (int64_t)c * kStep;
        cp_async16(slot_piece(slot, 0), col + p);
        cp_async16(slot_piece(slot, 1), val + p);
        if (NV == 2) cp_async16(slot_piece(slot, 2), val + p + 4);
    };
    // every step commits one group (possibly empty), so "all but the newest
    // kAsyncSlots - 1 groups complete" means chunk c has landed
    for (int c = 0; c < kAsyncSlots - 1; ++c) {
        if (c < nch) issue(c);
        cp_async_commit();
    }
    for (int c = 0; c < nch; ++c) {
        if (c + kAsyncSlots - 1 < nch) issue(c + kAsyncSlots - 1);
        cp_async_commit();
        cp_async_wait_group<kAsyncSlots - 1>();
        const int slot = c % kAsyncSlots;
        const uint4 cw = *slot_piece(slot, 0);
        float v[8];
        if (NV == 2) {
            const float4 a = *reinterpret_cast<const float4*>(slot_piece(slot, 1));
            const float4 b = *reinterpret_cast<const float4*>(slot_piece(slot, 2));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
            const uint4 a = *slot_piece(slot, 1);
            const __half2* h = reinterpret_cast<const __half2*>(&a);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float2 f = __half22float2(h[t]);
                v[2 * t] = f.x;
                v[2 * t + 1] = f.y;
            }
        }
        const uint32_t w[4] = {cw.x, cw.y, cw.z, cw.w};
        float2 x[8];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            x[2 * t] = g((int)(w[t] & 0xffffu));
            x[2 * t + 1] = g((int)(w[t] >> 16));
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) acc_fma(hs, hc, v[t], x[t]);
    }
    cp_async_wait_group<0>();
}

// Two rows per lane (rows a and b of A^T, both against the staged band):
// their chunks are walked as one stream a0, b0, a1, b1, ... (a row that has
// run out drops out of it), with the next chunk's loads issued before the
// current chunk's gathers, so a lane keeps one chunk in flight while it works
// on the other row.  Each row is summed in its own order, as row_part sums
// it (the same bits).
template <typename VT, typename G>
__device__ __forceinline__ void row_pair_walk(const uint16_t* __restrict__ col, const VT* __restrict__ val,
                                              int64_t base_a, int nch_a, int64_t base_b, int nch_b, const G& g,
                                              float2& da, float2& db)
{
    float hs[2] = {0.0f, 0.0f}, hc[2] = {0.0f, 0.0f};
    const int K = 2 * max(nch_a, nch_b);
    auto valid = [&](int k) { return (k & 1) ? (k >> 1) < nch_b : (k >> 1) < nch_a; };
    auto addr = [&](int k) { return ((k & 1) ? base_b : base_a) + (int64_t)(k >> 1) * kStep; };
    int k = 0;
    while (k < K && !valid(k)) ++k;
    int cc[8];
    float vv[8];
    if (k < K) {
        load8_col(col, addr(k), cc);
        Vals<VT>::load8(val, addr(k), vv);
    }
    while (k < K) {
        int kn = k + 1;
        while (kn < K && !valid(kn)) ++kn;
        int cn[8];
        float vn[8];
        if (kn < K) {
            load8_col(col, addr(kn), cn);
            Vals<VT>::load8(val, addr(kn), vn);
        }
        float2 x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = g(cc[t]);
        // accumulate into the row's pair: swap the pairs so that slot 0 holds it
        const bool rb = k & 1;
        float s0 = rb ? hs[1] : hs[0], c0 = rb ? hc[1] : hc[0];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc_fma(s0, c0, vv[t], x[t]);
        if (rb) {
            hs[1] = s0;
            hc[1] = c0;
        } else {
            hs[0] = s0;
            hc[0] = c0;
        }
        if (kn < K) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                cc[t] = cn[t];
                vv[t] = vn[t];
            }
        }
        k = kn;
    }
    da = acc_value(hs[0], hc[0]);
    db = acc_value(hs[1], hc[1]);
}

// PREFETCH: 0 = row_part; 1 = row_walk_prefetch; 2 = row_walk_async (ring
// given, after the band in shared memory).
template <typename VT, typename BT, int PREFETCH = 0>
__device__ __forceinline__ float2 band_dot(const BandView& bv, const VT* __restrict__ val, int tile,
                                           const BT* __restrict__ band, int64_t& t, uint4* ring = nullptr)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    t = (int64_t)tile * kTilePix + w * kSliceRows + lane;
    const int len = bv.len[t];
    float hs = 0.0f, hc = 0.0f;
    if (PREFETCH == 2)
        row_walk_async<VT>(bv.col16, val, bv.sp[t >> 5] + lane * kChunk, (len + kChunk - 1) / kChunk,
                           BandGather<BT>{band}, hs, hc, ring);
    else if (PREFETCH == 1)
        row_walk_prefetch<VT>(bv.col16, val, bv.sp[t >> 5] + lane * kChunk, (len + kChunk - 1) / kChunk,
                              BandGather<BT>{band}, hs, hc);
    else
        row_part<VT>(bv.col16, val, bv.sp[t >> 5] + lane * kChunk, (len + kChunk - 1) / kChunk, 0, 2,
                     BandGather<BT>{band}, hs, hc);
    return acc_value(hs, hc);
}


}  // namespace ct
