// The Fourier-domain data term (Sec. 2, Eqs. four_obj, SBFFT) evaluated by
// Gaussian gridding onto a 2N x 2N periodic grid (Sec. 3.1), with the two
// gridding products either kept separate (interpolate with G, spread with
// G^T) or fused into the precomputed sparse matrix C = G^T G (convolution
// fusing, Eq. fusedop):
//
//   F        = c Phi G FFT Z E,          c = 1 / (M_r^2 sqrt(n_bins))
//   Re F^H F = c^2 E Z^T FFT^H C FFT Z E (Phi, unit phases, cancels)
//
// E is the per-dimension deconvolution sqrt(pi/tau) exp(k^2 tau), Z the zero
// padding of the N x N image into the M_r = 2N grid (frequency k stored at
// k mod M_r), FFT the unnormalised 2-D DFT and FFT^H its conjugate.
//
// GB300 layout: C is stored by diagonal, one FP32 entry per grid point and
// offset d in [-2 m_sp, 2 m_sp]^2 of the periodic grid, no column indices,
// ordered tile by tile (16 x 16 grid points, all offsets of a tile in one
// contiguous run), so a block of the product streams one contiguous run
// with its input tile and halo staged in shared memory.  Grid and sample
// vectors are complex double-float (float4), accumulated with error-free
// transformations.  The gridding weights are separable: a sample keeps its
// window's floor point and 2 (2 m_sp + 1) FP32 weights.  The spread is a
// gather over the samples binned by cell (host counting sort), so every sum
// has a fixed order and results are bitwise reproducible.  The FFTs are
// radix-2 passes in shared memory, two transforms per block.  Tables are
// computed on the host in FP64 and rounded once: the weights, the phases
// and C to FP32, the FFT twiddles and the pixel scaling sqrt(c) E to
// double-float (a fixed-count CG tolerates a symmetric FP32 perturbation of
// the weights, but not a non-unitary FFT or a pixel scaling that is not
// separable).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "layout.cuh"
#include "op_epilogue.cuh"
#include "reduce.cuh"

namespace ct {

struct FourierOp {
    int n = 0, mr = 0, lg = 0;   // image side, grid side M_r = 2N, log2(M_r)
    int msp = 0, win = 0, nd = 0;  // window half-width, 2 msp + 1, 4 msp + 1
    int mode = CT_FOURIER_FUSED;
    double tau = 0.0;
    int n_bins = 0, n_kept = 0;
    int64_t J = 0;
    double c = 0.0;               // 1 / (M_r^2 sqrt(n_bins))
    std::vector<double> h_wx, h_wy;  // sample frequencies (host, FP64)
    float2* sE = nullptr;         // [n] sqrt(c) E(i - n/2), double-float
    int2* base = nullptr;         // [J] floor point of each sample's window, per dimension
    float* wgt = nullptr;         // [J][2][win] 1-D weights along x, then y
    float2* phase = nullptr;      // [J] exp(-i (w_x + w_y) / 2)
    int32_t* cell_start = nullptr;  // [M_r^2 + 1] samples binned by floor cell
    int32_t* cell_idx = nullptr;    // [J]
    float* C = nullptr;           // fused matrix by diagonal, tile-major (see c_index)
    uint8_t* tile_nz = nullptr;   // [(M_r/16)^2] 1 if a 16 x 16 tile has any nonzero of C
    float4* tw = nullptr;         // [M_r / 2] exp(-2 pi i k / M_r), double-float
    float2* sino_tw = nullptr;    // [2 n_bins] exp(-pi i q / n_bins)
    float4 *X = nullptr, *Y = nullptr, *S = nullptr;  // grid, grid, samples (complex double-float)
    int fft_T = 2;                // transforms per FFT block
};

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kFftThreads = 256;
constexpr int kDiaTile = 16;  // fused product: 16 x 16 grid points per block
// dynamic shared memory bounds: FFT 2 x (4096 + 1) complex double-float
// points, fused product (16 + 48)^2 points, fused build 96 KB of accumulators
constexpr int kFftSmemMax = 2 * 4097 * 16;
constexpr int kDiaSmemMax = 64 * 64 * 16;
constexpr int kBuildSmemMax = 96 * 1024;

// ---- complex double-float values: float4 (re.hi, re.lo, im.hi, im.lo) ------
// The grid and sample vectors of the solver's products are carried in
// double-float: a fixed number of CG steps amplifies rounding that changes
// from one product to the next, while the FP32 tables (weights, C) are a
// fixed, symmetric perturbation of the operator.
__device__ __forceinline__ float2 re_of(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 im_of(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cdf(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }

__device__ __forceinline__ float4 cdf_add(float4 a, float4 b)
{
    return cdf(df_add(re_of(a), re_of(b)), df_add(im_of(a), im_of(b)));
}
__device__ __forceinline__ float4 cdf_sub(float4 a, float4 b)
{
    return cdf(df_sub(re_of(a), re_of(b)), df_sub(im_of(a), im_of(b)));
}
// a * w for an FP32 complex w
__device__ __forceinline__ float4 cdf_mul_c(float4 a, float2 w)
{
    const float2 ar = re_of(a), ai = im_of(a);
    return cdf(df_sub(df_mul_f(ar, w.x), df_mul_f(ai, w.y)), df_add(df_mul_f(ar, w.y), df_mul_f(ai, w.x)));
}
__device__ __forceinline__ float4 cdf_mul_f(float4 a, float s) { return cdf(df_mul_f(re_of(a), s), df_mul_f(im_of(a), s)); }

// a * w for a double-float complex w = (wr, wi)
__device__ __forceinline__ float4 cdf_mul_cdf(float4 a, float2 wr, float2 wi)
{
    const float2 ar = re_of(a), ai = im_of(a);
    return cdf(df_sub(df_mul(ar, wr), df_mul(ai, wi)), df_add(df_mul(ar, wi), df_mul(ai, wr)));
}

// Compensated accumulator of a complex sum of FP32-weighted terms.
struct CAcc {
    float rs = 0.0f, rc = 0.0f, is = 0.0f, ic = 0.0f;
};
__device__ __forceinline__ void cacc_fma(CAcc& a, float w, float4 x)
{
    acc_fma(a.rs, a.rc, w, re_of(x));
    acc_fma(a.is, a.ic, w, im_of(x));
}
__device__ __forceinline__ float4 cacc_value(const CAcc& a)
{
    return cdf(acc_value(a.rs, a.rc), acc_value(a.is, a.ic));
}

// Position of the fused matrix's entry (m, m + d) for plane d (0 <= d < nd^2)
// and grid point m = (my, mx): the 4N^2 grid in 16 x 16 tiles, and per tile
// its nd^2 planes of 256 entries, so that a block of the product streams its
// tile's coefficients as one contiguous run.
__host__ __device__ __forceinline__ int64_t c_index(int64_t d, int my, int mx, int mr, int nd2)
{
    const int64_t tile = (int64_t)(my >> 4) * (mr >> 4) + (mx >> 4);
    return ((tile * nd2 + d) << 8) + ((my & 15) << 4) + (mx & 15);
}

// Work of a solver product is skipped once the split-Bregman run has stopped
// or (CG modes 1, 3) the slice has converged; the epilogue applies the same rule.
struct Gate {
    const int32_t* gate;
    const CgSlice* cg;
    int need_active;
};

__device__ __forceinline__ bool gated(const Gate& g)
{
    if (g.gate && *g.gate) return true;
    return g.need_active && g.cg && !g.cg->active;
}

// Image -> grid: X[k mod M_r] = sE(k_y) sE(k_x) x(k), zero elsewhere (sE =
// sqrt(c) E in double-float: the pixel scaling must be separable to full
// precision; per-pixel FP32 products sE_i sE_j perturb the operator enough
// for a 20-step CG to drift by 6e-3).  DF selects the solver's double-float
// tiled input, else a row-major FP32 image.
template <bool DF>
__global__ void __launch_bounds__(256) pad_kernel(const void* __restrict__ in, float4* __restrict__ X, int n,
                                                  int tn, int mr, const float2* __restrict__ sE, Gate g)
{
    if (gated(g)) return;
    const int64_t len = (int64_t)mr * mr;
    const int h = n / 2;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < len; m += (int64_t)gridDim.x * blockDim.x) {
        const int my = (int)(m / mr), mx = (int)(m - (int64_t)my * mr);
        const int ky = my < h ? my : my - mr, kx = mx < h ? mx : mx - mr;
        float2 v = df_zero();
        if (ky >= -h && kx >= -h) {
            const int i = ky + h, j = kx + h;
            const float2 x = DF ? static_cast<const float2*>(in)[tiled_index(i, j, tn)]
                                : make_float2(static_cast<const float*>(in)[(int64_t)i * n + j], 0.0f);
            v = df_mul(df_mul(x, sE[i]), sE[j]);
        }
        X[m] = cdf(v, df_zero());
    }
}

// T transforms of length L = 2^lg along one axis of the M_r x M_r grid:
// element t of transform r at data[r * rstride + t * estride].  Loaded in
// bit-reversed order into shared memory (row pitch L + 1), lg radix-2
// passes, stored back.  INV: conjugate twiddles (unnormalised inverse).
// The twiddles are double-float: FP32 twiddles make the transform slightly
// non-unitary, and the fixed-count CG of a later Bregman update amplifies
// that perturbation by orders of magnitude.
// keep > 0: only the transforms r < keep and r >= M_r - keep (the rows that
// hold the zero-padded image, or the rows the crop reads) are computed; block
// b takes the compact indices b T .. b T + T - 1.
template <bool INV>
__global__ void __launch_bounds__(kFftThreads) fft_kernel(float4* __restrict__ data, int lg, int T,
                                                          int64_t estride, int64_t rstride,
                                                          const float4* __restrict__ tw, int keep, Gate g)
{
    if (gated(g)) return;
    extern __shared__ float4 sbuf[];
    const int L = 1 << lg;
    const int pitch = L + 1;
    int64_t r0 = (int64_t)blockIdx.x * T;
    if (keep > 0 && r0 >= keep) r0 += L - 2 * keep;  // T divides keep: a block never straddles the gap
    const int total = T * L;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int r, t;
        if (estride == 1) {
            r = idx >> lg;
            t = idx & (L - 1);
        } else {
            t = idx / T;
            r = idx - t * T;
        }
        const int rv = (int)(__brev((unsigned)t) >> (32 - lg));
        sbuf[r * pitch + rv] = data[(r0 + r) * rstride + (int64_t)t * estride];
    }
    __syncthreads();
    for (int s = 0; s < lg; ++s) {
        const int half = 1 << s;
        for (int b = threadIdx.x; b < total / 2; b += blockDim.x) {
            const int r = b >> (lg - 1);
            const int k = b & (L / 2 - 1);
            const int pos = k & (half - 1);
            const int i0 = ((k >> s) << (s + 1)) + pos;
            const float4 w = tw[pos << (lg - 1 - s)];
            const float2 wr = make_float2(w.x, w.y);
            const float2 wi = INV ? make_float2(-w.z, -w.w) : make_float2(w.z, w.w);
            float4* row = sbuf + r * pitch;
            const float4 a = row[i0];
            const float4 bw = cdf_mul_cdf(row[i0 + half], wr, wi);
            row[i0] = cdf_add(a, bw);
            row[i0 + half] = cdf_sub(a, bw);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int r, t;
        if (estride == 1) {
            r = idx >> lg;
            t = idx & (L - 1);
        } else {
            t = idx / T;
            r = idx - t * T;
        }
        data[(r0 + r) * rstride + (int64_t)t * estride] = sbuf[r * pitch + t];
    }
}

// Y = C X with C by diagonal: Y[m] = sum_d C[d][m] X[(m + d) mod M_r].  A
// block takes a 16 x 16 tile of grid points; the tile of X with its halo of
// 2 m_sp on every side is staged in shared memory; the tile's coefficients
// are one contiguous run, read once in a fixed order.
// Tiles whose rows of C are all zero (no sample within reach: the corners
// of the frequency square outside the sampled disc) write zeros and read
// nothing.
__global__ void __launch_bounds__(256, 6) dia_kernel(const float* __restrict__ C, const float4* __restrict__ X,
                                                  float4* __restrict__ Y, int mr, int msp,
                                                  const uint8_t* __restrict__ tile_nz, Gate g)
{
    if (gated(g)) return;
    extern __shared__ float4 xs[];
    const int nd = 4 * msp + 1, h = 2 * msp;
    const int P = kDiaTile + nd - 1;
    const int tiles = mr / kDiaTile;
    const int y0 = (blockIdx.x / tiles) * kDiaTile, x0 = (blockIdx.x % tiles) * kDiaTile;
    if (!tile_nz[blockIdx.x]) {
        const int64_t m = (int64_t)(y0 + threadIdx.x / kDiaTile) * mr + x0 + threadIdx.x % kDiaTile;
        Y[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    for (int idx = threadIdx.x; idx < P * P; idx += blockDim.x) {
        const int ry = idx / P, cx = idx - ry * P;
        const int yy = (y0 - h + ry + 2 * mr) % mr;
        const int xx = (x0 - h + cx + 2 * mr) % mr;
        xs[idx] = X[(int64_t)yy * mr + xx];
    }
    __syncthreads();
    const int ty = threadIdx.x / kDiaTile, tx = threadIdx.x % kDiaTile;
    const int64_t m = (int64_t)(y0 + ty) * mr + x0 + tx;
    // eight plane loads issued before their arithmetic, so that enough bytes
    // are in flight to cover the memory latency
    CAcc acc;
    const float* Ct = C + (((int64_t)blockIdx.x * nd * nd) << 8) + threadIdx.x;  // this tile's run
    for (int dy = 0; dy < nd; ++dy) {
        const float* Cp = Ct + (((int64_t)dy * nd) << 8);
        const float4* xr = xs + (ty + dy) * P + tx;
        int dx = 0;
        for (; dx + 8 <= nd; dx += 8) {
            float cv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) cv[k] = __ldcs(Cp + ((dx + k) << 8));
#pragma unroll
            for (int k = 0; k < 8; ++k) cacc_fma(acc, cv[k], xr[dx + k]);
        }
        for (; dx < nd; ++dx) cacc_fma(acc, __ldcs(Cp + (dx << 8)), xr[dx]);
    }
    Y[m] = cacc_value(acc);
}

// Interpolation S_j = sum_t (w_x(t_x) w_y(t_y)) X[b_j + t] over the window,
// with the weight products rounded to FP32 exactly as the spread rounds them,
// so that interpolation and spread are transposes of one matrix and G^T G
// stays symmetric (an asymmetric perturbation of 1e-7 is enough to throw a
// fixed-count CG off by 1e-3).  PUB: FP32 complex output times the sample's
// phase (F x).
template <bool PUB>
__global__ void __launch_bounds__(256) interp_kernel(const float4* __restrict__ X, void* __restrict__ out, int64_t J,
                                                     int mr, int msp, const int2* __restrict__ base,
                                                     const float* __restrict__ wgt,
                                                     const float2* __restrict__ phase, Gate g)
{
    if (gated(g)) return;
    const int win = 2 * msp + 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
        const int2 b = base[j];
        const float* wx = wgt + j * 2 * win;
        const float* wy = wx + win;
        CAcc acc;
        for (int ty = 0; ty < win; ++ty) {
            const int yy = (b.y - msp + ty + 2 * mr) % mr;
            const float4* row = X + (int64_t)yy * mr;
            for (int tx = 0; tx < win; ++tx) cacc_fma(acc, wx[tx] * wy[ty], row[(b.x - msp + tx + 2 * mr) % mr]);
        }
        const float4 v = cacc_value(acc);
        if (PUB) {
            const float2 p = phase[j];
            const float vr = df_to_float(re_of(v)), vi = df_to_float(im_of(v));
            static_cast<float2*>(out)[j] = make_float2(vr * p.x - vi * p.y, vr * p.y + vi * p.x);
        } else {
            static_cast<float4*>(out)[j] = v;
        }
    }
}

// Spread as a gather: Y[m] = sum over samples j whose window holds m of
// w_j(m) S_j.  Sample j with floor point b covers m at offset t = m - b, so m
// visits the cells m - t, t in [-msp, msp]^2, in a fixed order.
__global__ void __launch_bounds__(256) spread_kernel(const float4* __restrict__ S, float4* __restrict__ Y, int mr,
                                                     int msp, const int32_t* __restrict__ cell_start,
                                                     const int32_t* __restrict__ cell_idx,
                                                     const float* __restrict__ wgt, Gate g)
{
    if (gated(g)) return;
    const int win = 2 * msp + 1;
    const int64_t len = (int64_t)mr * mr;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < len; m += (int64_t)gridDim.x * blockDim.x) {
        const int my = (int)(m / mr), mx = (int)(m - (int64_t)my * mr);
        CAcc acc;
        for (int ty = -msp; ty <= msp; ++ty) {
            const int cy = (my - ty + mr) % mr;
            for (int tx = -msp; tx <= msp; ++tx) {
                const int cx = (mx - tx + mr) % mr;
                const int64_t cell = (int64_t)cy * mr + cx;
                const int e = cell_start[cell + 1];
                for (int q = cell_start[cell]; q < e; ++q) {
                    const int j = cell_idx[q];
                    const float* w = wgt + (int64_t)j * 2 * win;
                    cacc_fma(acc, w[tx + msp] * w[win + ty + msp], S[j]);
                }
            }
        }
        Y[m] = cacc_value(acc);
    }
}

// C[d][m] = sum_j w_j(m) w_j(m + d) over the samples whose window holds both,
// with w_j the FP32-rounded weight products the interpolation and spread
// use.  A block owns G consecutive grid points of a row with their nd^2
// compensated accumulators in shared memory (near the origin thousands of
// samples overlap; plain FP32 sums there would perturb the operator's
// largest entries by ~1e-5); a warp walks one grid point's samples in the
// fixed cell order and its lanes take the sample's window points t' (d = t'
// - t is then distinct per lane).  The planes are written coalesced, each
// entry rounded once.
__global__ void __launch_bounds__(256) build_fused_kernel(float* __restrict__ C, int mr, int msp, int G,
                                                          const int32_t* __restrict__ cell_start,
                                                          const int32_t* __restrict__ cell_idx,
                                                          const float* __restrict__ wgt)
{
    extern __shared__ float2 acc[];
    const int win = 2 * msp + 1, nd = 4 * msp + 1, nd2 = nd * nd;
    const int64_t m0 = (int64_t)blockIdx.x * G;
    for (int i = threadIdx.x; i < G * nd2; i += blockDim.x) acc[i] = make_float2(0.0f, 0.0f);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int gp = warp; gp < G; gp += nwarps) {
        const int64_t m = m0 + gp;
        const int my = (int)(m / mr), mx = (int)(m - (int64_t)my * mr);
        float2* a = acc + gp * nd2;
        for (int ty = -msp; ty <= msp; ++ty) {
            const int cy = (my - ty + mr) % mr;
            for (int tx = -msp; tx <= msp; ++tx) {
                const int cx = (mx - tx + mr) % mr;
                const int64_t cell = (int64_t)cy * mr + cx;
                const int e = cell_start[cell + 1];
                for (int q = cell_start[cell]; q < e; ++q) {
                    const float* w = wgt + (int64_t)cell_idx[q] * 2 * win;
                    const float wm = w[tx + msp] * w[win + ty + msp];
                    for (int t2 = lane; t2 < win * win; t2 += 32) {
                        const int uy = t2 / win - msp, ux = t2 - (t2 / win) * win - msp;
                        const int slot = (uy - ty + 2 * msp) * nd + (ux - tx + 2 * msp);
                        float2 v = a[slot];
                        acc_fma(v.x, v.y, wm, make_float2(w[ux + msp] * w[win + uy + msp], 0.0f));
                        a[slot] = v;
                    }
                    __syncwarp();
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G * nd2; i += blockDim.x) {
        const int d = i / G, gp = i - d * G;
        const float2 v = acc[gp * nd2 + d];
        const int64_t m = m0 + gp;
        const int my = (int)(m / mr), mx = (int)(m - (int64_t)my * mr);
        C[c_index(d, my, mx, mr, nd2)] = acc_value(v.x, v.y).x;
    }
}

// tile_nz[t] = 1 if any plane of C has a nonzero entry in 16 x 16 tile t.
__global__ void __launch_bounds__(256) tile_nonzero_kernel(const float* __restrict__ C, int mr, int nd2,
                                                           uint8_t* __restrict__ tile_nz)
{
    const float* Ct = C + (((int64_t)blockIdx.x * nd2) << 8) + threadIdx.x;
    int nz = 0;
    for (int d = 0; d < nd2 && !nz; ++d) nz = Ct[(int64_t)d << 8] != 0.0f;
    nz = __syncthreads_or(nz);
    if (threadIdx.x == 0) tile_nz[blockIdx.x] = (uint8_t)(nz != 0);
}

// Makes the fused matrix exactly symmetric: the entry (m, m + d) of plane d
// and its mirror (m + d, m) of plane -d, accumulated in different orders,
// both become their mean.  Thread per (m, d) with d in the half-set
// d_y > 0, or d_y == 0 and d_x > 0, so every pair is visited once.
__global__ void __launch_bounds__(256) sym_fused_kernel(float* __restrict__ C, int mr, int msp)
{
    const int nd = 4 * msp + 1, h = 2 * msp;
    const int64_t plane = (int64_t)mr * mr;
    const int64_t half = (int64_t)(nd * nd - 1) / 2;  // planes after the centre one
    const int64_t total = half * plane;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t dp = (nd * nd - 1) / 2 + 1 + t / plane;  // plane index past the centre
        const int64_t m = t % plane;
        const int dy = (int)(dp / nd) - h, dx = (int)(dp % nd) - h;
        const int64_t dn = (int64_t)(-dy + h) * nd + (-dx + h);  // mirror plane
        const int my = (int)(m / mr), mx = (int)(m % mr);
        const int my2 = (my + dy + 2 * mr) % mr, mx2 = (mx + dx + 2 * mr) % mr;
        const int64_t a = c_index(dp, my, mx, mr, nd * nd), b = c_index(dn, my2, mx2, mr, nd * nd);
        const float v = 0.5f * (C[a] + C[b]);
        C[a] = v;
        C[b] = v;
    }
}

// Grid -> image, solver epilogue: N(p) = (c E E) Re(Y) at every pixel, then
// the CG operator epilogue of `MODE`.
template <int MODE>
__global__ void __launch_bounds__(256) crop_op_kernel(OpEpilogue a, const float4* __restrict__ Y, int n, int tn,
                                                      int64_t npad, int mr, const float2* __restrict__ sE)
{
    if (a.gate && *a.gate) return;
    if (MODE != 2 && !a.cg->active) return;
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    const int h = n / 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npad; p += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(p, tn, i, j);
        if (i >= n || j >= n) {
            a.out[p] = df_zero();
            if (MODE == 2) a.p_out[p] = df_zero();
            continue;
        }
        const int my = (i - h + mr) % mr, mx = (j - h + mr) % mr;
        const float2 v = df_mul(df_mul(re_of(Y[(int64_t)my * mr + mx]), sE[i]), sE[j]);
        op_epilogue<MODE>(a, n, tn, p, i, j, v, s0, c0, s1, c1);
    }
    op_finish<MODE>(a, s0, c0, s1, c1);
}

// Grid -> image: out = scale sE sE Re(Y), row-major FP32 or tiled double-float.
template <bool DF>
__global__ void __launch_bounds__(256) crop_kernel(const float4* __restrict__ Y, void* __restrict__ out, int n,
                                                   int tn, int mr, const float2* __restrict__ sE, float2 scale)
{
    const int h = n / 2;
    const int64_t len = DF ? padded_pixels(n) : (int64_t)n * n;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len; p += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        if (DF) {
            tiled_coords(p, tn, i, j);
            if (i >= n || j >= n) {
                static_cast<float2*>(out)[p] = df_zero();
                continue;
            }
        } else {
            i = (int)(p / n);
            j = (int)(p - (int64_t)i * n);
        }
        const int my = (i - h + mr) % mr, mx = (j - h + mr) % mr;
        const float2 v = df_mul(df_mul(df_mul(re_of(Y[(int64_t)my * mr + mx]), sE[i]), sE[j]), scale);
        if (DF)
            static_cast<float2*>(out)[p] = v;
        else
            static_cast<float*>(out)[p] = df_to_float(v);
    }
}

// fhat_j = n_bins^{-1/2} sum_b f_b exp(-i rho_m s_b) for one angle per block:
// the phase index (m - h)(2b - n_bins + 1) mod 2 n_bins steps by 2(m - h).
// PUB: FP32 complex output; else double-float times conj(Phi_j), the input
// of the adjoint.
template <bool PUB>
__global__ void __launch_bounds__(256) sino_dft_kernel(const float* __restrict__ f, void* __restrict__ out, int nb,
                                                       const float2* __restrict__ stw, float inv_sqrt_nb,
                                                       const float2* __restrict__ phase)
{
    extern __shared__ float frow[];
    const int k = blockIdx.x;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) frow[b] = f[(int64_t)k * nb + b];
    __syncthreads();
    const int two = 2 * nb, h = nb / 2;
    for (int m = threadIdx.x; m < nb; m += blockDim.x) {
        const int64_t a = ((int64_t)(m - h) % two + two) % two;
        const int step = (int)((2 * a) % two);
        int q = (int)(((a * (int64_t)(1 - nb)) % two + two) % two);
        CAcc acc;
        for (int b = 0; b < nb; ++b) {
            const float2 w = stw[q];
            acc_fma(acc.rs, acc.rc, w.x, make_float2(frow[b], 0.0f));
            acc_fma(acc.is, acc.ic, w.y, make_float2(frow[b], 0.0f));
            q += step;
            if (q >= two) q -= two;
        }
        const float4 v = cdf_mul_f(cacc_value(acc), inv_sqrt_nb);
        const int64_t j = (int64_t)k * nb + m;
        if (PUB) {
            static_cast<float2*>(out)[j] = make_float2(df_to_float(re_of(v)), df_to_float(im_of(v)));
        } else {
            const float2 p = phase[j];
            static_cast<float4*>(out)[j] = cdf_mul_c(v, make_float2(p.x, -p.y));
        }
    }
}

// S = conj(Phi) y for FP32 complex y (the adjoint's input).
__global__ void conj_phase_kernel(const float2* __restrict__ in, float4* __restrict__ out,
                                  const float2* __restrict__ phase, int64_t J)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = phase[j], y = in[j];
        out[j] = cdf_mul_c(cdf(make_float2(y.x, 0.0f), make_float2(y.y, 0.0f)), make_float2(p.x, -p.y));
    }
}

int alloc_bytes(void** p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 1);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return fail(CT_ERR_OOM, "device allocation failed (Fourier operator)");
    }
    CT_CUDA(e);
    return CT_OK;
}

template <typename T>
int upload(T** d, const std::vector<T>& h)
{
    CT_CHECK(alloc_bytes((void**)d, h.size() * sizeof(T)));
    CT_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return CT_OK;
}

int grid_blocks(const ct_matrix* M, int64_t items)
{
    return grid_for(M, items, 256, 8);
}

size_t fft_smem(const FourierOp& F) { return (size_t)F.fft_T * (F.mr + 1) * sizeof(float4); }

size_t dia_smem(const FourierOp& F)
{
    const size_t P = kDiaTile + F.nd - 1;
    return P * P * sizeof(float4);
}

// 2-D FFT of a grid buffer in place (rows, then columns).
// 2-D FFT of a grid buffer in place.  Forward: rows, then columns; only the
// N rows that hold the zero-padded image need a row transform.  Inverse: the
// mirror order, columns then rows, and only the N rows the crop reads.
int fft2(const FourierOp& F, float4* data, bool inv, const Gate& g, cudaStream_t st)
{
    const int all = F.mr / F.fft_T, half = F.n / F.fft_T, keep = F.n / 2;
    const size_t sm = fft_smem(F);
    if (inv) {
        fft_kernel<true><<<all, kFftThreads, sm, st>>>(data, F.lg, F.fft_T, F.mr, 1, F.tw, 0, g);
        fft_kernel<true><<<half, kFftThreads, sm, st>>>(data, F.lg, F.fft_T, 1, F.mr, F.tw, keep, g);
    } else {
        fft_kernel<false><<<half, kFftThreads, sm, st>>>(data, F.lg, F.fft_T, 1, F.mr, F.tw, keep, g);
        fft_kernel<false><<<all, kFftThreads, sm, st>>>(data, F.lg, F.fft_T, F.mr, 1, F.tw, 0, g);
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// Y = C X (fused) or Y = G^T G X (interpolate into S, spread back).
int grid_normal(const ct_matrix* M, const FourierOp& F, const Gate& g, cudaStream_t st)
{
    if (F.mode == CT_FOURIER_FUSED) {
        const int tiles = F.mr / kDiaTile;
        dia_kernel<<<tiles * tiles, kDiaTile * kDiaTile, dia_smem(F), st>>>(F.C, F.X, F.Y, F.mr, F.msp, F.tile_nz, g);
    } else {
        interp_kernel<false><<<grid_blocks(M, F.J), 256, 0, st>>>(F.X, F.S, F.J, F.mr, F.msp, F.base, F.wgt,
                                                                  nullptr, g);
        CT_CUDA(cudaGetLastError());
        spread_kernel<<<grid_blocks(M, (int64_t)F.mr * F.mr), 256, 0, st>>>(F.S, F.Y, F.mr, F.msp, F.cell_start,
                                                                            F.cell_idx, F.wgt, g);
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// Y = G^T S then the inverse FFT (the adjoint's grid side).
int spread_inverse(const ct_matrix* M, const FourierOp& F, cudaStream_t st)
{
    const Gate none{nullptr, nullptr, 0};
    spread_kernel<<<grid_blocks(M, (int64_t)F.mr * F.mr), 256, 0, st>>>(F.S, F.Y, F.mr, F.msp, F.cell_start,
                                                                        F.cell_idx, F.wgt, none);
    CT_CUDA(cudaGetLastError());
    return fft2(F, F.Y, true, none, st);
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

int64_t fourier_stored_weights(const ct_matrix* M)
{
    const FourierOp& F = *M->fourier;
    if (F.mode == CT_FOURIER_FUSED) return (int64_t)F.nd * F.nd * F.mr * F.mr;
    return F.J * F.win * F.win;
}

void free_fourier(ct_matrix* M)
{
    FourierOp* F = M->fourier;
    if (!F) return;
    void* ps[] = {F->sE, F->base, F->wgt, F->phase, F->cell_start, F->cell_idx, F->C, F->tile_nz, F->tw, F->sino_tw,
                  F->X, F->Y, F->S};
    for (void* p : ps) cudaFree(p);
    delete F;
    M->fourier = nullptr;
}

int check_fourier_params(const ct_geometry& g, const ct_fourier_params& P)
{
    const int n = g.n;
    if (!is_pow2(n) || n < 16 || n > 2048)
        return fail(CT_ERR_UNSUPPORTED, "the Fourier operator needs N a power of two in [16, 2048]");
    if (P.m_sp < 1 || P.m_sp > 12) return fail(CT_ERR_ARG, "m_sp must be in [1, 12]");
    if (2 * P.m_sp + 1 > 2 * n) return fail(CT_ERR_ARG, "the window 2 m_sp + 1 exceeds the 2N grid");
    if (!(P.tau >= 0.0) || !std::isfinite(P.tau)) return fail(CT_ERR_ARG, "tau must be finite and >= 0");
    if (P.mode != CT_FOURIER_FUSED && P.mode != CT_FOURIER_GRIDDING)
        return fail(CT_ERR_ARG, "mode must be CT_FOURIER_FUSED or CT_FOURIER_GRIDDING");
    return CT_OK;
}

int build_fourier(ct_matrix* M, const ct_fourier_params* P)
{
    const ct_geometry& g = M->g;
    const int n = g.n;
    CT_CHECK(check_fourier_params(g, *P));
    FourierOp* F = new (std::nothrow) FourierOp();
    if (!F) return fail(CT_ERR_OOM, "host allocation failed");
    M->fourier = F;
    F->n = n;
    F->mr = 2 * n;
    F->lg = 0;
    while ((1 << F->lg) < F->mr) ++F->lg;
    F->msp = P->m_sp;
    F->win = 2 * P->m_sp + 1;
    F->nd = 4 * P->m_sp + 1;
    F->mode = P->mode;
    F->tau = P->tau > 0.0 ? P->tau : (double)P->m_sp / ((double)n * n);
    F->n_bins = g.n_bins;
    std::vector<double> hc, hs;
    angle_directions(g, hc, hs);
    F->n_kept = (int)hc.size();
    M->n_kept = F->n_kept;
    F->J = (int64_t)F->n_kept * g.n_bins;
    M->rows = F->J;
    M->cols = (int64_t)n * n;
    M->tn = tiles_per_side(n);
    M->npad = padded_pixels(n);
    const int mr = F->mr, msp = F->msp, win = F->win, nb = g.n_bins;
    const int64_t J = F->J;
    F->c = 1.0 / ((double)mr * mr * std::sqrt((double)nb));

    // samples, windows and weights (FP64, rounded once)
    F->h_wx.resize(J);
    F->h_wy.resize(J);
    std::vector<int2> base(J);
    std::vector<float> wgt((size_t)J * 2 * win);
    std::vector<float2> phase(J);
    std::vector<int32_t> count((size_t)mr * mr + 1, 0);
    const double two_pi = 2.0 * kPi;
    for (int k = 0; k < F->n_kept; ++k) {
        for (int m = 0; m < nb; ++m) {
            const int64_t j = (int64_t)k * nb + m;
            const double rho = two_pi * (double)(m - nb / 2) / (double)nb;
            const double wv[2] = {hc[k] * rho, hs[k] * rho};
            F->h_wx[j] = wv[0];
            F->h_wy[j] = wv[1];
            int b[2];
            for (int a = 0; a < 2; ++a) {
                b[a] = (int)std::floor(wv[a] * mr / two_pi);
                for (int t = -msp; t <= msp; ++t) {
                    const double d = wv[a] - two_pi * (double)(b[a] + t) / mr;
                    wgt[(size_t)j * 2 * win + a * win + (t + msp)] = (float)std::exp(-(d * d) / (4.0 * F->tau));
                }
            }
            base[j] = make_int2(b[0], b[1]);
            const double ph = -0.5 * (wv[0] + wv[1]);
            phase[j] = make_float2((float)std::cos(ph), (float)std::sin(ph));
            const int64_t cell = (int64_t)(((b[1] % mr) + mr) % mr) * mr + (((b[0] % mr) + mr) % mr);
            ++count[cell + 1];
        }
    }
    // counting sort of the samples by cell (stable in j)
    for (size_t i = 1; i < count.size(); ++i) count[i] += count[i - 1];
    std::vector<int32_t> cell_idx(J);
    {
        std::vector<int32_t> fill(count.begin(), count.end() - 1);
        for (int64_t j = 0; j < J; ++j) {
            const int64_t cell = (int64_t)(((base[j].y % mr) + mr) % mr) * mr + (((base[j].x % mr) + mr) % mr);
            cell_idx[fill[cell]++] = (int32_t)j;
        }
    }
    std::vector<float2> sE(n);
    for (int i = 0; i < n; ++i) {
        const double k = (double)(i - n / 2);
        sE[i] = df_from_double(std::sqrt(F->c) * std::sqrt(kPi / F->tau) * std::exp(k * k * F->tau));
    }
    std::vector<float4> tw(mr / 2);
    std::vector<float2> stw(2 * nb);
    for (int k = 0; k < mr / 2; ++k) {
        const double a = two_pi * k / mr;
        const float2 c = df_from_double(std::cos(a)), sn = df_from_double(-std::sin(a));
        tw[k] = make_float4(c.x, c.y, sn.x, sn.y);
    }
    for (int q = 0; q < 2 * nb; ++q) {
        const double a = kPi * q / nb;
        stw[q] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    CT_CHECK(upload(&F->sE, sE));
    CT_CHECK(upload(&F->base, base));
    CT_CHECK(upload(&F->wgt, wgt));
    CT_CHECK(upload(&F->phase, phase));
    CT_CHECK(upload(&F->cell_start, count));
    CT_CHECK(upload(&F->cell_idx, cell_idx));
    CT_CHECK(upload(&F->tw, tw));
    CT_CHECK(upload(&F->sino_tw, stw));
    CT_CHECK(alloc_bytes((void**)&F->X, sizeof(float4) * (size_t)mr * mr));
    CT_CHECK(alloc_bytes((void**)&F->Y, sizeof(float4) * (size_t)mr * mr));
    CT_CHECK(alloc_bytes((void**)&F->S, sizeof(float4) * (size_t)J));

    F->fft_T = 2;
    // the shared-memory limits are per kernel, not per handle: raise them to
    // the largest any handle uses (N <= 2048, m_sp <= 12)
    CT_CUDA(cudaFuncSetAttribute(fft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemMax));
    CT_CUDA(cudaFuncSetAttribute(fft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemMax));
    CT_CUDA(cudaFuncSetAttribute(dia_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDiaSmemMax));
    CT_CUDA(cudaFuncSetAttribute(build_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBuildSmemMax));
    if (fft_smem(*F) > (size_t)kFftSmemMax || dia_smem(*F) > (size_t)kDiaSmemMax)
        return fail(CT_ERR_CUDA, "internal: Fourier kernel shared memory above its limit");
    if (F->mode == CT_FOURIER_FUSED) {
        const size_t planes = (size_t)F->nd * F->nd;
        CT_CHECK(alloc_bytes((void**)&F->C, sizeof(float) * planes * mr * mr));
        int G = 32;
        while (G > 1 && (size_t)G * planes * sizeof(float2) > (size_t)kBuildSmemMax) G /= 2;
        const size_t sm = (size_t)G * planes * sizeof(float2);
        const int64_t blocks = (int64_t)mr * mr / G;
        build_fused_kernel<<<(unsigned)blocks, 256, sm>>>(F->C, mr, msp, G, F->cell_start, F->cell_idx, F->wgt);
        CT_CUDA(cudaGetLastError());
        sym_fused_kernel<<<grid_blocks(M, (int64_t)mr * mr * ((F->nd * F->nd - 1) / 2)), 256>>>(F->C, mr, msp);
        CT_CUDA(cudaGetLastError());
        const int tiles = mr / kDiaTile;
        CT_CHECK(alloc_bytes((void**)&F->tile_nz, (size_t)tiles * tiles));
        tile_nonzero_kernel<<<tiles * tiles, kDiaTile * kDiaTile>>>(F->C, mr, F->nd * F->nd, F->tile_nz);
        CT_CUDA(cudaGetLastError());
    }
    CT_CUDA(cudaDeviceSynchronize());
    return CT_OK;
}

int launch_fourier_op_df(const ct_matrix* M, const OpEpilogue& ep, cudaStream_t st)
{
    const FourierOp& F = *M->fourier;
    const Gate g{ep.gate, ep.cg, ep.mode != 2};
    const int64_t len = (int64_t)F.mr * F.mr;
    pad_kernel<true><<<grid_blocks(M, len), 256, 0, st>>>(ep.in, F.X, F.n, M->tn, F.mr, F.sE, g);
    CT_CUDA(cudaGetLastError());
    CT_CHECK(fft2(F, F.X, false, g, st));
    CT_CHECK(grid_normal(M, F, g, st));
    CT_CHECK(fft2(F, F.Y, true, g, st));
    const int grid = grid_for(M, M->npad, 256, 8);
    switch (ep.mode) {
    case 1: crop_op_kernel<1><<<grid, 256, 0, st>>>(ep, F.Y, F.n, M->tn, M->npad, F.mr, F.sE); break;
    case 2: crop_op_kernel<2><<<grid, 256, 0, st>>>(ep, F.Y, F.n, M->tn, M->npad, F.mr, F.sE); break;
    default: crop_op_kernel<3><<<grid, 256, 0, st>>>(ep, F.Y, F.n, M->tn, M->npad, F.mr, F.sE); break;
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int fourier_backproject_df(const ct_matrix* M, const float* f, float2* out, double scale, cudaStream_t st)
{
    const FourierOp& F = *M->fourier;
    sino_dft_kernel<false><<<F.n_kept, 256, F.n_bins * sizeof(float), st>>>(f, F.S, F.n_bins, F.sino_tw,
                                                                     (float)(1.0 / std::sqrt((double)F.n_bins)),
                                                                     F.phase);
    CT_CUDA(cudaGetLastError());
    CT_CHECK(spread_inverse(M, F, st));
    crop_kernel<true><<<grid_for(M, M->npad, 256, 8), 256, 0, st>>>(F.Y, out, F.n, M->tn, F.mr, F.sE,
                                                                    df_from_double(scale));
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

void fourier_point_response(const ct_matrix* M, int r, std::vector<double>& h)
{
    const FourierOp& F = *M->fourier;
    const int w = 2 * r + 1;
    h.assign((size_t)w * w, 0.0);
    for (int di = -r; di <= r; ++di) {
        for (int dj = -r; dj <= r; ++dj) {
            double s = 0.0;
            for (int64_t j = 0; j < F.J; ++j) s += std::cos(F.h_wx[j] * dj + F.h_wy[j] * di);
            h[(size_t)(di + r) * w + (dj + r)] = s / F.n_bins;
        }
    }
}

int fourier_forward(const ct_matrix* M, const float* x, float* y, cudaStream_t st)
{
    const FourierOp& F = *M->fourier;
    const Gate none{nullptr, nullptr, 0};
    const int64_t len = (int64_t)F.mr * F.mr;
    pad_kernel<false><<<grid_blocks(M, len), 256, 0, st>>>(x, F.X, F.n, M->tn, F.mr, F.sE, none);
    CT_CUDA(cudaGetLastError());
    CT_CHECK(fft2(F, F.X, false, none, st));
    interp_kernel<true><<<grid_blocks(M, F.J), 256, 0, st>>>(F.X, y, F.J, F.mr, F.msp, F.base,
                                                       F.wgt, F.phase, none);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int fourier_adjoint(const ct_matrix* M, const float* y, float* x, cudaStream_t st)
{
    const FourierOp& F = *M->fourier;
    conj_phase_kernel<<<grid_blocks(M, F.J), 256, 0, st>>>(reinterpret_cast<const float2*>(y), F.S, F.phase, F.J);
    CT_CUDA(cudaGetLastError());
    CT_CHECK(spread_inverse(M, F, st));
    crop_kernel<false><<<grid_blocks(M, M->cols), 256, 0, st>>>(F.Y, x, F.n, M->tn, F.mr, F.sE, df_from_double(1.0));
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int fourier_normal(const ct_matrix* M, const float* x, float* out, cudaStream_t st)
{
    const FourierOp& F = *M->fourier;
    const Gate none{nullptr, nullptr, 0};
    const int64_t len = (int64_t)F.mr * F.mr;
    pad_kernel<false><<<grid_blocks(M, len), 256, 0, st>>>(x, F.X, F.n, M->tn, F.mr, F.sE, none);
    CT_CUDA(cudaGetLastError());
    CT_CHECK(fft2(F, F.X, false, none, st));
    CT_CHECK(grid_normal(M, F, none, st));
    CT_CHECK(fft2(F, F.Y, true, none, st));
    crop_kernel<false><<<grid_blocks(M, M->cols), 256, 0, st>>>(F.Y, out, F.n, M->tn, F.mr, F.sE, df_from_double(1.0));
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

int fourier_data(const ct_matrix* M, const float* f, float* fhat, cudaStream_t st)
{
    const FourierOp& F = *M->fourier;
    sino_dft_kernel<true><<<F.n_kept, 256, F.n_bins * sizeof(float), st>>>(
        f, fhat, F.n_bins, F.sino_tw, (float)(1.0 / std::sqrt((double)F.n_bins)),
        nullptr);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ct
