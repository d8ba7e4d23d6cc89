// Builder of the sparse system matrices A = M R and A^T (Sec. 3: the matrices
// depend only on the geometry and are precomputed once, offline), and of the
// surrogate stencil of Sec. 3.2.
//
// Every entry is the exact length of a ray inside a pixel.  Instead of walking
// the ray (Siddon), each candidate (ray, pixel) pair is evaluated with the
// closed-form chord of a unit square: for a line with unit normal (c, s) at
// distance t from the pixel centre, with a = max(|c|,|s|), b = min(|c|,|s|),
//     L(t) = 1/a                       for t <= (a-b)/2
//          = ((a+b)/2 - t) / (a b)     for (a-b)/2 < t < (a+b)/2
//          = 0                         otherwise,
// and for b = 0 (axis-aligned ray) L = 1 inside, 1/2 on an edge (the edge
// reading: half the length to each of the two pixels sharing the edge).
// A is built ray by ray (rows = rays, columns ascending), A^T pixel by pixel
// (rows = pixels, ray index ascending), so neither needs a transpose or
// atomics; both evaluate the same function with the same operation order, so
// A^T holds bit-identical values.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ct_internal.cuh"

namespace ct {
namespace {

constexpr double kMinLen = 1e-12;  // lengths below this are dropped
constexpr double kPi = 3.14159265358979323846;

// Per kept angle: cos, sin, a = max(|cos|,|sin|), b = min(...), t2 = support half-width.
struct AngleRow {
    double c, s, a, b, t2;
};

__device__ __forceinline__ double ray_offset(double xc, double yc, double c, double s, double sb)
{
    // explicit round-to-nearest operations: no FMA contraction, so that the A
    // and A^T builders produce identical bits for the same (ray, pixel) pair
    return fabs(__dadd_rn(__dadd_rn(__dmul_rn(xc, c), __dmul_rn(yc, s)), -sb));
}

__device__ __forceinline__ double chord(double t, const AngleRow& g)
{
    if (g.b == 0.0) return t < 0.5 ? 1.0 : (t == 0.5 ? 0.5 : 0.0);
    const double t1 = __dmul_rn(0.5, __dsub_rn(g.a, g.b));
    if (t <= t1) return __ddiv_rn(1.0, g.a);
    if (t >= g.t2) return 0.0;
    return __ddiv_rn(__dsub_rn(g.t2, t), __dmul_rn(g.a, g.b));
}

// IEEE-754 binary16 from a double, round to nearest, ties to even, written
// from the format's definition (1 sign, 5 exponent bits with bias 15, 10
// fraction bits; subnormals are multiples of 2^-24).
__host__ __device__ inline uint16_t f64_to_f16_bits(double x)
{
    uint16_t sign = std::signbit(x) ? 0x8000u : 0u;
    double a = std::fabs(x);
    if (a != a) return sign | 0x7e00u;
    if (a < 6.103515625e-05) {  // below 2^-14: subnormal (or zero)
        double m = std::rint(a * 16777216.0);  // a / 2^-24, rounded to nearest even
        return sign | (uint16_t)m;             // m == 1024 is the smallest normal
    }
    int e;
    std::frexp(a, &e);  // a = f 2^e, f in [0.5, 1)
    int E = e - 1;      // a = 1.xxx 2^E
    if (E > 15) return sign | 0x7c00u;
    double m = std::rint(std::ldexp(a, 10 - E));  // in [1024, 2048]
    unsigned mi = (unsigned)m;
    if (mi == 2048u) {
        mi = 1024u;
        ++E;
        if (E > 15) return sign | 0x7c00u;
    }
    return sign | (uint16_t)(((E + 15) << 10) | (mi - 1024u));
}

__device__ __forceinline__ __half f16_from_bits(uint16_t b)
{
    __half_raw r;
    r.x = b;
    return __half(r);
}

// Position of entry j of a row whose entry 0 sits at `base` (SELL layout).
__device__ __forceinline__ int64_t entry_pos(int64_t base, int64_t j) { return base + ((j >> 3) << 8) + (j & 7); }

// One thread per ray q = k*n_bins + b: sweep the image rows, evaluate the
// pixels of each row the line can reach, keep lengths >= kMinLen.
template <bool FILL>
__global__ void a_rows_kernel(int n, int tn, int nb, int n_kept, const AngleRow* __restrict__ ang,
                              int32_t* __restrict__ row_len, float* __restrict__ row_max,
                              const int64_t* __restrict__ slice_ptr, int32_t* __restrict__ col,
                              float* __restrict__ val, __half* __restrict__ qval,
                              const float* __restrict__ scale)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n_kept * nb) return;
    const int k = (int)(q / nb), b = (int)(q % nb);
    const AngleRow g = ang[k];
    const double sb = b - 0.5 * (nb - 1);
    const double half = 0.5 * n;
    int cnt = 0;
    double mx = 0.0;
    int64_t base = 0;
    double sq = 1.0;
    if (FILL) {
        base = slice_ptr[q >> 5] + ((q & 31) << 3);
        if (qval) sq = (double)scale[q];
    }
    int32_t last = 0;
    for (int i = 0; i < n; ++i) {
        const double yc = i - half + 0.5;
        int jlo, jhi;
        if (g.c == 0.0) {
            if (fabs(yc * g.s - sb) > g.t2 + 1e-9) continue;
            jlo = 0;
            jhi = n - 1;
        } else {
            const double jc = (sb - yc * g.s) / g.c + half - 0.5;
            const double w = g.t2 / fabs(g.c);
            const double lo = fmax(floor(jc - w) - 1.0, 0.0);
            const double hi = fmin(ceil(jc + w) + 1.0, n - 1.0);
            if (lo > hi) continue;
            jlo = (int)lo;
            jhi = (int)hi;
        }
        for (int j = jlo; j <= jhi; ++j) {
            const double xc = j - half + 0.5;
            const double len = chord(ray_offset(xc, yc, g.c, g.s, sb), g);
            if (len < kMinLen) continue;
            last = (int32_t)tiled_index(i, j, tn);
            if (FILL) {
                const int64_t e = entry_pos(base, cnt);
                col[e] = last;
                if (val) val[e] = (float)len;
                if (qval) qval[e] = f16_from_bits(f64_to_f16_bits(len / sq));
            } else {
                mx = fmax(mx, len);
            }
            ++cnt;
        }
    }
    if (!FILL) {
        row_len[q] = cnt;
        if (row_max) row_max[q] = (float)mx;
    } else {
        // the rest of the row's last chunk repeats the last column with value 0
        for (int j = cnt; j % kChunk != 0; ++j) {
            const int64_t e = entry_pos(base, j);
            col[e] = last;
            if (val) val[e] = 0.0f;
            if (qval) qval[e] = __float2half(0.0f);
        }
    }
}

// One thread per internal pixel index t (tile order): for every kept angle,
// evaluate the bins whose rays can cross the pixel; entries come out by angle,
// then bin, with the column written as the band-local index
// off_k + (b - band_lo(tile, k)).  Padding pixels get empty rows.
template <bool FILL>
__global__ void at_rows_kernel(int n, int tn, int nb, int n_kept, const AngleRow* __restrict__ ang,
                               const int32_t* __restrict__ band_lo, const int32_t* __restrict__ band_off,
                               int64_t npad,
                               int32_t* __restrict__ row_len, const int64_t* __restrict__ slice_ptr,
                               uint16_t* __restrict__ col16, float* __restrict__ val,
                               __half* __restrict__ qval, const float* __restrict__ scale,
                               int32_t* __restrict__ bad)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= npad) return;
    int i, j;
    tiled_coords(t, tn, i, j);
    if (i >= n || j >= n) {
        if (!FILL) row_len[t] = 0;
        return;
    }
    const int32_t* blo = band_lo + (t >> 8) * (int64_t)n_kept;
    const double half = 0.5 * n;
    const double xc = j - half + 0.5, yc = i - half + 0.5;
    const double mid = 0.5 * (nb - 1);
    int cnt = 0;
    const int64_t base = FILL ? slice_ptr[t >> 5] + ((t & 31) << 3) : 0;
    uint16_t last = 0;
    for (int k = 0; k < n_kept; ++k) {
        const AngleRow g = ang[k];
        const double tc = xc * g.c + yc * g.s + mid;
        const double lo = fmax(floor(tc - g.t2) - 1.0, 0.0);
        const double hi = fmin(ceil(tc + g.t2) + 1.0, nb - 1.0);
        for (int b = (int)lo; b <= (int)hi; ++b) {
            const double sb = b - mid;
            const double len = chord(ray_offset(xc, yc, g.c, g.s, sb), g);
            if (len < kMinLen) continue;
            const int w = b - blo[k];
            if (w < 0 || w >= band_off[k + 1] - band_off[k]) {
                atomicExch(bad, 1);
                continue;
            }
            last = (uint16_t)(band_off[k] + w);
            if (FILL) {
                const int64_t e = entry_pos(base, cnt);
                col16[e] = last;
                if (val) val[e] = (float)len;
                if (qval) qval[e] = f16_from_bits(f64_to_f16_bits(len / (double)scale[(int64_t)k * nb + b]));
            }
            ++cnt;
        }
    }
    if (!FILL) {
        row_len[t] = cnt;
    } else {
        for (int j = cnt; j % kChunk != 0; ++j) {
            const int64_t e = entry_pos(base, j);
            col16[e] = last;
            if (val) val[e] = 0.0f;
            if (qval) qval[e] = __float2half(0.0f);
        }
    }
}

// h(d) = sum_q A[q, c] A[q, c + d] for every offset d of the square window
// [-r, r]^2 around c = (N/2, N/2), in FP64.  One block per offset; the sum
// runs in a fixed order (per-thread angle strides, then a tree).
__global__ void point_response_kernel(int n, int nb, int n_kept, const AngleRow* __restrict__ ang,
                                      int r, double* __restrict__ h)
{
    const int w = 2 * r + 1;
    const int di = (int)blockIdx.x / w - r, dj = (int)blockIdx.x % w - r;
    const int ci = n / 2, cj = n / 2;
    const int ti = ci + di, tj = cj + dj;
    const double half = 0.5 * n, mid = 0.5 * (nb - 1);
    const double xc = cj - half + 0.5, yc = ci - half + 0.5;
    const double xt = tj - half + 0.5, yt = ti - half + 0.5;
    const bool inside = ti >= 0 && ti < n && tj >= 0 && tj < n;
    double acc = 0.0;
    if (inside) {
        for (int k = threadIdx.x; k < n_kept; k += blockDim.x) {
            const AngleRow g = ang[k];
            const double tc = xc * g.c + yc * g.s + mid;
            const double lo = fmax(floor(tc - g.t2) - 1.0, 0.0);
            const double hi = fmin(ceil(tc + g.t2) + 1.0, nb - 1.0);
            for (int b = (int)lo; b <= (int)hi; ++b) {
                const double sb = b - mid;
                const double l1 = chord(ray_offset(xc, yc, g.c, g.s, sb), g);
                if (l1 < kMinLen) continue;
                const double l2 = chord(ray_offset(xt, yt, g.c, g.s, sb), g);
                if (l2 < kMinLen) continue;
                acc += l1 * l2;
            }
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) h[blockIdx.x] = red[0];
}

int alloc_dev(void** p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return fail(CT_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    CT_CUDA(e);
    return CT_OK;
}

// Slice offsets of the SELL layout from the row lengths (host).
int finish_layout(Sell& m, const std::vector<int32_t>& len)
{
    const int64_t nslices = ((int64_t)len.size() + kSliceRows - 1) / kSliceRows;
    std::vector<int64_t> sp(nslices + 1, 0);
    int64_t nnz = 0;
    for (int64_t s = 0; s < nslices; ++s) {
        int64_t longest = 0;
        for (int64_t r = s * kSliceRows; r < (s + 1) * kSliceRows && r < (int64_t)len.size(); ++r) {
            nnz += len[r];
            longest = len[r] > longest ? len[r] : longest;
        }
        sp[s + 1] = sp[s] + (longest + kChunk - 1) / kChunk * kChunk * kSliceRows;
    }
    m.nnz = nnz;
    m.nnz_pad = sp.back();
    CT_CHECK(alloc_dev((void**)&m.slice_ptr, sp.size() * sizeof(int64_t)));
    CT_CUDA(cudaMemcpy(m.slice_ptr, sp.data(), sp.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    return CT_OK;
}

// First bin of every (tile, angle) band.  The tile's square projects onto
// [t_min, t_min + L_k], L_k = 16 (|cos| + |sin|), t over the square's corners;
// a ray at s_b can give the tile a nonzero length only for s_b in that closed
// interval (on its ends only along an edge, by the edge reading).  The band
// starts at ceil(t_min + mid - 1e-6) and has floor(L_k + 2e-6) + 2 bins,
// which covers the interval with a margin of 1e-6 at either end.
std::vector<int32_t> band_table(const ct_geometry& g, const std::vector<double>& hc,
                                const std::vector<double>& hs, int tn)
{
    const int nk = (int)hc.size();
    const double half = 0.5 * g.n, mid = 0.5 * (g.n_bins - 1);
    std::vector<int32_t> lo((size_t)tn * tn * nk);
    for (int ti = 0; ti < tn; ++ti) {
        for (int tj = 0; tj < tn; ++tj) {
            const double x0 = tj * kTile - half, y0 = ti * kTile - half;
            for (int k = 0; k < nk; ++k) {
                double tmin = 1e300;
                for (int cx = 0; cx < 2; ++cx)
                    for (int cy = 0; cy < 2; ++cy)
                        tmin = std::fmin(tmin, (x0 + cx * kTile) * hc[k] + (y0 + cy * kTile) * hs[k]);
                const double b = std::ceil(tmin + mid - 1e-6);
                lo[((size_t)ti * tn + tj) * nk + k] = (int32_t)std::fmax(b, 0.0);
            }
        }
    }
    return lo;
}

// Offsets of the angles' slots within a band: off[k+1] - off[k] = W_k.
std::vector<int32_t> band_offsets(const std::vector<double>& hc, const std::vector<double>& hs)
{
    std::vector<int32_t> off(hc.size() + 1, 0);
    for (size_t k = 0; k < hc.size(); ++k) {
        const double len = kTile * (std::fabs(hc[k]) + std::fabs(hs[k]));
        off[k + 1] = off[k] + (int32_t)std::floor(len + 2e-6) + 2;
    }
    return off;
}

std::vector<AngleRow> angle_table(const ct_geometry& g, std::vector<double>& hc, std::vector<double>& hs)
{
    const int n_kept = (g.n_angles_total + g.keep_every - 1) / g.keep_every;
    std::vector<AngleRow> t(n_kept);
    hc.resize(n_kept);
    hs.resize(n_kept);
    for (int kk = 0; kk < n_kept; ++kk) {
        const int k = kk * g.keep_every;
        double c, s;
        if (k == 0) {
            c = 1.0;
            s = 0.0;
        } else if (2 * k == g.n_angles_total) {
            c = 0.0;
            s = 1.0;
        } else {
            const double th = (double)k * kPi / (double)g.n_angles_total;
            c = std::cos(th);
            s = std::sin(th);
        }
        const double a = std::fmax(std::fabs(c), std::fabs(s));
        const double b = std::fmin(std::fabs(c), std::fabs(s));
        t[kk] = AngleRow{c, s, a, b, b == 0.0 ? 0.5 : 0.5 * (a + b)};
        hc[kk] = c;
        hs[kk] = s;
    }
    return t;
}

}  // namespace

void angle_directions(const ct_geometry& g, std::vector<double>& c, std::vector<double>& s)
{
    (void)angle_table(g, c, s);
}

void free_sell(Sell& c)
{
    cudaFree(c.slice_ptr);
    cudaFree(c.row_len);
    cudaFree(c.col);
    cudaFree(c.col16);
    cudaFree(c.val);
    cudaFree(c.qval);
    c = Sell{};
}

int build_matrices(ct_matrix* M)
{
    const ct_geometry& g = M->g;
    std::vector<AngleRow> tab = angle_table(g, M->h_cos, M->h_sin);
    M->n_kept = (int)tab.size();
    const int n = g.n, nb = g.n_bins, nk = M->n_kept;
    M->rows = (int64_t)nk * nb;
    M->cols = (int64_t)n * n;
    const bool f16 = (M->flags & CT_VAL_FP16_ROWSCALE) != 0;
    const bool f32 = !f16 || (M->flags & CT_KEEP_FP32_COPY);

    AngleRow* d_ang = nullptr;
    CT_CHECK(alloc_dev((void**)&d_ang, tab.size() * sizeof(AngleRow)));
    CT_CUDA(cudaMemcpy(d_ang, tab.data(), tab.size() * sizeof(AngleRow), cudaMemcpyHostToDevice));
    M->dirs = (double*)d_ang;

    M->tn = tiles_per_side(n);
    M->npad = padded_pixels(n);
    const int tn = M->tn;
    M->h_band_off = band_offsets(M->h_cos, M->h_sin);
    M->band_total = M->h_band_off.back();
    for (int k = 0; k < nk; ++k)
        if (M->h_band_off[k + 1] - M->h_band_off[k] > kBandMax)
            return fail(CT_ERR_CUDA, "internal: band wider than kBandMax");
    if (M->band_total > 65536)
        return fail(CT_ERR_UNSUPPORTED, "too many kept angles for 16-bit band indices (" +
                                             std::to_string(M->band_total) + " band slots > 65536)");
    // Angle chunks of the band: the adjoint stages one chunk of a tile's band
    // at a time in shared memory, so chunks stay within kBandChunkSlots slots
    // (at 180 angles the whole band is one chunk).
    M->h_band_chunk.assign(1, 0);
    for (int k = 0; k < nk; ++k) {
        const int start = M->h_band_chunk.back();
        if (M->h_band_off[k + 1] - M->h_band_off[start] > kBandChunkSlots) M->h_band_chunk.push_back(k);
    }
    M->h_band_chunk.push_back(nk);
    M->band_chunk_slots = 0;
    for (size_t j = 0; j + 1 < M->h_band_chunk.size(); ++j)
        M->band_chunk_slots = std::max(M->band_chunk_slots,
                                       M->h_band_off[M->h_band_chunk[j + 1]] - M->h_band_off[M->h_band_chunk[j]]);
    CT_CHECK(alloc_dev((void**)&M->band_chunk, M->h_band_chunk.size() * sizeof(int32_t)));
    CT_CUDA(cudaMemcpy(M->band_chunk, M->h_band_chunk.data(), M->h_band_chunk.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice));
    M->h_band_angle.resize(M->band_total);
    for (int k = 0; k < nk; ++k)
        for (int c = M->h_band_off[k]; c < M->h_band_off[k + 1]; ++c) M->h_band_angle[c] = (uint16_t)k;
    M->h_band_lo = band_table(g, M->h_cos, M->h_sin, tn);
    CT_CHECK(alloc_dev((void**)&M->band_lo, M->h_band_lo.size() * sizeof(int32_t)));
    CT_CUDA(cudaMemcpy(M->band_lo, M->h_band_lo.data(), M->h_band_lo.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice));
    CT_CHECK(alloc_dev((void**)&M->band_off, M->h_band_off.size() * sizeof(int32_t)));
    CT_CUDA(cudaMemcpy(M->band_off, M->h_band_off.data(), M->h_band_off.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice));
    CT_CHECK(alloc_dev((void**)&M->band_angle, M->h_band_angle.size() * sizeof(uint16_t)));
    CT_CUDA(cudaMemcpy(M->band_angle, M->h_band_angle.data(), M->h_band_angle.size() * sizeof(uint16_t),
                       cudaMemcpyHostToDevice));
    int32_t* d_bad = nullptr;
    CT_CHECK(alloc_dev((void**)&d_bad, sizeof(int32_t)));
    CT_CUDA(cudaMemset(d_bad, 0, sizeof(int32_t)));

    Sell& A = M->A;
    Sell& T = M->At;
    A.rows = M->rows;
    A.cols = M->npad;
    T.rows = M->npad;
    T.cols = M->band_total;
    CT_CHECK(alloc_dev((void**)&A.row_len, A.rows * sizeof(int32_t)));
    CT_CHECK(alloc_dev((void**)&T.row_len, T.rows * sizeof(int32_t)));
    if (f16) CT_CHECK(alloc_dev((void**)&M->row_scale, A.rows * sizeof(float)));

    const int tpb = 128;
    // pass 1: counts (and row maxima for the FP16 scale)
    a_rows_kernel<false><<<(unsigned)((A.rows + tpb - 1) / tpb), tpb>>>(
        n, tn, nb, nk, d_ang, A.row_len, f16 ? M->row_scale : nullptr, nullptr, nullptr, nullptr,
        nullptr, nullptr);
    CT_CUDA(cudaGetLastError());
    at_rows_kernel<false><<<(unsigned)((T.rows + tpb - 1) / tpb), tpb>>>(
        n, tn, nb, nk, d_ang, M->band_lo, M->band_off, M->npad, T.row_len, nullptr, nullptr, nullptr, nullptr, nullptr, d_bad);
    CT_CUDA(cudaGetLastError());
    std::vector<int32_t> la(A.rows), lt(T.rows);
    CT_CUDA(cudaMemcpy(la.data(), A.row_len, A.rows * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(lt.data(), T.row_len, T.rows * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CT_CHECK(finish_layout(A, la));
    CT_CHECK(finish_layout(T, lt));
    if (A.nnz != T.nnz)
        return fail(CT_ERR_CUDA, "internal: A and A^T entry counts differ (" + std::to_string(A.nnz) +
                                     " vs " + std::to_string(T.nnz) + ")");
    CT_CHECK(alloc_dev((void**)&A.col, A.nnz_pad * sizeof(int32_t)));
    CT_CHECK(alloc_dev((void**)&T.col16, T.nnz_pad * sizeof(uint16_t)));
    CT_CUDA(cudaMemset(A.col, 0, A.nnz_pad * sizeof(int32_t)));
    CT_CUDA(cudaMemset(T.col16, 0, T.nnz_pad * sizeof(uint16_t)));
    for (Sell* m : {&A, &T}) {
        if (f32) {
            CT_CHECK(alloc_dev((void**)&m->val, m->nnz_pad * sizeof(float)));
            CT_CUDA(cudaMemset(m->val, 0, m->nnz_pad * sizeof(float)));
        }
        if (f16) {
            CT_CHECK(alloc_dev((void**)&m->qval, m->nnz_pad * sizeof(__half)));
            CT_CUDA(cudaMemset(m->qval, 0, m->nnz_pad * sizeof(__half)));
        }
    }
    // pass 2: fill
    a_rows_kernel<true><<<(unsigned)((A.rows + tpb - 1) / tpb), tpb>>>(
        n, tn, nb, nk, d_ang, nullptr, nullptr, A.slice_ptr, A.col, A.val, A.qval, M->row_scale);
    CT_CUDA(cudaGetLastError());
    at_rows_kernel<true><<<(unsigned)((T.rows + tpb - 1) / tpb), tpb>>>(
        n, tn, nb, nk, d_ang, M->band_lo, M->band_off, M->npad, nullptr, T.slice_ptr, T.col16, T.val, T.qval, M->row_scale, d_bad);
    CT_CUDA(cudaGetLastError());
    int32_t bad = 0;
    CT_CUDA(cudaMemcpy(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost));
    cudaFree(d_bad);
    if (bad) return fail(CT_ERR_CUDA, "internal: an A^T entry fell outside its tile band");
    return CT_OK;
}

int make_stencil(ct_matrix* M, int r, int square, Stencil** out)
{
    auto key = std::make_pair(r, square ? 1 : 0);
    auto it = M->stencils.find(key);
    if (it != M->stencils.end()) {
        *out = &it->second;
        return CT_OK;
    }
    if (r <= 0 || r > 16) return fail(CT_ERR_ARG, "surrogate radius must be in [1, 16]");
    const int w = 2 * r + 1;
    std::vector<double> h((size_t)w * w);
    if (M->fourier) {
        fourier_point_response(M, r, h);
    } else {
        double* d_h = nullptr;
        CT_CHECK(alloc_dev((void**)&d_h, (size_t)w * w * sizeof(double)));
        point_response_kernel<<<w * w, 256>>>(M->g.n, M->g.n_bins, M->n_kept, (const AngleRow*)M->dirs, r, d_h);
        CT_CUDA(cudaGetLastError());
        cudaError_t e = cudaMemcpy(h.data(), d_h, h.size() * sizeof(double), cudaMemcpyDeviceToHost);
        cudaFree(d_h);
        CT_CUDA(e);
    }
    Stencil S;
    S.r = r;
    std::vector<float> wf;
    std::vector<int32_t> dd;
    for (int di = -r; di <= r; ++di) {
        for (int dj = -r; dj <= r; ++dj) {
            if (!square && di * di + dj * dj > r * r) continue;
            const double v = 0.5 * (h[(size_t)(di + r) * w + (dj + r)] + h[(size_t)(-di + r) * w + (-dj + r)]);
            S.h_di.push_back(di);
            S.h_dj.push_back(dj);
            S.h_w.push_back(v);
            const float hi = (float)v;
            wf.push_back(hi);
            wf.push_back((float)(v - (double)hi));
            dd.push_back(di);
            dd.push_back(dj);
        }
    }
    S.ntaps = (int)S.h_w.size();
    CT_CHECK(alloc_dev((void**)&S.d, dd.size() * sizeof(int32_t)));
    CT_CHECK(alloc_dev((void**)&S.w, wf.size() * sizeof(float)));
    CT_CUDA(cudaMemcpy(S.d, dd.data(), dd.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CT_CUDA(cudaMemcpy(S.w, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice));
    auto res = M->stencils.emplace(key, std::move(S));
    *out = &res.first->second;
    return CT_OK;
}

void free_stencil(Stencil& s)
{
    cudaFree(s.d);
    cudaFree(s.w);
    s.d = nullptr;
    s.w = nullptr;
}

}  // namespace ct
