// Persistent ragged batch: one Bregman update of every problem of a
// ct_split_bregman_ragged call (single-slice runs of possibly different
// geometries) in a single cooperative kernel launch.
//
// The update of one problem is a fixed chain of phases (Sec. 4's update with
// inexact CG, Eq. SB_solve): the residual r = rhs - Op(u) (a forward product
// and the fused A^T kernel), then per CG step y = A p, q = Op(p) with p.q,
// u += alpha p / r -= alpha q with r.r, p = r + beta p, and at the end the
// shrink / Bregman step with ||u - u_old||_1.  Each phase is split into work
// items (a few 32-ray slices, one 16 x 16 image tile, or a run of pixels).
// The host lays every problem's phases out in one queue, step by step across
// the problems, so that small problems run beside large ones.  The kernel's
// CTAs (all resident: a cooperative launch sized by occupancy) take items in
// queue order from one ticket counter.  An item first waits until the
// previous phase of its problem is complete; the last item of a phase to
// finish sums the phase's per-item partial sums in a fixed order, updates
// the problem's CG or Bregman scalars and marks the phase complete.  Items
// only ever wait on items earlier in the queue, which are held by running
// CTAs, so the waits end.  Every wait is bounded: after `limit` polls the
// CTA records CT_ERR_TIMEOUT with the phase it waited for, raises an abort
// flag that every CTA checks before taking an item and while waiting, and
// returns; the host reads the status after the launch.
//
// The launch is captured into a CUDA graph (counters cleared by a memset
// node, then the kernel) and replayed once per Bregman update.  Data written
// within the launch (p, u, r, q, y) is read through L2 (ld.global.cg or
// plain loads after an acquire), never through the non-coherent path.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

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

constexpr int kRgThreads = 256;
constexpr int kRgMinBlocks = 4;        // CTAs per SM the registers are sized for
constexpr int kRgFwdSlices = 4;        // 32-ray slices per forward item
constexpr int kRgVecPixels = 8192;     // pixels per vector item
constexpr int kRgUnroll = 8;           // chunks in flight per lane in the forward items

enum RgKind : int32_t {
    RG_FWD_U = 0,   // y = A u (start of the inner solve)
    RG_OP_RES = 1,  // r = rhs - Op(u), p = r; r.r, rhs.rhs
    RG_FWD_P = 2,   // y = A p
    RG_OP_Q = 3,    // q = Op(p); p.q
    RG_UPD = 4,     // u += alpha p, r -= alpha q; r.r
    RG_DIR = 5,     // p = r + beta p
    RG_SHRINK = 6   // d, b, v; ||u - u_old||_1
};

// One problem as the kernel sees it.
struct RgProb {
    SellView A;
    const int32_t* Acol;
    const void* Aval;      // float or __half
    const float* row_scale;
    BandView bv;
    const void* Atval;     // float or __half
    int f16, chunked;
    int n, tn;
    int64_t npad;
    OpEpilogue ep_res;     // the plan's epilogue for r = rhs - Op(u), p = r (mode 2)
    OpEpilogue ep_q;       // ... and for q = Op(p) (mode 1)
    float2 *u, *r, *p, *q, *y, *u_old, *bx, *by, *vx, *vy;
    CgSlice* cg;
    SbSlice* sb;
    float2* partials;
    float2 gamma;
    double stop_tol;
};

struct RgPhase {
    int32_t prob, kind, first, count, dep;  // dep: index of the phase to wait for, or -1
};

// Control words of one call.  ticket, arrive[] and done[] are cleared before
// every launch; status, where and abort persist over the call's launches.
struct RgCtl {
    int ticket;
    int status;
    int where;
    int abort;
    int never;  // a flag nothing sets (the held-dependency test)
};

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_cg_int(const int* p) { return __ldcg(p); }

// Sum of NQ per-thread double-float values over the block in a fixed order;
// the result is valid in thread 0.
template <int NQ>
__device__ __forceinline__ void block_sum(float2 (&v)[NQ], float2 (*sh)[32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const float2 s = warp_sum_df(v[k]);
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            float2 s = sh[k][0];
            for (int w = 1; w < nwarp; ++w) s = df_add(s, sh[k][w]);
            v[k] = s;
        }
    }
    __syncthreads();
}

// Grid totals of a phase's NQ partial sums (partials[k * count + item]), in a
// fixed order, by the whole block; valid in thread 0.
template <int NQ>
__device__ __forceinline__ void phase_totals(const float2* partials, int count, double (&tot)[NQ],
                                             float2 (*sh)[32])
{
    float2 v[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        float2 s = df_zero();
        for (int b = threadIdx.x; b < count; b += blockDim.x) s = df_add(s, __ldcg(partials + (size_t)k * count + b));
        v[k] = s;
    }
    block_sum<NQ>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) tot[k] = df_to_double(v[k]);
    }
}

// ---------------------------------------------------------------------------
// work items
// ---------------------------------------------------------------------------
// y = A x over kRgFwdSlices slices of 32 rays.
template <typename VT>
__device__ __forceinline__ void rg_fwd_item(const RgProb& P, const float2* x, int item)
{
    const int64_t nslices = (P.A.rows + kSliceRows - 1) / kSliceRows;
    const ProdArgs a{P.f16 ? P.row_scale : nullptr, P.f16 ? 2 : 0, make_float2(1.0f, 0.0f), nullptr, nullptr};
    for (int k = 0; k < kRgFwdSlices; ++k) {
        const int64_t s = (int64_t)item * kRgFwdSlices + k;
        if (s >= nslices) break;
        fwd_slice<VT, float2, float2, kRgUnroll, true>(P.A, P.Acol, static_cast<const VT*>(P.Aval), x, P.y, a, s);
    }
}

// A^T y over one image tile fused with the CG operator epilogue; the tile's
// two dot-product partials go to partials[tile] and partials[tiles + tile].
template <typename VT, int MODE>
__device__ __forceinline__ void rg_op_item(const RgProb& P, int tile, float2* band, float2 (*sh)[32])
{
    const OpEpilogue& a = MODE == 1 ? P.ep_q : P.ep_res;
    const VT* val = static_cast<const VT*>(P.Atval);
    int64_t t;
    float2 d;
    if (P.chunked) {
        t = (int64_t)tile * kTilePix + threadIdx.x;
        d = band_dot_chunked<VT, float2, true, false>(P.bv, val, tile, P.y, band, t);
    } else {
        stage_band<float2, true>(P.bv, tile, P.y, band);
        d = band_dot<VT, float2, false>(P.bv, val, tile, band, t);
    }
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
    int i, j;
    tiled_coords(t, P.tn, i, j);
    if (i < P.n && j < P.n) {
        op_epilogue<MODE>(a, P.n, P.tn, t, i, j, d, s0, c0, s1, c1);
    } else {
        a.out[t] = df_zero();
        if (MODE == 2) a.p_out[t] = df_zero();
    }
    float2 v[2] = {acc_value(s0, c0), acc_value(s1, c1)};
    block_sum<2>(v, sh);  // also keeps the band until every lane is done with it
    if (threadIdx.x == 0) {
        const int tiles = P.tn * P.tn;
        P.partials[tile] = v[0];
        P.partials[tiles + tile] = v[1];
    }
}

__device__ __forceinline__ void rg_upd_item(const RgProb& P, int item, float2 (*sh)[32])
{
    const float2 al = __ldcg(&P.cg->alpha_df);
    const int64_t end = min(P.npad, (int64_t)(item + 1) * kRgVecPixels);
    float s = 0.0f, c = 0.0f;
    for (int64_t i = (int64_t)item * kRgVecPixels + threadIdx.x; i < end; i += blockDim.x) {
        P.u[i] = df_add(P.u[i], df_mul(al, P.p[i]));
        const float2 rn = df_sub(P.r[i], df_mul(al, P.q[i]));
        P.r[i] = rn;
        acc_add(s, c, df_mul(rn, rn));
    }
    float2 v[1] = {acc_value(s, c)};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) P.partials[item] = v[0];
}

__device__ __forceinline__ void rg_dir_item(const RgProb& P, int item)
{
    const float2 be = __ldcg(&P.cg->beta_df);
    const int64_t end = min(P.npad, (int64_t)(item + 1) * kRgVecPixels);
    for (int64_t i = (int64_t)item * kRgVecPixels + threadIdx.x; i < end; i += blockDim.x)
        P.p[i] = df_add(P.r[i], df_mul(be, P.p[i]));
}

// shrink(x, gamma) = sign(x) max(|x| - gamma, 0) in double-float.
__device__ __forceinline__ float2 rg_shrink(float2 x, float2 gamma)
{
    const float2 ax = df_abs(x);
    if (!df_gt(ax, gamma)) return df_zero();
    return x.x < 0.0f ? df_add(x, gamma) : df_sub(x, gamma);
}

// g = grad u, d = shrink(g + b, 1/lambda), b += g - d, v = d - b, the L1 size
// of the update, u_old = u (the Bregman step after the inner solve).
__device__ __forceinline__ void rg_shrink_item(const RgProb& P, int item, float2 (*sh)[32])
{
    const int n = P.n, tn = P.tn;
    const int64_t end = min(P.npad, (int64_t)(item + 1) * kRgVecPixels);
    float s = 0.0f, cc = 0.0f;
    for (int64_t p = (int64_t)item * kRgVecPixels + threadIdx.x; p < end; p += blockDim.x) {
        int i, j;
        tiled_coords(p, tn, i, j);
        if (i >= n || j >= n) continue;
        const float2 c = P.u[p];
        const float2 gx = (j < n - 1) ? df_sub(P.u[tiled_index(i, j + 1, tn)], c) : df_zero();
        const float2 gy = (i < n - 1) ? df_sub(P.u[tiled_index(i + 1, j, tn)], c) : df_zero();
        const float2 tx = df_add(gx, P.bx[p]), ty = df_add(gy, P.by[p]);
        const float2 dx = rg_shrink(tx, P.gamma), dy = rg_shrink(ty, P.gamma);
        const float2 bxn = df_sub(tx, dx), byn = df_sub(ty, dy);
        P.bx[p] = bxn;
        P.by[p] = byn;
        P.vx[p] = df_sub(dx, bxn);
        P.vy[p] = df_sub(dy, byn);
        acc_add(s, cc, df_abs(df_sub(c, P.u_old[p])));
        P.u_old[p] = c;
    }
    float2 v[1] = {acc_value(s, cc)};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) P.partials[item] = v[0];
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <typename VT>
__device__ __forceinline__ void rg_run_item(const RgProb& P, int kind, int item, float2* band, float2 (*sh)[32])
{
    switch (kind) {
    case RG_FWD_U: rg_fwd_item<VT>(P, P.u, item); break;
    case RG_FWD_P: rg_fwd_item<VT>(P, P.p, item); break;
    case RG_OP_RES: rg_op_item<VT, 2>(P, item, band, sh); break;
    case RG_OP_Q: rg_op_item<VT, 1>(P, item, band, sh); break;
    case RG_UPD: rg_upd_item(P, item, sh); break;
    case RG_DIR: rg_dir_item(P, item); break;
    default: rg_shrink_item(P, item, sh); break;
    }
}

// The last item of a phase: the phase's totals and the scalar update.
__device__ __forceinline__ void rg_finalize(const RgProb& P, int kind, int count, float2 (*sh)[32])
{
    if (kind == RG_OP_RES || kind == RG_OP_Q) {
        double tot[2];
        phase_totals<2>(P.partials, count, tot, sh);
        if (threadIdx.x == 0) {
            if (kind == RG_OP_RES)
                cg_after_residual(*P.cg, tot[0], tot[1], P.ep_res.tol);
            else
                cg_after_pq(*P.cg, tot[0]);
        }
    } else if (kind == RG_UPD || kind == RG_SHRINK) {
        double tot[1];
        phase_totals<1>(P.partials, count, tot, sh);
        if (threadIdx.x == 0) {
            if (kind == RG_UPD) {
                cg_after_update(*P.cg, tot[0], P.ep_q.tol);
            } else if (P.cg->status != CT_OK) {
                P.sb->status = P.cg->status;
                P.sb->stopped = 1;
            } else {
                sb_after_update(*P.sb, tot[0], P.stop_tol);
            }
        }
    }
}

__global__ void __launch_bounds__(kRgThreads, kRgMinBlocks)
    ragged_kernel(const RgProb* __restrict__ probs, const RgPhase* __restrict__ phases, int nphases, int total,
                  int* arrive, int* done, RgCtl* ctl, long long limit, int hold)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float2* band = reinterpret_cast<float2*>(smem);
    __shared__ float2 sh[2][32];
    __shared__ int s_phase, s_item, s_go, s_work, s_last;
    for (;;) {
        if (threadIdx.x == 0) {
            int go = 0, ph = -1, work = 0;
            const int t = ld_acquire(&ctl->abort) ? -1 : atomicAdd(&ctl->ticket, 1);
            if (t >= 0 && t < total) {
                int lo = 0, hi = nphases - 1;  // the last phase starting at or before t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (phases[mid].first <= t) lo = mid; else hi = mid - 1;
                }
                ph = lo;
                const RgPhase f = phases[ph];
                const int* flag = f.dep >= 0 ? done + f.dep : (hold ? &ctl->never : nullptr);
                go = 1;
                if (flag) {
                    long long polls = 0;
                    while (ld_acquire(flag) == 0) {
                        if (ld_acquire(&ctl->abort)) {
                            go = 0;
                            break;
                        }
                        if (++polls > limit) {
                            go = 0;
                            if (atomicCAS(&ctl->status, 0, CT_ERR_TIMEOUT) == 0) atomicExch(&ctl->where, ph);
                            atomicExch(&ctl->abort, 1);
                            break;
                        }
                        __nanosleep(128);
                    }
                }
                if (go) {
                    const RgProb& P = probs[f.prob];
                    const bool stopped = ld_cg_int(&P.sb->stopped) != 0;
                    const bool gated = f.kind == RG_FWD_P || f.kind == RG_OP_Q || f.kind == RG_UPD || f.kind == RG_DIR;
                    work = !stopped && !(gated && ld_cg_int(&P.cg->active) == 0);
                }
                s_item = t - f.first;
            }
            s_phase = ph;
            s_go = go;
            s_work = work;
        }
        __syncthreads();
        if (!s_go) break;
        const RgPhase f = phases[s_phase];
        const RgProb& P = probs[f.prob];
        if (s_work) {
            if (P.f16)
                rg_run_item<__half>(P, f.kind, s_item, band, sh);
            else
                rg_run_item<float>(P, f.kind, s_item, band, sh);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(arrive + s_phase, 1) == f.count - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (s_work) rg_finalize(P, f.kind, f.count, sh);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                st_release(done + s_phase, 1);
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace ct

namespace ct {
namespace {

constexpr long long kDefaultWaitLimit = 1LL << 22;  // polls of 128 ns and more: about a second
std::mutex g_wait_mutex;
long long g_wait_limit = kDefaultWaitLimit;
int g_wait_hold = 0;

const char* kind_name(int k)
{
    static const char* names[] = {"y = A u", "r = rhs - Op(u)", "y = A p", "q = Op(p)", "u, r update",
                                  "p = r + beta p", "shrink"};
    return k >= 0 && k < 7 ? names[k] : "?";
}

template <typename T>
int dev_upload(T** dst, const std::vector<T>& src)
{
    cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(src.size(), 1));
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return fail(CT_ERR_OOM, "device allocation for the ragged work queue failed");
    }
    CT_CUDA(e);
    if (!src.empty()) CT_CUDA(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return CT_OK;
}

}  // namespace

void set_wait_limit(long long polls, int hold)
{
    std::lock_guard<std::mutex> lock(g_wait_mutex);
    g_wait_limit = polls > 0 ? polls : kDefaultWaitLimit;
    g_wait_hold = hold ? 1 : 0;
}

// Runs `outer` Bregman updates of every prepared single-slice run as one
// persistent launch per update (see the top of this file).  *used = false
// (and nothing runs) when a run is not the exact sparse operator (surrogate,
// residual refresh), which the kernel does not cover.
int ragged_persistent(const std::vector<Sb1Run*>& runs, int outer, cudaStream_t st, cudaStream_t cap, bool* used)
{
    *used = false;
    if (runs.empty()) return CT_OK;
    std::vector<RgProb> hp;
    int inner = -1;
    size_t smem = 0;
    int device = -1, sms = 0;
    for (Sb1Run* r : runs) {
        Sb1Desc d;
        sb1_describe(r, &d);
        if (!d.exact || (inner >= 0 && d.inner != inner)) return CT_OK;
        inner = d.inner;
        const ct_matrix* M = d.M;
        Workspace& w = *d.w;
        device = M->device;
        sms = M->sm_count;
        RgProb p;
        std::memset(&p, 0, sizeof(p));
        p.f16 = d.vk == ValKind::F16;
        p.A = SellView{M->A.slice_ptr, M->A.row_len, M->A.rows};
        p.Acol = M->A.col;
        p.Aval = p.f16 ? static_cast<const void*>(M->A.qval) : static_cast<const void*>(M->A.val);
        p.row_scale = M->row_scale;
        p.bv = BandView{M->At.slice_ptr, M->At.row_len, M->At.col16, M->band_lo, M->band_off, M->band_chunk,
                        (int)M->h_band_chunk.size() - 1, M->band_total, M->g.n, M->tn, M->g.n_bins, M->n_kept};
        p.Atval = p.f16 ? static_cast<const void*>(M->At.qval) : static_cast<const void*>(M->At.val);
        p.chunked = M->h_band_chunk.size() > 2;
        p.n = M->g.n;
        p.tn = M->tn;
        p.npad = M->npad;
        p.ep_res = d.base;
        p.ep_res.mode = 2;
        p.ep_res.in = w.u;
        p.ep_res.out = w.r;
        p.ep_res.p_out = w.p;
        p.ep_res.rhs = nullptr;
        p.ep_q = d.base;
        p.ep_q.mode = 1;
        p.ep_q.in = w.p;
        p.ep_q.out = w.q;
        p.u = w.u;
        p.r = w.r;
        p.p = w.p;
        p.q = w.q;
        p.y = w.y;
        p.u_old = w.u_old;
        p.bx = w.bx;
        p.by = w.by;
        p.vx = w.vx;
        p.vy = w.vy;
        p.cg = w.cg;
        p.sb = w.sb;
        p.partials = w.partials;
        p.gamma = df_from_double(d.gamma);
        p.stop_tol = d.stop_tol;
        const int64_t vec_items = (M->npad + kRgVecPixels - 1) / kRgVecPixels;
        if (w.partials_len < std::max<int64_t>(2 * (int64_t)M->tn * M->tn, vec_items))
            return fail(CT_ERR_CUDA, "internal: reduction partials too small for the ragged kernel");
        smem = std::max(smem, (size_t)M->band_chunk_slots * sizeof(float2));
        hp.push_back(p);
    }
    // the queue: every problem's phases, step by step across the problems
    const int P = (int)hp.size();
    std::vector<int> kinds = {RG_FWD_U, RG_OP_RES};
    for (int it = 0; it < inner; ++it) {
        kinds.push_back(RG_FWD_P);
        kinds.push_back(RG_OP_Q);
        kinds.push_back(RG_UPD);
        kinds.push_back(RG_DIR);
    }
    kinds.push_back(RG_SHRINK);
    std::vector<RgPhase> ph;
    std::vector<int> last(P, -1);
    int64_t cursor = 0;
    for (int k : kinds) {
        for (int i = 0; i < P; ++i) {
            const RgProb& p = hp[i];
            int64_t count;
            if (k == RG_FWD_U || k == RG_FWD_P)
                count = ((p.A.rows + kSliceRows - 1) / kSliceRows + kRgFwdSlices - 1) / kRgFwdSlices;
            else if (k == RG_OP_RES || k == RG_OP_Q)
                count = (int64_t)p.tn * p.tn;
            else
                count = (p.npad + kRgVecPixels - 1) / kRgVecPixels;
            ph.push_back(RgPhase{i, k, (int32_t)cursor, (int32_t)count, last[i]});
            last[i] = (int)ph.size() - 1;
            cursor += count;
            if (cursor >= ((int64_t)1 << 31)) return fail(CT_ERR_UNSUPPORTED, "ragged work queue too long");
        }
    }
    const int nph = (int)ph.size(), total = (int)cursor;
    (void)device;
    if (smem > 48 * 1024)
        CT_CUDA(cudaFuncSetAttribute(ragged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ragged_kernel, kRgThreads, smem));
    if (per_sm < 1) return fail(CT_ERR_UNSUPPORTED, "the ragged kernel does not fit an SM");
    const int grid = per_sm * (sms > 0 ? sms : 1);
    long long limit;
    int hold;
    {
        std::lock_guard<std::mutex> lock(g_wait_mutex);
        limit = g_wait_limit;
        hold = g_wait_hold;
    }
    RgProb* d_probs = nullptr;
    RgPhase* d_phases = nullptr;
    int* d_cnt = nullptr;
    RgCtl* d_ctl = nullptr;
    auto release = [&]() {
        cudaFree(d_probs);
        cudaFree(d_phases);
        cudaFree(d_cnt);
        cudaFree(d_ctl);
    };
    int rc = dev_upload(&d_probs, hp);
    if (rc == CT_OK) rc = dev_upload(&d_phases, ph);
    if (rc == CT_OK) rc = dev_upload(&d_cnt, std::vector<int>(2 * (size_t)nph, 0));
    if (rc == CT_OK) rc = dev_upload(&d_ctl, std::vector<RgCtl>(1, RgCtl{0, 0, -1, 0, 0}));
    if (rc != CT_OK) {
        release();
        return rc;
    }
    int* d_arrive = d_cnt;
    int* d_done = d_cnt + nph;
    auto update = [&](cudaStream_t s) -> int {
        CT_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int) * 2 * (size_t)nph, s));
        CT_CUDA(cudaMemsetAsync(&d_ctl->ticket, 0, sizeof(int), s));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kRgThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CT_CUDA(cudaLaunchKernelEx(&cfg, ragged_kernel, (const RgProb*)d_probs, (const RgPhase*)d_phases, nph, total,
                                   d_arrive, d_done, d_ctl, limit, hold));
        return CT_OK;
    };
    rc = run_updates({update}, {cap}, outer, st);
    bool direct = false;
    if (rc != CT_OK) {
        // a capture the runtime refused: run the updates directly on st
        (void)cudaGetLastError();
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            rc = CT_OK;
            direct = true;
            for (int k = 0; k < outer && rc == CT_OK; ++k) rc = update(st);
        }
    }
    RgCtl h{};
    if (rc == CT_OK) {
        cudaError_t e = cudaMemcpyAsync(&h, d_ctl, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "reading the ragged kernel's status", __FILE__, __LINE__);
    } else {
        cudaStreamSynchronize(st);
    }
    release();
    if (rc != CT_OK) return rc;
    *used = true;
    // a note, not a failure: ct_last_error() tells that the updates ran as
    // separate launches because the graph capture was refused
    set_error(direct ? "ragged: the CUDA graph capture of the persistent kernel was refused; the updates ran as "
                       "direct launches"
                     : "");
    if (h.status != CT_OK) {
        const int w = h.where;
        std::string where = "?";
        if (w >= 0 && w < nph) {
            const int dep = ph[w].dep;
            where = "problem " + std::to_string(ph[w].prob) + ", phase '" + kind_name(ph[w].kind) + "'" +
                    (dep >= 0 ? std::string(" waiting for '") + kind_name(ph[dep].kind) + "'" : std::string(" (held)"));
        }
        return fail(h.status, "a bounded wait of the ragged kernel expired (" + where + ")");
    }
    return CT_OK;
}

}  // namespace ct
