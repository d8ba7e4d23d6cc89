// Conjugate gradients for (c_id I + c_ata A^T A + c_grad grad^T grad) u = rhs
// (Eqs. KKT, PD_resolve, SB_solve) and anisotropic-TV split Bregman (Sec. 4),
// with every scalar kept on the device so that a whole reconstruction is one
// stream of kernels (captured as a CUDA graph per Bregman update) and the host
// never waits inside the loop.
//
// One CG step is four kernels: y = A p; q = Op(p) fused into the A^T product
// (with p.q); u += alpha p, r -= alpha q (with r.r); p = r + beta p.  The
// iteration vectors are double-float pairs (a fixed number of CG steps
// amplifies their rounding by orders of magnitude, see solver_ops.cu); each
// reduction is finished by the last block of its kernel in a fixed order, so
// results are bitwise reproducible run to run.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>

#include "ct_internal.cuh"
#include "dfloat.cuh"
#include "grad.cuh"
#include "reduce.cuh"

namespace ct {
namespace {

__global__ void __launch_bounds__(256) cg_update_kernel(float2* __restrict__ u, float2* __restrict__ r,
                                                        const float2* __restrict__ p,
                                                        const float2* __restrict__ q, int64_t len,
                                                        CgSlice* cg, double tol, float2* partials,
                                                        unsigned* counter, const int32_t* gate)
{
    if (gate && *gate) return;
    if (!cg->active) return;
    const float2 al = cg->alpha_df;
    float s = 0.0f, c = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        u[i] = df_add(u[i], df_mul(al, p[i]));
        const float2 rn = df_sub(r[i], df_mul(al, q[i]));
        r[i] = rn;
        acc_add(s, c, df_mul(rn, rn));
    }
    float2 v[1] = {acc_value(s, c)};
    double tot[1];
    if (grid_reduce_last<1>(v, partials, counter, tot)) cg_after_update(*cg, tot[0], tol);
}

__global__ void __launch_bounds__(256) cg_direction_kernel(float2* __restrict__ p, const float2* __restrict__ r,
                                                           int64_t len, const CgSlice* cg, const int32_t* gate)
{
    if (gate && *gate) return;
    if (!cg->active) return;
    const float2 be = cg->beta_df;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = df_add(r[i], df_mul(be, p[i]));
}

// shrink(x, gamma) = sign(x) max(|x| - gamma, 0) in double-float.
__device__ __forceinline__ float2 shrink_df(float2 x, float2 gamma)
{
    const float2 ax = df_abs(x);
    if (!df_gt(ax, gamma)) return df_zero();
    return x.x < 0.0f ? df_add(x, gamma) : df_sub(x, gamma);
}

// After the inner solve: g = grad u, d = shrink(g + b, 1/lambda), b += g - d,
// v = d - b (the next right-hand side's split term), ||u - u_old||_1, u_old = u.
__global__ void __launch_bounds__(256) sb_shrink_kernel(const float2* __restrict__ u,
                                                        float2* __restrict__ u_old,
                                                        float2* __restrict__ bx, float2* __restrict__ by,
                                                        float2* __restrict__ vx, float2* __restrict__ vy,
                                                        int n, int tn, float2 gamma, SbSlice* sb,
                                                        const CgSlice* cg, double tol,
                                                        float2* partials, unsigned* counter)
{
    if (sb->stopped) return;
    const int64_t npad = padded_pixels(n);
    float s = 0.0f, cc = 0.0f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npad;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(p, tn, i, j);
        if (i >= n || j >= n) continue;
        const float2 c = u[p];
        const float2 gx = (j < n - 1) ? df_sub(u[tiled_index(i, j + 1, tn)], c) : df_zero();
        const float2 gy = (i < n - 1) ? df_sub(u[tiled_index(i + 1, j, tn)], c) : df_zero();
        const float2 tx = df_add(gx, bx[p]), ty = df_add(gy, by[p]);
        const float2 dx = shrink_df(tx, gamma), dy = shrink_df(ty, gamma);
        const float2 bxn = df_sub(tx, dx), byn = df_sub(ty, dy);
        bx[p] = bxn;
        by[p] = byn;
        vx[p] = df_sub(dx, bxn);
        vy[p] = df_sub(dy, byn);
        acc_add(s, cc, df_abs(df_sub(c, u_old[p])));
        u_old[p] = c;
    }
    float2 v[1] = {acc_value(s, cc)};
    double tot[1];
    if (grid_reduce_last<1>(v, partials, counter, tot)) {
        if (cg->status != CT_OK) {
            sb->status = cg->status;
            sb->stopped = 1;
        } else {
            sb_after_update(*sb, tot[0], tol);
        }
    }
}

// ---------------------------------------------------------------------------
// Chambolle-Pock primal-dual steps around the resolvent of Eq. PD_resolve
// (Sec. 2), for alpha/2 ||A u - g||^2 + ||grad u||_1: the dual ascent and
// projection onto the box |p| <= 1, the resolvent's right-hand side, and the
// extrapolation with the size of the update.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 clip_unit(float2 x)
{
    const float2 one = make_float2(1.0f, 0.0f), mone = make_float2(-1.0f, 0.0f);
    if (df_gt(x, one)) return one;
    if (df_gt(mone, x)) return mone;
    return x;
}

// p = clip(p + sigma grad(ubar), -1, 1), per component.
__global__ void __launch_bounds__(256) cp_dual_kernel(const float2* __restrict__ ubar, float2* __restrict__ px,
                                                      float2* __restrict__ py, int n, int tn, float2 sigma,
                                                      const SbSlice* sb)
{
    if (sb->stopped) return;
    const int64_t npad = padded_pixels(n);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npad;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(p, tn, i, j);
        if (i >= n || j >= n) continue;
        const float2 c = ubar[p];
        const float2 gx = (j < n - 1) ? df_sub(ubar[tiled_index(i, j + 1, tn)], c) : df_zero();
        const float2 gy = (i < n - 1) ? df_sub(ubar[tiled_index(i + 1, j, tn)], c) : df_zero();
        px[p] = clip_unit(df_add(px[p], df_mul(sigma, gx)));
        py[p] = clip_unit(df_add(py[p], df_mul(sigma, gy)));
    }
}

// rhs = u - tau grad^T p + tau alpha A^T g (Eq. PD_resolve with u~ = u - tau grad^T p);
// u_old = u.
__global__ void __launch_bounds__(256) cp_rhs_kernel(const float2* __restrict__ u, const float2* __restrict__ px,
                                                     const float2* __restrict__ py, const float2* __restrict__ atf,
                                                     float2* __restrict__ rhs, float2* __restrict__ u_old, int n,
                                                     int tn, float2 ntau, const SbSlice* sb)
{
    if (sb->stopped) return;
    const int64_t npad = padded_pixels(n);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npad;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(p, tn, i, j);
        if (i >= n || j >= n) continue;
        const float2 c = u[p];
        rhs[p] = df_add(df_add(c, atf[p]), df_mul(ntau, grad_adj_df(px, py, p, i, j, n, tn)));
        u_old[p] = c;
    }
}

// ubar = u + theta (u - u_old); the L1 size of the update ends in the
// slice's update bookkeeping (the last block).
__global__ void __launch_bounds__(256) cp_extrap_kernel(const float2* __restrict__ u,
                                                        const float2* __restrict__ u_old, float2* __restrict__ ubar,
                                                        int n, int tn, float2 theta, SbSlice* sb, const CgSlice* cg,
                                                        float2* partials, unsigned* counter)
{
    if (sb->stopped) return;
    const int64_t npad = padded_pixels(n);
    float s = 0.0f, cc = 0.0f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npad;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(p, tn, i, j);
        if (i >= n || j >= n) continue;
        const float2 d = df_sub(u[p], u_old[p]);
        ubar[p] = df_add(u[p], df_mul(theta, d));
        acc_add(s, cc, df_abs(d));
    }
    float2 v[1] = {acc_value(s, cc)};
    double tot[1];
    if (grid_reduce_last<1>(v, partials, counter, tot)) {
        if (cg->status != CT_OK) {
            sb->status = cg->status;
            sb->stopped = 1;
        } else {
            sb_after_update(*sb, tot[0], 0.0);
        }
    }
}

// Caller's row-major FP32 image -> internal tiled double-float (padding zero).
__global__ void widen_kernel(const float* __restrict__ in, float2* __restrict__ out, int n, int tn)
{
    const int64_t npad = padded_pixels(n);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npad;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(t, tn, i, j);
        out[t] = (i < n && j < n) ? make_float2(in[(int64_t)i * n + j], 0.0f) : make_float2(0.0f, 0.0f);
    }
}

__global__ void narrow_kernel(const float2* __restrict__ in, float* __restrict__ out, int n, int tn)
{
    const int64_t npad = padded_pixels(n);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npad;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(t, tn, i, j);
        if (i < n && j < n) out[(int64_t)i * n + j] = df_to_float(in[t]);
    }
}

template <typename T>
int alloc_n(T** p, int64_t n)
{
    cudaError_t e = cudaMalloc((void**)p, (size_t)(n > 0 ? n : 1) * sizeof(T));
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return fail(CT_ERR_OOM, "workspace allocation failed");
    }
    CT_CUDA(e);
    return CT_OK;
}

struct Plan {
    ct_matrix* M;
    Workspace* w;      // vectors, scalars and reduction buffers of this solve
    ValKind vk;
    bool sparse;       // A^T A through the sparse products (else stencil / none)
    const Stencil* S;  // surrogate stencil, or null
    OpEpilogue base;
    int64_t n2;
    int refresh;       // residual replacement period (FP16 storage), 0 = off
};

// Op applied to `in` with the given epilogue (y = A in, then A^T y fused).
int apply_op(const Plan& P, OpEpilogue ep, const float2* in, cudaStream_t st, bool fp32_refresh = false)
{
    Workspace& w = *P.w;
    ep.in = in;
    if (P.sparse && P.M->fourier) {
        CT_CHECK(launch_fourier_op_df(P.M, ep, st));
    } else if (P.sparse) {
        const ValKind vk = fp32_refresh ? ValKind::F32 : P.vk;
        CT_CHECK(launch_forward_df(P.M, vk, in, w.y, vk == ValKind::F16 ? 2 : 0,
                                   ep.mode == 2 ? nullptr : ep.cg, ep.gate, st));
        CT_CHECK(launch_adjoint_op_df(P.M, vk, w.y, ep, st));
    } else {
        CT_CHECK(launch_stencil_op_df(P.M, P.S, ep, st));
    }
    return CT_OK;
}

// Residual r = rhs - Op(u), p = r, then `iters` CG steps on the iterate w.u.
int enqueue_cg(const Plan& P, const float2* rhs, int iters, cudaStream_t st)
{
    Workspace& w = *P.w;
    OpEpilogue ep = P.base;
    ep.mode = 2;
    ep.out = w.r;
    ep.p_out = w.p;
    ep.rhs = rhs;
    CT_CHECK(apply_op(P, ep, w.u, st));
    const int gv = grid_for(P.M, P.n2, 256, 8);
    for (int it = 0; it < iters; ++it) {
        OpEpilogue e1 = P.base;
        e1.mode = 1;
        e1.out = w.q;
        CT_CHECK(apply_op(P, e1, w.p, st));
        cg_update_kernel<<<gv, 256, 0, st>>>(w.u, w.r, w.p, w.q, P.n2, w.cg, P.base.tol, w.partials,
                                             w.counter, P.base.gate);
        CT_CUDA(cudaGetLastError());
        cg_direction_kernel<<<gv, 256, 0, st>>>(w.p, w.r, P.n2, w.cg, P.base.gate);
        CT_CUDA(cudaGetLastError());
        if (P.refresh > 0 && (it + 1) % P.refresh == 0 && it + 1 < iters) {
            OpEpilogue e3 = P.base;
            e3.mode = 3;
            e3.out = w.r;
            e3.rhs = rhs;
            CT_CHECK(apply_op(P, e3, w.u, st, true));
        }
    }
    return CT_OK;
}

int make_plan(ct_matrix* M, Workspace* ws, double c_id, double c_ata, double c_grad, double tol, int surr_r,
              int surr_square, int refresh, Plan& P)
{
    P.M = M;
    P.w = ws;
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
            return fail(CT_ERR_UNSUPPORTED,
                        "refresh_every needs FP16 storage built with CT_KEEP_FP32_COPY");
        if (!P.sparse) refresh = 0;
    }
    P.refresh = refresh;
    Workspace& w = *ws;
    if (w.partials_len < (int64_t)2 * M->tn * M->tn)
        return fail(CT_ERR_CUDA, "internal: reduction partials smaller than the fused adjoint's grid needs");
    OpEpilogue& b = P.base;
    std::memset(&b, 0, sizeof(b));
    b.c_id = df_from_double(c_id);
    b.c_ata = df_from_double(c_ata);
    b.c_grad = df_from_double(c_grad);
    b.cg = w.cg;
    b.partials = w.partials;
    b.counter = w.counter;
    b.tol = tol;
    return CT_OK;
}

// w.atf = scale A^T f for a real sinogram f (double-float, tiled): the
// Siddon adjoint, or Re(F^H fhat) of the data's DFTs on a Fourier handle.
int backproject_data(ct_matrix* M, ValKind vk, const float* f, Workspace& w, double scale, cudaStream_t st)
{
    if (M->fourier) return fourier_backproject_df(M, f, w.atf, scale, st);
    CT_CHECK(launch_to_df(M, f, vk == ValKind::F16 ? M->row_scale : nullptr, w.y, M->rows, st));
    return launch_adjoint_df(M, vk, w.y, w.atf, scale, st);
}

}  // namespace

void free_workspace(Workspace& w)
{
    float2* vs[] = {w.u, w.r, w.p, w.q, w.rhs, w.atf, w.u_old, w.bx, w.by, w.vx, w.vy, w.y, w.pub_y2};
    for (float2* v : vs) cudaFree(v);
    cudaFree(w.stage_a);
    cudaFree(w.stage_b);
    cudaFree(w.pub_x);
    cudaFree(w.f64_y);
    cudaFree(w.f64_a);
    cudaFree(w.f64_b);
    cudaFree(w.f64_c);
    cudaFree(w.partials);
    cudaFree(w.counter);
    cudaFree(w.cg);
    cudaFree(w.sb);
    cudaFree(w.ragged_ptrs);
    if (w.cap_stream) cudaStreamDestroy(w.cap_stream);
    w = Workspace{};
}

int ensure_workspace(ct_matrix* M, int32_t batch, bool /*solver*/) { return ensure_workspace_in(M, M->ws, batch); }

int ensure_workspace_in(ct_matrix* M, Workspace& w, int32_t batch)
{
    if (w.batch >= batch && w.r) return CT_OK;
    CT_CUDA(cudaDeviceSynchronize());
    cudaStream_t keep = w.cap_stream;
    float** rptr = w.ragged_ptrs;
    const int32_t rcap = w.ragged_cap;
    float* sa = w.stage_a;
    float* sb = w.stage_b;
    float2* py = w.pub_y2;
    float* pxx = w.pub_x;
    const int64_t la = w.stage_a_len, lb = w.stage_b_len, lp = w.pub_y2_len, lxx = w.pub_x_len;
    w.cap_stream = nullptr;
    w.ragged_ptrs = nullptr;
    w.stage_a = w.stage_b = nullptr;
    w.pub_y2 = nullptr;
    w.pub_x = nullptr;
    free_workspace(w);
    w.cap_stream = keep;
    w.ragged_ptrs = rptr;
    w.ragged_cap = rcap;
    w.stage_a = sa;
    w.stage_b = sb;
    w.pub_y2 = py;
    w.stage_a_len = la;
    w.stage_b_len = lb;
    w.pub_y2_len = lp;
    w.pub_x = pxx;
    w.pub_x_len = lxx;
    w.batch = batch;
    w.n2 = M->npad;
    w.rows = M->rows;
    const int64_t nv = w.n2 * batch;
    float2** vs[] = {&w.u, &w.r, &w.p, &w.q, &w.rhs, &w.atf, &w.u_old, &w.bx, &w.by, &w.vx, &w.vy};
    for (float2** v : vs) CT_CHECK(alloc_n(v, nv));
    CT_CHECK(alloc_n(&w.y, w.rows * batch));
    // grid-wide reductions write NQ <= 2 partials per block: the batched
    // kernels run at most 8 blocks per SM per 32-slice chunk, the fused
    // adjoint one block per image tile
    w.partials_len = std::max((int64_t)4 * (M->sm_count > 0 ? M->sm_count : 148) * 8 * batch,
                              (int64_t)2 * M->tn * M->tn);
    CT_CHECK(alloc_n(&w.partials, w.partials_len));
    CT_CHECK(alloc_n(&w.counter, 16));
    CT_CUDA(cudaMemset(w.counter, 0, 16 * sizeof(unsigned)));
    CT_CHECK(alloc_n(&w.cg, batch));
    CT_CUDA(cudaMemset(w.cg, 0, sizeof(CgSlice) * batch));
    CT_CHECK(alloc_n(&w.sb, batch));
    CT_CUDA(cudaMemset(w.sb, 0, sizeof(SbSlice) * batch));
    if (!w.cap_stream) CT_CUDA(cudaStreamCreateWithFlags(&w.cap_stream, cudaStreamNonBlocking));
    return CT_OK;
}

int cg_solve_in(ct_matrix* M, Workspace& w, const ct_cg_params* Pp, const float* rhs, float* u,
                ct_cg_stats* stats, cudaStream_t st)
{
    Plan P;
    CT_CHECK(make_plan(M, &w, Pp->c_id, Pp->c_ata, Pp->c_grad, Pp->rel_tol, Pp->surrogate_r,
                       Pp->surrogate_square, Pp->refresh_every, P));
    const int gv = grid_for(M, P.n2, 256, 8);
    widen_kernel<<<gv, 256, 0, st>>>(rhs, w.rhs, M->g.n, M->tn);
    widen_kernel<<<gv, 256, 0, st>>>(u, w.u, M->g.n, M->tn);
    CT_CUDA(cudaGetLastError());
    CT_CHECK(enqueue_cg(P, w.rhs, Pp->max_iters, st));
    narrow_kernel<<<gv, 256, 0, st>>>(w.u, u, M->g.n, M->tn);
    CT_CUDA(cudaGetLastError());
    if (stats) {
        CgSlice h;
        CT_CUDA(cudaMemcpyAsync(&h, w.cg, sizeof(h), cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaStreamSynchronize(st));
        stats->iters = h.iters;
        stats->final_rel_res = h.rhs2 > 0 ? std::sqrt(h.rr / h.rhs2) : 0.0;
        stats->status = h.status;
        if (h.status != CT_OK)
            return fail(h.status, h.status == CT_ERR_BREAKDOWN ? "CG breakdown: p^T Op p <= 0"
                                                               : "non-finite value in CG");
    }
    return CT_OK;
}

int cg_solve(ct_matrix* M, const ct_cg_params* Pp, const float* rhs, float* u, int32_t batch,
             ct_cg_stats* stats, cudaStream_t st)
{
    if (Pp->max_iters < 0) return fail(CT_ERR_ARG, "max_iters < 0");
    if (batch != 1 && M->fourier) return fail(CT_ERR_UNSUPPORTED, "the Fourier operator solves one slice per call");
    if (batch != 1) return cg_solve_batched(M, Pp, rhs, u, batch, stats, st);
    CT_CHECK(tune_single(M, st));
    CT_CHECK(ensure_workspace(M, batch, true));
    return cg_solve_in(M, M->ws, Pp, rhs, u, stats, st);
}

namespace {

__global__ void fill_df_kernel(float2* __restrict__ v, int n, int tn, float hi)
{
    const int64_t npad = padded_pixels(n);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npad;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i, j;
        tiled_coords(t, tn, i, j);
        v[t] = (i < n && j < n) ? make_float2(hi, 0.0f) : make_float2(0.0f, 0.0f);
    }
}

// p = r = 1 on the image, u = q = 0 and an active slice: every product of a
// CG step is then finite with p.q > 0, so the scalars keep the slice active
// through any number of launches (for timing).
int prime_cg_workspace(ct_matrix* M, Workspace& w, int64_t n2, cudaStream_t st)
{
    const int gv = grid_for(M, n2, 256, 8);
    fill_df_kernel<<<gv, 256, 0, st>>>(w.p, M->g.n, M->tn, 1.0f);
    fill_df_kernel<<<gv, 256, 0, st>>>(w.r, M->g.n, M->tn, 1.0f);
    fill_df_kernel<<<gv, 256, 0, st>>>(w.u, M->g.n, M->tn, 0.0f);
    fill_df_kernel<<<gv, 256, 0, st>>>(w.q, M->g.n, M->tn, 0.0f);
    CT_CUDA(cudaGetLastError());
    CgSlice h;
    std::memset(&h, 0, sizeof(h));
    h.rr = h.rhs2 = 1.0;
    h.active = 1;
    CT_CUDA(cudaMemcpyAsync(w.cg, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    return CT_OK;
}

// Mean ms per launch of fn over `reps` launches after one untimed one.
template <typename F>
int time_launches(F fn, int reps, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st, float* ms)
{
    CT_CHECK(fn());
    CT_CUDA(cudaEventRecord(e0, st));
    for (int i = 0; i < reps; ++i) CT_CHECK(fn());
    CT_CUDA(cudaEventRecord(e1, st));
    CT_CUDA(cudaEventSynchronize(e1));
    float t = 0.0f;
    CT_CUDA(cudaEventElapsedTime(&t, e0, e1));
    *ms = t / reps;
    return CT_OK;
}

struct TuneKey {
    int n, nt, keep, nb;
    uint32_t flags;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(n, nt, keep, nb, flags) < std::tie(o.n, o.nt, o.keep, o.nb, o.flags);
    }
};
struct TuneVal {
    int fwd_warps, fwd_unroll, op_ctas, op_pixels;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneVal> g_tune_cache;  // choices already measured in this process, by geometry

}  // namespace

// Chooses the launch shape of the single-slice products for this handle: the
// warps per block and chunks in flight of y = A x, and the register budget
// (CTAs per SM) of the fused A^T operator kernel.  Every candidate computes
// the same bits (each row is summed in the same order whatever the shape),
// so only speed depends on the choice.  The candidates are timed on the
// handle's own matrices and workspace; the choice is kept with the handle
// and in a process-wide cache keyed by geometry and storage, so a later
// handle of the same geometry takes it without timing.  Never runs while st
// is being captured; a choice pinned with ct_set_tuning stays.
int tune_single(ct_matrix* M, cudaStream_t st)
{
    if (M->fourier || (M->fwd_warps > 0 && M->fwd_unroll > 0 && M->op_ctas > 0 && M->op_pixels > 0)) return CT_OK;
    const TuneKey key{M->g.n, M->g.n_angles_total, M->g.keep_every, M->g.n_bins, M->flags};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            if (M->fwd_warps <= 0) M->fwd_warps = it->second.fwd_warps;
            if (M->fwd_unroll <= 0) M->fwd_unroll = it->second.fwd_unroll;
            if (M->op_ctas <= 0) M->op_ctas = it->second.op_ctas;
            if (M->op_pixels <= 0) M->op_pixels = it->second.op_pixels;
            return CT_OK;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CT_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return CT_OK;
    CT_CHECK(ensure_workspace(M, 1, true));
    Workspace& w = M->ws;
    Plan P;
    CT_CHECK(make_plan(M, &w, 0.0, 1.0, 1.0, 0.0, 0, 0, 0, P));
    CT_CHECK(prime_cg_workspace(M, w, P.n2, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CT_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate", __FILE__, __LINE__);
    }
    const int pin_w = M->fwd_warps, pin_u = M->fwd_unroll, pin_c = M->op_ctas, pin_p = M->op_pixels;
    const int rpow = P.vk == ValKind::F16 ? 2 : 0;
    const int reps = 3;
    int rc = CT_OK;
    float best = 0.0f;
    int bw = pin_w > 0 ? pin_w : 8, bu = pin_u > 0 ? pin_u : 8;
    bool first = true;
    for (int wv : {8, 4}) {
        for (int uv : {8, 4, 2, 16}) {
            if ((pin_w > 0 && wv != pin_w) || (pin_u > 0 && uv != pin_u) || rc != CT_OK) continue;
            M->fwd_warps = wv;
            M->fwd_unroll = uv;
            float ms = 0.0f;
            rc = time_launches([&]() { return launch_forward_df(M, P.vk, w.p, w.y, rpow, w.cg, nullptr, st); },
                               reps, e0, e1, st, &ms);
            if (rc == CT_OK && (first || ms < best)) {
                best = ms;
                bw = wv;
                bu = uv;
                first = false;
            }
        }
    }
    M->fwd_warps = bw;
    M->fwd_unroll = bu;
    // the fused A^T kernel: (CTAs per SM, pixel rows per lane)
    const bool chunked = M->h_band_chunk.size() > 2;
    int bc = pin_c > 0 ? pin_c : (chunked ? 5 : 7), bp = pin_p > 0 ? pin_p : 1;
    if ((pin_c <= 0 || pin_p <= 0) && rc == CT_OK) {
        OpEpilogue ep = P.base;
        ep.mode = 1;
        ep.out = w.q;
        ep.in = w.p;
        first = true;
        const int cands[4][2] = {{chunked ? 5 : 7, 1}, {chunked ? 3 : 4, 1}, {chunked ? 0 : 3, 1}, {chunked ? 0 : 7, 2}};
        for (const auto& cand : cands) {
            const int cv = cand[0], pv = cand[1];
            if (cv == 0 || rc != CT_OK) continue;
            if ((pin_c > 0 && cv != pin_c) || (pin_p > 0 && pv != pin_p)) continue;
            M->op_ctas = cv;
            M->op_pixels = pv;
            float ms = 0.0f;
            rc = time_launches([&]() { return launch_adjoint_op_df(M, P.vk, w.y, ep, st); }, reps, e0, e1, st, &ms);
            if (rc == CT_OK && (first || ms < best)) {
                best = ms;
                bc = cv;
                bp = pv;
                first = false;
            }
        }
    }
    M->op_ctas = bc;
    M->op_pixels = bp;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CT_OK) return rc;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (pin_w <= 0 && pin_u <= 0 && pin_c <= 0 && pin_p <= 0)
        g_tune_cache[key] = TuneVal{M->fwd_warps, M->fwd_unroll, M->op_ctas, M->op_pixels};
    return CT_OK;
}

// Mean launch time of each kernel of one CG step, launched as the solver
// launches it (same template instances and launch shapes, the handle's
// workspace), `reps` times back to back between two events on st.
int time_cg_kernels(ct_matrix* M, double c_ata, double c_grad, int32_t reps, double* ms, cudaStream_t st)
{
    if (reps < 1) return fail(CT_ERR_ARG, "reps must be >= 1");
    if (M->fourier) return fail(CT_ERR_UNSUPPORTED, "kernel timing needs the Siddon matrices");
    CT_CHECK(tune_single(M, st));
    CT_CHECK(ensure_workspace(M, 1, true));
    Workspace& w = M->ws;
    Plan P;
    CT_CHECK(make_plan(M, &w, 0.0, c_ata, c_grad, 0.0, 0, 0, 0, P));
    const int gv = grid_for(M, P.n2, 256, 8);
    CT_CHECK(prime_cg_workspace(M, w, P.n2, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CT_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate", __FILE__, __LINE__);
    }
    OpEpilogue e1p = P.base;
    e1p.mode = 1;
    e1p.out = w.q;
    e1p.in = w.p;
    int rc = CT_OK;
    for (int k = 0; k < 4 && rc == CT_OK; ++k) {
        auto launch = [&]() -> int {
            switch (k) {
            case 0: return launch_forward_df(M, P.vk, w.p, w.y, P.vk == ValKind::F16 ? 2 : 0, w.cg, nullptr, st);
            case 1: return launch_adjoint_op_df(M, P.vk, w.y, e1p, st);
            case 2:
                cg_update_kernel<<<gv, 256, 0, st>>>(w.u, w.r, w.p, w.q, P.n2, w.cg, 0.0, w.partials, w.counter,
                                                     nullptr);
                return cudaGetLastError() == cudaSuccess ? CT_OK : fail(CT_ERR_CUDA, "launch failed");
            default:
                cg_direction_kernel<<<gv, 256, 0, st>>>(w.p, w.r, P.n2, w.cg, nullptr);
                return cudaGetLastError() == cudaSuccess ? CT_OK : fail(CT_ERR_CUDA, "launch failed");
            }
        };
        for (int i = 0; i < 3 && rc == CT_OK; ++i) rc = launch();  // warm-up
        if (rc != CT_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) rc = fail(CT_ERR_CUDA, "cudaEventRecord failed");
        for (int i = 0; i < reps && rc == CT_OK; ++i) rc = launch();
        if (rc == CT_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = fail(CT_ERR_CUDA, "cudaEventRecord failed");
        if (rc == CT_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(CT_ERR_CUDA, "cudaEventSynchronize failed");
        float t = 0.0f;
        if (rc == CT_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = fail(CT_ERR_CUDA, "event timing failed");
        if (rc == CT_OK) ms[k] = (double)t / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CT_OK) return rc;
    CgSlice back;
    CT_CUDA(cudaMemcpyAsync(&back, w.cg, sizeof(back), cudaMemcpyDeviceToHost, st));
    CT_CUDA(cudaStreamSynchronize(st));
    if (!back.active) return fail(CT_ERR_CUDA, "internal: the timed CG scalars went inactive");
    return CT_OK;
}

namespace {

int enqueue_sb_outer(const Plan& P, const ct_sb_params* Sp, cudaStream_t st)
{
    Workspace& w = *P.w;
    CT_CHECK(enqueue_cg(P, nullptr, Sp->inner_cg_iters, st));
    const int gv = grid_for(P.M, P.n2, 256, 8);
    sb_shrink_kernel<<<gv, 256, 0, st>>>(w.u, w.u_old, w.bx, w.by, w.vx, w.vy, P.M->g.n, P.M->tn,
                                         df_from_double(1.0 / Sp->lambda), w.sb, w.cg, Sp->stop_rel_update,
                                         w.partials, w.counter);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

// Single-slice split Bregman in phases: set-up, one Bregman update (replayed
// by run_updates), read-out.
struct Sb1Run {
    ct_matrix* M = nullptr;
    const ct_sb_params* Sp = nullptr;
    Plan P;
};

void sb1_free(Sb1Run* r) { delete r; }

void sb1_describe(const Sb1Run* r, Sb1Desc* d)
{
    d->M = r->M;
    d->w = r->P.w;
    d->base = r->P.base;
    d->vk = r->P.vk;
    d->exact = r->P.sparse && !r->M->fourier && r->P.refresh == 0;
    d->gamma = 1.0 / r->Sp->lambda;
    d->stop_tol = r->Sp->stop_rel_update;
    d->inner = r->Sp->inner_cg_iters;
}

int sb1_prepare(ct_matrix* M, Workspace& w, const ct_sb_params* Sp, const float* f, const float* u, Sb1Run** out,
                cudaStream_t st)
{
    *out = nullptr;
    const int32_t batch = 1;
    std::unique_ptr<Sb1Run> R(new (std::nothrow) Sb1Run());
    if (!R) return fail(CT_ERR_OOM, "host allocation failed");
    R->M = M;
    R->Sp = Sp;
    CT_CHECK(tune_single(M, st));
    CT_CHECK(ensure_workspace_in(M, w, batch));
    Plan& P = R->P;
    CT_CHECK(make_plan(M, &w, 0.0, Sp->alpha, Sp->lambda, Sp->cg_rel_tol, Sp->surrogate_r, Sp->surrogate_square,
                       Sp->refresh_every, P));
    P.base.gate = &w.sb->stopped;
    P.base.atf = w.atf;
    P.base.vx = w.vx;
    P.base.vy = w.vy;
    P.base.lam = df_from_double(Sp->lambda);
    const int64_t n2 = P.n2;
    const int gv = grid_for(M, n2, 256, 8);
    // alpha A^T f, once (the right-hand side keeps the exact back-projection
    // also with the surrogate, Eq. surr_SBupd); FP16 storage applies A^T as
    // Q^T (s .* f); the Fourier data term back-projects the data's DFTs
    CT_CHECK(backproject_data(M, P.vk, f, w, Sp->alpha, st));
    widen_kernel<<<gv, 256, 0, st>>>(u, w.u, M->g.n, M->tn);
    CT_CUDA(cudaGetLastError());
    CT_CUDA(cudaMemsetAsync(w.bx, 0, n2 * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.by, 0, n2 * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.vx, 0, n2 * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.vy, 0, n2 * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.sb, 0, sizeof(SbSlice), st));
    CT_CUDA(cudaMemcpyAsync(w.u_old, w.u, n2 * sizeof(float2), cudaMemcpyDeviceToDevice, st));

    *out = R.release();
    return CT_OK;
}

int sb1_update(Sb1Run* r, cudaStream_t s) { return enqueue_sb_outer(r->P, r->Sp, s); }

int sb1_finish(Sb1Run* r, float* u, ct_sb_stats* stats, cudaStream_t st)
{
    ct_matrix* M = r->M;
    Workspace& w = *r->P.w;
    const int gv = grid_for(M, r->P.n2, 256, 8);
    narrow_kernel<<<gv, 256, 0, st>>>(w.u, u, M->g.n, M->tn);
    CT_CUDA(cudaGetLastError());
    if (stats) {
        SbSlice h;
        CT_CUDA(cudaMemcpyAsync(&h, w.sb, sizeof(h), cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaStreamSynchronize(st));
        stats->outer_done = h.outer_done;
        stats->first_update_l1 = h.first_upd;
        stats->last_update_l1 = h.last_upd;
        stats->status = h.status;
        if (stats->status != CT_OK) return fail(stats->status, "split Bregman inner solve failed");
    }
    return CT_OK;
}

int run_updates(const std::vector<UpdateFn>& fns, const std::vector<cudaStream_t>& caps, int outer_iters,
                cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CT_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone || outer_iters <= 2) {
        for (int k = 0; k < outer_iters; ++k)
            for (const UpdateFn& f : fns) CT_CHECK(f(st));
        return CT_OK;
    }
    const int nr = (int)fns.size();
    std::vector<cudaEvent_t> ev(nr, nullptr);
    auto destroy_events = [&]() {
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
    };
    for (int i = 0; i < nr; ++i) {
        const cudaError_t e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            destroy_events();
            return cuda_fail(e, "cudaEventCreateWithFlags", __FILE__, __LINE__);
        }
    }
    cudaStream_t origin = caps[0];
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        destroy_events();
        return cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
    }
    // fork every further run onto its own capture stream, join them back
    int rc = CT_OK;
    if (nr > 1) e = cudaEventRecord(ev[0], origin);
    for (int i = 1; i < nr && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(caps[i], ev[0], 0);
    for (int i = 0; i < nr && e == cudaSuccess && rc == CT_OK; ++i) rc = fns[i](caps[i]);
    for (int i = 1; i < nr && e == cudaSuccess && rc == CT_OK; ++i) {
        e = cudaEventRecord(ev[i], caps[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ev[i], 0);
    }
    const cudaError_t e_end = cudaStreamEndCapture(origin, &graph);
    if (rc != CT_OK || e != cudaSuccess || e_end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        destroy_events();
        if (rc != CT_OK) return rc;
        return cuda_fail(e != cudaSuccess ? e : e_end, "graph capture of a Bregman update", __FILE__, __LINE__);
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    destroy_events();
    CT_CUDA(e);
    for (int k = 0; k < outer_iters; ++k) {
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) break;
    }
    cudaGraphExecDestroy(exec);
    CT_CUDA(e);
    return CT_OK;
}

int split_bregman(ct_matrix* M, const ct_sb_params* Sp, const float* f, float* u, int32_t batch,
                  ct_sb_stats* stats, cudaStream_t st)
{
    if (!(Sp->lambda > 0.0) || Sp->outer_iters < 0 || Sp->inner_cg_iters < 0 || !(Sp->cg_rel_tol >= 0.0))
        return fail(CT_ERR_ARG, "split Bregman needs lambda > 0, non-negative iteration counts and cg_rel_tol >= 0");
    if (batch != 1 && M->fourier) return fail(CT_ERR_UNSUPPORTED, "the Fourier operator solves one slice per call");
    if (batch != 1) return split_bregman_batched(M, Sp, f, u, batch, stats, st);
    Sb1Run* r = nullptr;
    CT_CHECK(sb1_prepare(M, M->ws, Sp, f, u, &r, st));
    std::unique_ptr<Sb1Run> hold(r);
    CT_CHECK(run_updates({[r](cudaStream_t s) { return sb1_update(r, s); }}, {M->ws.cap_stream}, Sp->outer_iters,
                         st));
    return sb1_finish(r, u, stats, st);
}

int chambolle_pock(ct_matrix* M, const ct_cp_params* Cp, const float* g, float* u, int32_t batch,
                   ct_sb_stats* stats, cudaStream_t st)
{
    if (!(Cp->tau > 0.0) || !(Cp->sigma > 0.0) || !(Cp->alpha >= 0.0) || !(Cp->theta >= 0.0 && Cp->theta <= 1.0) ||
        Cp->outer_iters < 0 || Cp->inner_cg_iters < 0)
        return fail(CT_ERR_ARG, "Chambolle-Pock needs tau, sigma > 0, alpha >= 0, theta in [0, 1] and "
                                "non-negative iteration counts");
    if (batch != 1) return fail(CT_ERR_UNSUPPORTED, "ct_chambolle_pock solves one slice per call (batch 1)");
    CT_CHECK(tune_single(M, st));
    CT_CHECK(ensure_workspace(M, 1, true));
    Workspace& w = M->ws;
    Plan P;
    const double ta = Cp->tau * Cp->alpha;
    CT_CHECK(make_plan(M, &w, 1.0, ta, 0.0, 0.0, 0, 0, 0, P));
    P.base.gate = &w.sb->stopped;
    const int64_t n2 = P.n2;
    const int gv = grid_for(M, n2, 256, 8);
    // tau alpha A^T g once; FP16 storage applies A^T as Q^T (s .* g)
    CT_CHECK(backproject_data(M, P.vk, g, w, ta, st));
    widen_kernel<<<gv, 256, 0, st>>>(u, w.u, M->g.n, M->tn);
    CT_CUDA(cudaGetLastError());
    // ubar (vx) = u; dual (bx, by) = 0
    CT_CUDA(cudaMemcpyAsync(w.vx, w.u, n2 * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    CT_CUDA(cudaMemsetAsync(w.bx, 0, n2 * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.by, 0, n2 * sizeof(float2), st));
    CT_CUDA(cudaMemsetAsync(w.sb, 0, sizeof(SbSlice), st));
    const float2 sigma = df_from_double(Cp->sigma), ntau = df_from_double(-Cp->tau),
                 theta = df_from_double(Cp->theta);
    const int n = M->g.n, tn = M->tn, inner = Cp->inner_cg_iters;
    auto update = [&](cudaStream_t s) -> int {
        cp_dual_kernel<<<gv, 256, 0, s>>>(w.vx, w.bx, w.by, n, tn, sigma, w.sb);
        CT_CUDA(cudaGetLastError());
        cp_rhs_kernel<<<gv, 256, 0, s>>>(w.u, w.bx, w.by, w.atf, w.rhs, w.u_old, n, tn, ntau, w.sb);
        CT_CUDA(cudaGetLastError());
        CT_CHECK(enqueue_cg(P, w.rhs, inner, s));
        cp_extrap_kernel<<<gv, 256, 0, s>>>(w.u, w.u_old, w.vx, n, tn, theta, w.sb, w.cg, w.partials, w.counter);
        CT_CUDA(cudaGetLastError());
        return CT_OK;
    };
    CT_CHECK(run_updates({update}, {w.cap_stream}, Cp->outer_iters, st));
    narrow_kernel<<<gv, 256, 0, st>>>(w.u, u, n, tn);
    CT_CUDA(cudaGetLastError());
    if (stats) {
        SbSlice h;
        CT_CUDA(cudaMemcpyAsync(&h, w.sb, sizeof(h), cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaStreamSynchronize(st));
        stats->outer_done = h.outer_done;
        stats->first_update_l1 = h.first_upd;
        stats->last_update_l1 = h.last_upd;
        stats->status = h.status;
        if (stats->status != CT_OK) return fail(stats->status, "Chambolle-Pock resolvent solve failed");
    }
    return CT_OK;
}

}  // namespace ct
