// extern "C" entry points of libct (declared and documented in include/ct.h).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ct_internal.cuh"

namespace ct {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line)
{
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_last_error = buf;
    return e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA;
}

namespace {

// 1 = device (or managed) memory, 0 = host memory.
int is_device_ptr(const void* p)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_handle(ct_matrix_t A)
{
    if (!A) return fail(CT_ERR_ARG, "NULL matrix handle");
    int dev = -1;
    CT_CUDA(cudaGetDevice(&dev));
    if (dev != A->device)
        return fail(CT_ERR_ARG, "matrix lives on device " + std::to_string(A->device) +
                                    " but device " + std::to_string(dev) + " is current");
    return CT_OK;
}

// Calls that need the Siddon matrices reject ct_build_fourier handles.
int no_fourier(ct_matrix_t A, const char* what)
{
    if (A->fourier)
        return fail(CT_ERR_UNSUPPORTED, std::string(what) + " is not available for a Fourier-operator handle");
    return CT_OK;
}

// Classifies the vector arguments: all device (0) or all host (1).
int classify(const void* a, const void* b, int* host)
{
    if (!a || !b) return fail(CT_ERR_ARG, "NULL vector pointer");
    const int da = is_device_ptr(a), db = is_device_ptr(b);
    if (da != db) return fail(CT_ERR_ARG, "mixing host and device vector pointers in one call");
    *host = !da;
    return CT_OK;
}

int ensure_stage(float** buf, int64_t* len, int64_t need)
{
    if (*len >= need) return CT_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *len = 0;
    cudaError_t e = cudaMalloc((void**)buf, (size_t)need * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(staging)", __FILE__, __LINE__);
    *len = need;
    return CT_OK;
}

ValKind storage_kind(const ct_matrix* M)
{
    return (M->flags & CT_VAL_FP16_ROWSCALE) ? ValKind::F16 : ValKind::F32;
}

}  // namespace
}  // namespace ct

using namespace ct;

extern "C" {

int ct_build_matrix(const ct_geometry* g, uint32_t flags, ct_matrix_t* out)
{
    if (!out) return fail(CT_ERR_ARG, "NULL output handle pointer");
    *out = nullptr;
    if (!g) return fail(CT_ERR_ARG, "NULL geometry");
    if (g->n <= 0 || g->n_angles_total <= 0 || g->keep_every <= 0 || g->n_bins <= 0)
        return fail(CT_ERR_ARG, "geometry sizes must be positive");
    if ((int64_t)g->n * g->n >= ((int64_t)1 << 31) || padded_pixels(g->n) >= ((int64_t)1 << 31))
        return fail(CT_ERR_ARG, "N*N (padded to whole 16 x 16 tiles) must be below 2^31");
    const int64_t n_kept = (g->n_angles_total + g->keep_every - 1) / g->keep_every;
    if (n_kept * g->n_bins >= ((int64_t)1 << 31))
        return fail(CT_ERR_ARG, "kept angles * bins must be below 2^31");
    const uint32_t known = CT_VAL_FP16_ROWSCALE | CT_KEEP_FP32_COPY | CT_F64_FP64_PIPE;
    if (flags & ~known) return fail(CT_ERR_ARG, "unknown flag bits");
    if ((flags & CT_KEEP_FP32_COPY) && !(flags & CT_VAL_FP16_ROWSCALE))
        return fail(CT_ERR_ARG, "CT_KEEP_FP32_COPY needs CT_VAL_FP16_ROWSCALE");
    ct_matrix* M = new (std::nothrow) ct_matrix();
    if (!M) return fail(CT_ERR_OOM, "host allocation failed");
    M->g = *g;
    M->flags = flags;
    cudaError_t e = cudaGetDevice(&M->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&M->sm_count, cudaDevAttrMultiProcessorCount, M->device);
    if (e != cudaSuccess) {
        delete M;
        return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    }
    int rc = build_matrices(M);
    if (rc != CT_OK) {
        ct_destroy_matrix(M);
        return rc;
    }
    noalloc_reserve();  // commit ct_cg_solve_noalloc's scratch while allocating is allowed
    *out = M;
    return CT_OK;
}

int ct_build_fourier(const ct_geometry* g, const ct_fourier_params* params, ct_matrix_t* out)
{
    if (!out) return fail(CT_ERR_ARG, "NULL output handle pointer");
    *out = nullptr;
    if (!g || !params) return fail(CT_ERR_ARG, "NULL geometry or params");
    if (g->n <= 0 || g->n_angles_total <= 0 || g->keep_every <= 0 || g->n_bins <= 0)
        return fail(CT_ERR_ARG, "geometry sizes must be positive");
    const int64_t n_kept = (g->n_angles_total + g->keep_every - 1) / g->keep_every;
    if (n_kept * g->n_bins >= ((int64_t)1 << 31)) return fail(CT_ERR_ARG, "kept angles * bins must be below 2^31");
    CT_CHECK(check_fourier_params(*g, *params));
    ct_matrix* M = new (std::nothrow) ct_matrix();
    if (!M) return fail(CT_ERR_OOM, "host allocation failed");
    M->g = *g;
    M->flags = 0;
    cudaError_t e = cudaGetDevice(&M->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&M->sm_count, cudaDevAttrMultiProcessorCount, M->device);
    if (e != cudaSuccess) {
        delete M;
        return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    }
    int rc = build_fourier(M, params);
    if (rc != CT_OK) {
        ct_destroy_matrix(M);
        return rc;
    }
    noalloc_reserve();  // commit ct_cg_solve_noalloc's scratch while allocating is allowed
    *out = M;
    return CT_OK;
}

int ct_matrix_info(ct_matrix_t A, int64_t* rows, int64_t* cols, int64_t* nnz)
{
    if (!A) return fail(CT_ERR_ARG, "NULL matrix handle");
    if (rows) *rows = A->rows;
    if (cols) *cols = A->cols;
    if (nnz) *nnz = A->fourier ? fourier_stored_weights(A) : A->A.nnz;
    return CT_OK;
}

void ct_destroy_matrix(ct_matrix_t A)
{
    if (!A) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != A->device) cudaSetDevice(A->device);
    cudaDeviceSynchronize();
    free_workspace(A->ws);
    for (auto& w : A->ws_pool) free_workspace(*w);
    for (auto& kv : A->stencils) free_stencil(kv.second);
    free_fourier(A);
    free_sell(A->A);
    free_sell(A->At);
    cudaFree(A->row_scale);
    cudaFree(A->dirs);
    cudaFree(A->band_lo);
    cudaFree(A->band_off);
    cudaFree(A->band_chunk);
    cudaFree(A->band_angle);
    if (prev >= 0 && prev != A->device) cudaSetDevice(prev);
    delete A;
}

int ct_forward(ct_matrix_t A, const float* x, float* y, int32_t batch, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_forward"));
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    int host = 0;
    CT_CHECK(classify(x, y, &host));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const ValKind vk = storage_kind(A);
    if (!host) return launch_forward(A, vk, x, y, batch, st);
    Workspace& w = A->ws;
    const int64_t nx = A->cols * batch, ny = A->rows * batch;
    CT_CHECK(ensure_stage(&w.stage_a, &w.stage_a_len, nx));
    CT_CHECK(ensure_stage(&w.stage_b, &w.stage_b_len, ny));
    CT_CUDA(cudaMemcpyAsync(w.stage_a, x, nx * sizeof(float), cudaMemcpyHostToDevice, st));
    CT_CHECK(launch_forward(A, vk, w.stage_a, w.stage_b, batch, st));
    CT_CUDA(cudaMemcpyAsync(y, w.stage_b, ny * sizeof(float), cudaMemcpyDeviceToHost, st));
    CT_CUDA(cudaStreamSynchronize(st));
    return CT_OK;
}

int ct_adjoint(ct_matrix_t A, const float* y, float* x, int32_t batch, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_adjoint"));
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    int host = 0;
    CT_CHECK(classify(y, x, &host));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const ValKind vk = storage_kind(A);
    if (!host) return launch_adjoint(A, vk, y, x, batch, st);
    Workspace& w = A->ws;
    const int64_t nx = A->cols * batch, ny = A->rows * batch;
    CT_CHECK(ensure_stage(&w.stage_a, &w.stage_a_len, nx));
    CT_CHECK(ensure_stage(&w.stage_b, &w.stage_b_len, ny));
    CT_CUDA(cudaMemcpyAsync(w.stage_b, y, ny * sizeof(float), cudaMemcpyHostToDevice, st));
    CT_CHECK(launch_adjoint(A, vk, w.stage_b, w.stage_a, batch, st));
    CT_CUDA(cudaMemcpyAsync(x, w.stage_a, nx * sizeof(float), cudaMemcpyDeviceToHost, st));
    CT_CUDA(cudaStreamSynchronize(st));
    return CT_OK;
}

int ct_forward_f64(ct_matrix_t A, const double* x, double* y, int32_t batch, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_forward_f64"));
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    int host = 0;
    CT_CHECK(classify(x, y, &host));
    if (host) return fail(CT_ERR_ARG, "ct_forward_f64 needs device pointers");
    return launch_forward_f64(A, storage_kind(A), x, y, batch, (cudaStream_t)cuda_stream);
}

int ct_adjoint_f64(ct_matrix_t A, const double* y, double* x, int32_t batch, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_adjoint_f64"));
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    int host = 0;
    CT_CHECK(classify(y, x, &host));
    if (host) return fail(CT_ERR_ARG, "ct_adjoint_f64 needs device pointers");
    return launch_adjoint_f64(A, storage_kind(A), y, x, batch, (cudaStream_t)cuda_stream);
}

int ct_normal_f64(ct_matrix_t A, double alpha, double lambda, const double* x, double* out, int32_t batch,
                  void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_normal_f64"));
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    if (!x || !out || !is_device_ptr(x) || !is_device_ptr(out))
        return fail(CT_ERR_ARG, "ct_normal_f64 needs device pointers");
    if (x == out) return fail(CT_ERR_ARG, "ct_normal_f64 cannot work in place");
    return normal_f64(A, alpha, lambda, x, out, batch, (cudaStream_t)cuda_stream);
}

int ct_cg_solve(ct_matrix_t A, const ct_cg_params* params, const float* rhs, float* u,
                int32_t batch, ct_cg_stats* stats, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    if (!params) return fail(CT_ERR_ARG, "NULL params");
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    int host = 0;
    CT_CHECK(classify(rhs, u, &host));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!host) return cg_solve(A, params, rhs, u, batch, stats, st);
    Workspace& w = A->ws;
    const int64_t nx = A->cols * batch;
    CT_CHECK(ensure_stage(&w.stage_a, &w.stage_a_len, nx));
    CT_CHECK(ensure_stage(&w.stage_b, &w.stage_b_len, nx));
    CT_CUDA(cudaMemcpyAsync(w.stage_a, rhs, nx * sizeof(float), cudaMemcpyHostToDevice, st));
    CT_CUDA(cudaMemcpyAsync(w.stage_b, u, nx * sizeof(float), cudaMemcpyHostToDevice, st));
    int rc = cg_solve(A, params, w.stage_a, w.stage_b, batch, stats, st);
    if (rc != CT_OK && rc != CT_ERR_BREAKDOWN && rc != CT_ERR_NONFINITE) return rc;
    CT_CUDA(cudaMemcpyAsync(u, w.stage_b, nx * sizeof(float), cudaMemcpyDeviceToHost, st));
    CT_CUDA(cudaStreamSynchronize(st));
    return rc;
}

int ct_split_bregman(ct_matrix_t A, const ct_sb_params* params, const float* f, float* u,
                     int32_t batch, ct_sb_stats* stats, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    if (!params) return fail(CT_ERR_ARG, "NULL params");
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    int host = 0;
    CT_CHECK(classify(f, u, &host));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!host) return split_bregman(A, params, f, u, batch, stats, st);
    Workspace& w = A->ws;
    const int64_t nx = A->cols * batch, ny = A->rows * batch;
    CT_CHECK(ensure_stage(&w.stage_a, &w.stage_a_len, nx));
    CT_CHECK(ensure_stage(&w.stage_b, &w.stage_b_len, ny));
    CT_CUDA(cudaMemcpyAsync(w.stage_b, f, ny * sizeof(float), cudaMemcpyHostToDevice, st));
    CT_CUDA(cudaMemcpyAsync(w.stage_a, u, nx * sizeof(float), cudaMemcpyHostToDevice, st));
    int rc = split_bregman(A, params, w.stage_b, w.stage_a, batch, stats, st);
    if (rc != CT_OK && rc != CT_ERR_BREAKDOWN && rc != CT_ERR_NONFINITE) return rc;
    CT_CUDA(cudaMemcpyAsync(u, w.stage_a, nx * sizeof(float), cudaMemcpyDeviceToHost, st));
    CT_CUDA(cudaStreamSynchronize(st));
    return rc;
}

int ct_chambolle_pock(ct_matrix_t A, const ct_cp_params* params, const float* g, float* u, int32_t batch,
                      ct_sb_stats* stats, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    if (!params) return fail(CT_ERR_ARG, "NULL params");
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    int host = 0;
    CT_CHECK(classify(g, u, &host));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!host) return chambolle_pock(A, params, g, u, batch, stats, st);
    Workspace& w = A->ws;
    const int64_t nx = A->cols * batch, ny = A->rows * batch;
    CT_CHECK(ensure_stage(&w.stage_a, &w.stage_a_len, nx));
    CT_CHECK(ensure_stage(&w.stage_b, &w.stage_b_len, ny));
    CT_CUDA(cudaMemcpyAsync(w.stage_b, g, ny * sizeof(float), cudaMemcpyHostToDevice, st));
    CT_CUDA(cudaMemcpyAsync(w.stage_a, u, nx * sizeof(float), cudaMemcpyHostToDevice, st));
    int rc = chambolle_pock(A, params, w.stage_b, w.stage_a, batch, stats, st);
    if (rc != CT_OK && rc != CT_ERR_BREAKDOWN && rc != CT_ERR_NONFINITE) return rc;
    CT_CUDA(cudaMemcpyAsync(u, w.stage_a, nx * sizeof(float), cudaMemcpyDeviceToHost, st));
    CT_CUDA(cudaStreamSynchronize(st));
    return rc;
}

int ct_split_bregman_ragged(int32_t count, const ct_matrix_t* A, const float* const* f, float* const* u,
                            const ct_sb_params* params, ct_sb_stats* stats, void* cuda_stream)
{
    if (count < 1) return fail(CT_ERR_ARG, "count must be >= 1");
    if (!A || !f || !u) return fail(CT_ERR_ARG, "NULL array of handles or vector pointers");
    if (!params) return fail(CT_ERR_ARG, "NULL params");
    if (!(params->lambda > 0.0) || params->outer_iters < 0 || params->inner_cg_iters < 0 || !(params->cg_rel_tol >= 0.0))
        return fail(CT_ERR_ARG, "split Bregman needs lambda > 0, non-negative iteration counts and cg_rel_tol >= 0");
    for (int32_t i = 0; i < count; ++i) {
        CT_CHECK(check_handle(A[i]));
        CT_CHECK(no_fourier(A[i], "ct_split_bregman_ragged"));
        if (!f[i] || !u[i]) return fail(CT_ERR_ARG, "NULL vector pointer for problem " + std::to_string(i));
        if (!is_device_ptr(f[i]) || !is_device_ptr(u[i]))
            return fail(CT_ERR_ARG, "ct_split_bregman_ragged needs device pointers (problem " + std::to_string(i) + ")");
    }
    return split_bregman_ragged(count, A, f, u, params, stats, (cudaStream_t)cuda_stream);
}

int ct_get_tuning(ct_matrix_t A, int32_t batch, ct_tuning* t)
{
    CT_CHECK(check_handle(A));
    if (!t) return fail(CT_ERR_ARG, "NULL output pointer");
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    std::memset(t, 0, sizeof(*t));
    if (batch == 1) {
        t->fwd_warps = A->fwd_warps;
        t->fwd_unroll = A->fwd_unroll;
        t->op_ctas = A->op_ctas;
        t->op_pixels = A->op_pixels;
    } else {
        auto it = A->spmm_unroll.find(batch);
        t->spmm_unroll = it == A->spmm_unroll.end() ? 0 : it->second;
    }
    return CT_OK;
}

int ct_set_tuning(ct_matrix_t A, int32_t batch, const ct_tuning* t)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_set_tuning"));
    if (!t) return fail(CT_ERR_ARG, "NULL tuning");
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    if (batch == 1) {
        const bool chunked = A->h_band_chunk.size() > 2;
        if (t->fwd_warps != 0 && t->fwd_warps != 4 && t->fwd_warps != 8)
            return fail(CT_ERR_ARG, "fwd_warps must be 0, 4 or 8");
        if (t->fwd_unroll != 0 && t->fwd_unroll != 2 && t->fwd_unroll != 4 && t->fwd_unroll != 8 &&
            t->fwd_unroll != 16)
            return fail(CT_ERR_ARG, "fwd_unroll must be 0, 2, 4, 8 or 16");
        if (t->op_ctas != 0 && t->op_ctas != (chunked ? 5 : 7) && t->op_ctas != (chunked ? 3 : 4) &&
            (chunked || t->op_ctas != 3))
            return fail(CT_ERR_ARG, chunked ? "op_ctas must be 0, 5 or 3 for this matrix (band staged in chunks)"
                                            : "op_ctas must be 0, 7, 4 or 3 for this matrix");
        if (t->op_pixels != 0 && t->op_pixels != 1 && t->op_pixels != 2)
            return fail(CT_ERR_ARG, "op_pixels must be 0, 1 or 2");
        if (t->op_pixels == 2 && (chunked || (t->op_ctas != 0 && t->op_ctas != 7)))
            return fail(CT_ERR_ARG, "op_pixels = 2 needs a single-chunk band and op_ctas 0 or 7");
        if (t->spmm_unroll != 0) return fail(CT_ERR_ARG, "spmm_unroll applies to batches of 2 or more");
        A->fwd_warps = t->fwd_warps;
        A->fwd_unroll = t->fwd_unroll;
        A->op_ctas = t->op_ctas;
        A->op_pixels = t->op_pixels;
        return CT_OK;
    }
    if (t->fwd_warps || t->fwd_unroll || t->op_ctas || t->op_pixels)
        return fail(CT_ERR_ARG, "fwd_warps, fwd_unroll, op_ctas and op_pixels apply to batch 1");
    return ct_set_spmm_unroll(A, batch, t->spmm_unroll);
}

int ct_tune(ct_matrix_t A, int32_t batch, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_tune"));
    if (batch < 1) return fail(CT_ERR_ARG, "batch must be >= 1");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (batch == 1) return tune_single(A, st);
    return tune_batched(A, batch, st);
}

int ct_time_cg_kernels(ct_matrix_t A, double c_ata, double c_grad, int32_t reps, double* ms, void* cuda_stream)
{
    CT_CHECK(check_handle(A));
    if (!ms) return fail(CT_ERR_ARG, "NULL output array");
    CT_CHECK(no_fourier(A, "ct_time_cg_kernels"));
    return time_cg_kernels(A, c_ata, c_grad, reps, ms, (cudaStream_t)cuda_stream);
}

int ct_set_wait_limit(int64_t polls, int32_t hold_first)
{
    set_wait_limit((long long)polls, hold_first);
    return CT_OK;
}

int ct_set_spmm_unroll(ct_matrix_t A, int32_t batch, int32_t unroll)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_set_spmm_unroll"));
    if (batch < 2) return fail(CT_ERR_ARG, "batch must be >= 2 (batch 1 does not use the batched products)");
    if (unroll != 0 && unroll != 4 && unroll != 8 && unroll != 16)
        return fail(CT_ERR_ARG, "unroll must be 0, 4, 8 or 16");
    if (unroll == 0)
        A->spmm_unroll.erase(batch);
    else
        A->spmm_unroll[batch] = unroll;
    return CT_OK;
}

int ct_get_spmm_unroll(ct_matrix_t A, int32_t batch, int32_t* unroll)
{
    CT_CHECK(check_handle(A));
    if (!unroll) return fail(CT_ERR_ARG, "NULL output pointer");
    auto it = A->spmm_unroll.find(batch);
    *unroll = it == A->spmm_unroll.end() ? 0 : it->second;
    return CT_OK;
}

int ct_matrix_export(ct_matrix_t A, int32_t which, int64_t* row_ptr, int32_t* cols, float* vals)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_matrix_export"));
    if (which != 0 && which != 1) return fail(CT_ERR_ARG, "which must be 0 (A) or 1 (A^T)");
    if (!row_ptr || !cols || !vals) return fail(CT_ERR_ARG, "NULL output array");
    const Sell& C = which == 0 ? A->A : A->At;
    const int n = A->g.n, tn = A->tn, nb = A->g.n_bins, nk = A->n_kept;
    std::vector<int64_t> sp((C.rows + kSliceRows - 1) / kSliceRows + 1);
    std::vector<int32_t> len(C.rows), col;
    std::vector<uint16_t> col16;
    std::vector<float> val(C.nnz_pad);
    std::vector<uint16_t> q;
    std::vector<float> s;
    CT_CUDA(cudaMemcpy(sp.data(), C.slice_ptr, sp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(len.data(), C.row_len, len.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (which == 0) {
        col.resize(C.nnz_pad);
        CT_CUDA(cudaMemcpy(col.data(), C.col, col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    } else {
        col16.resize(C.nnz_pad);
        CT_CUDA(cudaMemcpy(col16.data(), C.col16, col16.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    }
    const bool f16 = (A->flags & CT_VAL_FP16_ROWSCALE) != 0;
    if (f16) {
        q.resize(C.nnz_pad);
        s.resize(A->rows);
        CT_CUDA(cudaMemcpy(q.data(), C.qval, q.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost));
        CT_CUDA(cudaMemcpy(s.data(), A->row_scale, s.size() * sizeof(float), cudaMemcpyDeviceToHost));
    } else {
        CT_CUDA(cudaMemcpy(val.data(), C.val, val.size() * sizeof(float), cudaMemcpyDeviceToHost));
    }
    auto value = [&](int64_t k, int64_t ray) -> float {
        if (!f16) return val[k];
        __half_raw hr;
        hr.x = q[k];
        return __half2float(__half(hr)) * s[ray];
    };
    int64_t o = 0;
    row_ptr[0] = 0;
    if (which == 0) {
        // entries are stored in row-major pixel order; columns are tile-order indices
        for (int64_t r = 0; r < C.rows; ++r) {
            for (int64_t e = 0; e < len[r]; ++e, ++o) {
                const int64_t k = sell_pos(sp.data(), r, e);
                int i, j;
                tiled_coords(col[k], tn, i, j);
                cols[o] = i * n + j;
                vals[o] = value(k, r);
            }
            row_ptr[r + 1] = o;
        }
        return CT_OK;
    }
    // A^T: rows in tile order, columns band-local; emit by row-major pixel
    std::vector<int64_t> row_of((size_t)n * n, -1);
    for (int64_t t = 0; t < C.rows; ++t) {
        int i, j;
        tiled_coords(t, tn, i, j);
        if (i < n && j < n) row_of[(size_t)i * n + j] = t;
    }
    for (int64_t p = 0; p < (int64_t)n * n; ++p) {
        const int64_t t = row_of[p];
        for (int64_t e = 0; e < len[t]; ++e, ++o) {
            const int64_t k = sell_pos(sp.data(), t, e);
            const int c = col16[k];
            const int a = A->h_band_angle[c];
            const int64_t ray =
                (int64_t)a * nb + A->h_band_lo[(size_t)(t >> 8) * nk + a] + (c - A->h_band_off[a]);
            cols[o] = (int32_t)ray;
            vals[o] = value(k, ray);
        }
        row_ptr[p + 1] = o;
    }
    return CT_OK;
}

int ct_matrix_export_fp16(ct_matrix_t A, uint16_t* q_bits, float* scale)
{
    CT_CHECK(check_handle(A));
    CT_CHECK(no_fourier(A, "ct_matrix_export_fp16"));
    if (!(A->flags & CT_VAL_FP16_ROWSCALE)) return fail(CT_ERR_UNSUPPORTED, "matrix has no FP16 storage");
    if (!q_bits || !scale) return fail(CT_ERR_ARG, "NULL output array");
    const Sell& C = A->A;
    std::vector<int64_t> sp((C.rows + kSliceRows - 1) / kSliceRows + 1);
    std::vector<int32_t> len(C.rows);
    std::vector<uint16_t> q(C.nnz_pad);
    CT_CUDA(cudaMemcpy(sp.data(), C.slice_ptr, sp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(len.data(), C.row_len, len.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(q.data(), C.qval, q.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(scale, A->row_scale, A->rows * sizeof(float), cudaMemcpyDeviceToHost));
    int64_t o = 0;
    for (int64_t r = 0; r < C.rows; ++r)
        for (int64_t e = 0; e < len[r]; ++e) q_bits[o++] = q[sell_pos(sp.data(), r, e)];
    return CT_OK;
}

int ct_surrogate_stencil(ct_matrix_t A, int32_t r, int32_t square, int32_t capacity, int32_t* di,
                         int32_t* dj, double* val, int32_t* count)
{
    CT_CHECK(check_handle(A));
    if (!count) return fail(CT_ERR_ARG, "NULL count");
    Stencil* S = nullptr;
    CT_CHECK(make_stencil(A, r, square, &S));
    *count = S->ntaps;
    if (capacity < S->ntaps) return fail(CT_ERR_ARG, "capacity below the number of taps");
    if (!di || !dj || !val) return fail(CT_ERR_ARG, "NULL output array");
    for (int t = 0; t < S->ntaps; ++t) {
        di[t] = S->h_di[t];
        dj[t] = S->h_dj[t];
        val[t] = S->h_w[t];
    }
    return CT_OK;
}

// Fourier-operator products: device pointers only, complex samples
// interleaved (8-byte aligned).
static int fourier_args(ct_matrix_t F, const void* a, const void* b, const void* complex_arg)
{
    CT_CHECK(check_handle(F));
    if (!F->fourier) return fail(CT_ERR_UNSUPPORTED, "not a Fourier-operator handle (ct_build_fourier)");
    if (!a || !b) return fail(CT_ERR_ARG, "NULL vector pointer");
    if (!is_device_ptr(a) || !is_device_ptr(b)) return fail(CT_ERR_ARG, "the Fourier products need device pointers");
    if (complex_arg && reinterpret_cast<uintptr_t>(complex_arg) % 8 != 0)
        return fail(CT_ERR_ARG, "complex sample arrays must be 8-byte aligned");
    return CT_OK;
}

int ct_fourier_forward(ct_matrix_t F, const float* x, float* y, void* cuda_stream)
{
    CT_CHECK(fourier_args(F, x, y, y));
    return fourier_forward(F, x, y, (cudaStream_t)cuda_stream);
}

int ct_fourier_adjoint(ct_matrix_t F, const float* y, float* x, void* cuda_stream)
{
    CT_CHECK(fourier_args(F, y, x, y));
    return fourier_adjoint(F, y, x, (cudaStream_t)cuda_stream);
}

int ct_fourier_normal(ct_matrix_t F, const float* x, float* out, void* cuda_stream)
{
    CT_CHECK(fourier_args(F, x, out, nullptr));
    return fourier_normal(F, x, out, (cudaStream_t)cuda_stream);
}

int ct_fourier_data(ct_matrix_t F, const float* f, float* fhat, void* cuda_stream)
{
    CT_CHECK(fourier_args(F, f, fhat, fhat));
    return fourier_data(F, f, fhat, (cudaStream_t)cuda_stream);
}

const char* ct_status_string(int status)
{
    switch (status) {
    case CT_OK: return "ok";
    case CT_ERR_ARG: return "invalid argument";
    case CT_ERR_CUDA: return "CUDA error";
    case CT_ERR_OOM: return "out of memory";
    case CT_ERR_BREAKDOWN: return "CG breakdown (operator not positive definite)";
    case CT_ERR_NONFINITE: return "non-finite value";
    case CT_ERR_TIMEOUT: return "device wait timed out";
    case CT_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
    }
}

const char* ct_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
