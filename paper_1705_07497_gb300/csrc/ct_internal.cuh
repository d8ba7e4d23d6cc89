// Internal declarations of libct (CUDA, sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "ct.h"
#include "dfloat.cuh"
#include "layout.cuh"

namespace ct {

// Rows of both CSR matrices are padded to a multiple of this many entries so
// that every row starts on a 16-byte boundary for int32/FP32 (and FP16) vector
// loads; padding entries repeat the row's last column with value 0.
constexpr int kSliceRows = 32;  // rows per SELL slice (one warp, one row per lane)
constexpr int kChunk = 8;       // entries per lane-contiguous chunk (16/32-byte loads)

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CT_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::ct::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define CT_CHECK(expr)                 \
    do {                               \
        int rc_ = (expr);              \
        if (rc_ != CT_OK) return rc_;  \
    } while (0)

// ---------------------------------------------------------------------------
// device data
// ---------------------------------------------------------------------------
// Sparse matrix in sliced-ELL form (SELL-32): rows are grouped in slices of
// 32 consecutive rows; slice s stores 32 * L_s entries, L_s = its longest row
// rounded up to kChunk, and entry j of row r sits at
//     slice_ptr[r / 32] + (j / 8) * 256 + (r % 32) * 8 + j % 8,
// so a warp with one row per lane reads 32 contiguous 8-entry chunks per step
// and a lane reads its own 8 entries with one vector load.  Entries past a
// row's length have value 0 and a valid column.
struct Sell {
    int64_t rows = 0, cols = 0;
    int64_t nnz = 0;       // stored nonzeros
    int64_t nnz_pad = 0;   // entries including padding
    int64_t* slice_ptr = nullptr;  // [ceil(rows/32)+1] slice offsets
    int32_t* row_len = nullptr;    // [rows] lengths
    int32_t* col = nullptr;      // [nnz_pad] column indices (A: internal pixel index)
    uint16_t* col16 = nullptr;   // [nnz_pad] A^T: local band index off_k + (b - band_lo)
    float* val = nullptr;        // [nnz_pad] FP32 values (may be null)
    __half* qval = nullptr;      // [nnz_pad] FP16 Q values (may be null)
};

__host__ __device__ inline int64_t sell_pos(const int64_t* slice_ptr, int64_t r, int64_t j)
{
    return slice_ptr[r >> 5] + ((j >> 3) << 8) + ((r & 31) << 3) + (j & 7);
}

// Per-slice conjugate-gradient scalars, resident on the device.
struct CgSlice {
    double rr;       // r.r of the current residual
    double rhs2;     // rhs.rhs
    double alpha;    // step of the current iteration
    double beta;     // rr_new / rr
    float2 alpha_df; // alpha and beta as double-float pairs for the vector kernels
    float2 beta_df;
    int32_t active;  // 1 while the slice keeps iterating
    int32_t iters;   // steps taken
    int32_t status;  // CT_OK / CT_ERR_BREAKDOWN / CT_ERR_NONFINITE
    int32_t pad;
};

// Per-slice split-Bregman scalars.
struct SbSlice {
    double first_upd;
    double last_upd;
    int32_t outer_done;
    int32_t stopped;
    int32_t status;
    int32_t pad;
};

struct Stencil {
    int ntaps = 0;
    int r = 0;
    int32_t* d = nullptr;  // device [ntaps][2] offsets (di, dj)
    float* w = nullptr;    // device [ntaps][2] taps as FP32 pairs (hi, lo)
    std::vector<int32_t> h_di, h_dj;
    std::vector<double> h_w;  // FP64 taps (host copy)
};

struct Workspace {
    int device = -1;
    int32_t batch = 0;
    int64_t n2 = 0, rows = 0;
    // Solver vectors ([len][batch]) are double-float pairs (hi, lo).
    float2 *u = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *rhs = nullptr;
    float2 *atf = nullptr, *u_old = nullptr, *bx = nullptr, *by = nullptr, *vx = nullptr, *vy = nullptr;
    float2* y = nullptr;                   // sinogram temp [rows][batch]
    double* f64_y = nullptr;               // ct_normal_f64: the sinogram temp [rows][batch]
    int64_t f64_y_len = 0;
    // FP64-vector products in double-float (the default): the split input,
    // the product, and (ct_normal_f64) the second product, [len][batch]
    float2 *f64_a = nullptr, *f64_b = nullptr, *f64_c = nullptr;
    int64_t f64_a_len = 0, f64_b_len = 0, f64_c_len = 0;
    float2* pub_y2 = nullptr;              // ct_adjoint with FP16 storage: s .* y
    int64_t pub_y2_len = 0;
    float* pub_x = nullptr;                // ct_forward: the caller's image in tile order
    int64_t pub_x_len = 0;
    float2* partials = nullptr;            // reduction partials
    int64_t partials_len = 0;
    unsigned* counter = nullptr;           // last-block counter (one per workspace)
    CgSlice* cg = nullptr;
    SbSlice* sb = nullptr;
    // staging for host pointers (FP32, caller layout)
    float *stage_a = nullptr, *stage_b = nullptr;
    int64_t stage_a_len = 0, stage_b_len = 0;
    cudaStream_t cap_stream = nullptr;
    // ct_split_bregman_ragged: per-slice f and u pointers of one group [2][cap]
    float** ragged_ptrs = nullptr;
    int32_t ragged_cap = 0;
};

struct FourierOp;  // fourier.cu: the Fourier-domain data term of a ct_build_fourier handle

}  // namespace ct

struct ct_matrix {
    ct_geometry g{};
    uint32_t flags = 0;
    int device = 0;
    int sm_count = 0;
    int n_kept = 0;
    int64_t rows = 0, cols = 0;
    int tn = 0;              // image tiles per side
    int64_t npad = 0;        // padded internal image length (tn * 16)^2
    int32_t* band_lo = nullptr;  // device [tn*tn][n_kept]: first bin of each (tile, angle) band
    int32_t* band_off = nullptr; // device [n_kept+1]: offset of each angle's slots in a band
    uint16_t* band_angle = nullptr;  // device [band_total]: kept angle of each band slot
    int band_total = 0;          // slots of one tile's band (sum of the angles' widths)
    int32_t* band_chunk = nullptr;  // device [nchunks+1]: first kept angle of each staged band chunk
    int band_chunk_slots = 0;       // slots of the largest chunk
    std::vector<int32_t> h_band_lo, h_band_off, h_band_chunk;
    std::vector<uint16_t> h_band_angle;
    double* dirs = nullptr;  // device [n_kept][2]: cos, sin
    std::vector<double> h_cos, h_sin;
    ct::Sell A, At;
    float* row_scale = nullptr;  // FP16 form: s [rows]
    std::map<std::pair<int, int>, ct::Stencil> stencils;
    std::map<int, int> spmm_unroll;  // batch size -> staged-entry unroll of the batched products (tuned or pinned)
    // launch shape of the single-slice products (0 = not chosen: the defaults)
    int fwd_warps = 0;       // y = A x: warps per block (4 or 8)
    int fwd_unroll = 0;      // y = A x: chunks in flight per lane (2, 4 or 8)
    int op_ctas = 0;         // A^T kernels: CTAs per SM the registers are sized for
    int op_pixels = 0;       // A^T kernels: pixel rows per lane (1, or 2 with four warps per tile)
    ct::Workspace ws;
    // extra single-slice workspaces: ct_split_bregman_ragged runs the
    // problems of a small group on one handle side by side
    std::vector<std::unique_ptr<ct::Workspace>> ws_pool;
    // ct_build_fourier handles: the data term is Re(F^H F) (no Siddon matrices)
    ct::FourierOp* fourier = nullptr;
};

namespace ct {

// build.cu
int build_matrices(ct_matrix* M);
// cos, sin of the kept angles (theta exactly 0 or pi/2 snapped), FP64
void angle_directions(const ct_geometry& g, std::vector<double>& c, std::vector<double>& s);
void free_sell(Sell& c);
int make_stencil(ct_matrix* M, int r, int square, Stencil** out);
void free_stencil(Stencil& s);

// workspace.cu (in solve.cu)
int ensure_workspace(ct_matrix* M, int32_t batch, bool solver);
int ensure_workspace_in(ct_matrix* M, Workspace& w, int32_t batch);
void free_workspace(Workspace& w);

// spmv.cu
enum class ValKind { F32 = 0, F16 = 1 };
int launch_forward(const ct_matrix* M, ValKind vk, const float* x, float* y, int32_t batch, cudaStream_t st);
int launch_adjoint(const ct_matrix* M, ValKind vk, const float* y, float* x, int32_t batch, cudaStream_t st);
int launch_forward_f64(const ct_matrix* M, ValKind vk, const double* x, double* y, int32_t batch, cudaStream_t st);
int launch_adjoint_f64(const ct_matrix* M, ValKind vk, const double* y, double* x, int32_t batch, cudaStream_t st);
// out = alpha A^T A x + lambda grad^T grad x in FP64 (row-major vectors)
int normal_f64(const ct_matrix* M, double alpha, double lam, const double* x, double* out, int32_t B,
               cudaStream_t st);

// Epilogue of the adjoint product inside the CG operator (double-float vectors).
struct OpEpilogue {
    int mode;             // 1: q = Op(p) and p.q; 2: r = rhs - Op(u), p = r (CG start);
                          // 3: r = rhs - Op(u) only (residual replacement)
    float2 c_id, c_ata, c_grad;  // coefficients as double-float pairs
    const float2* in;     // p (mode 1) or u (modes 2, 3)
    float2* out;          // q (mode 1) or r (modes 2, 3)
    float2* p_out;        // mode 2: p = r
    const float2* rhs;    // modes 2, 3: explicit rhs, or null to build atf + lambda grad^T v
    const float2* atf;    // SB: alpha A^T f
    const float2* vx;     // SB: v = d - b
    const float2* vy;
    float2 lam;
    const int32_t* gate;  // skip all work when *gate != 0 (stopped SB)
    CgSlice* cg;
    float2* partials;
    unsigned* counter;
    double tol;
};

// solver_ops.cu: products used inside the solvers (double-float accumulation)
// y = A x, rows scaled by s^rpow (FP16 storage), gated by cg->active / *gate.
int launch_forward_df(const ct_matrix* M, ValKind vk, const float2* x, float2* y, int rpow,
                      const CgSlice* cg, const int32_t* gate, cudaStream_t st);
// out = scale * A^T y.
int launch_adjoint_df(const ct_matrix* M, ValKind vk, const float2* y, float2* out, double scale,
                      cudaStream_t st);
// A^T y fused with the CG operator epilogue.
int launch_adjoint_op_df(const ct_matrix* M, ValKind vk, const float2* y, const OpEpilogue& ep,
                         cudaStream_t st);
// Surrogate stencil (or no sparse term at all when S is null) fused with the epilogue.
int launch_stencil_op_df(const ct_matrix* M, const Stencil* S, const OpEpilogue& ep, cudaStream_t st);
// Public single-slice products with FP32 vectors (same kernel template).
int launch_forward_f32(const ct_matrix* M, ValKind vk, const float* x, float* y, cudaStream_t st);
int launch_adjoint_f32(const ct_matrix* M, ValKind vk, const float* y, const float2* y_scaled, float* x,
                       cudaStream_t st);
// out = (in * scale, exactly as a double-float pair) for FP32 input (scale may be null).
int launch_to_df(const ct_matrix* M, const float* in, const float* scale, float2* out, int64_t len,
                 cudaStream_t st);

// solve.cu
// CG on a caller-prepared workspace view (u, r, p, q, rhs, y, partials,
// counter and cg must be set; the counter must be zero).
int cg_solve_in(ct_matrix* M, Workspace& w, const ct_cg_params* P, const float* rhs, float* u,
                ct_cg_stats* stats, cudaStream_t st);
int cg_solve(ct_matrix* M, const ct_cg_params* P, const float* rhs, float* u, int32_t batch,
             ct_cg_stats* stats, cudaStream_t st);
int split_bregman(ct_matrix* M, const ct_sb_params* P, const float* f, float* u, int32_t batch,
                  ct_sb_stats* stats, cudaStream_t st);
int time_cg_kernels(ct_matrix* M, double c_ata, double c_grad, int32_t reps, double* ms, cudaStream_t st);
// launch shape of the single-slice products (timed on the handle, cached by geometry)
int tune_single(ct_matrix* M, cudaStream_t st);
int tune_batched(ct_matrix* M, int32_t B, cudaStream_t st);

int grid_for(const ct_matrix* M, int64_t work_items, int items_per_block, int max_per_sm);

// batch.cu: many slices sharing one geometry (vectors [len][B])
// which = 0: y = A x; which = 1: x = A^T y (FP32 vectors, double-float accumulation).
int batched_forward_adjoint(const ct_matrix* M, int which, const float* in, float* out, int32_t B,
                            cudaStream_t st);
// Batched double-float products in the internal layouts ([npad][B] tiled
// images, [rows][B] sinograms): which = 0: out = s^rpow .* (A in) (rpow 0
// without FP16 storage); which = 1: out = A^T in (with FP16 storage Q^T in:
// the caller scales the sinogram).
int batched_product_df(const ct_matrix* M, int which, const float2* in, float2* out, int32_t B, int rpow,
                       cudaStream_t st);
int cg_solve_batched(ct_matrix* M, const ct_cg_params* P, const float* rhs, float* u, int32_t B,
                     ct_cg_stats* stats, cudaStream_t st);
// Bregman updates of one or more runs, outer_iters times: one captured graph
// with every run on its own capture stream caps[i] (forked from caps[0]),
// replayed on st; or directly on st when st is capturing or outer_iters <= 2.
using UpdateFn = std::function<int(cudaStream_t)>;
int run_updates(const std::vector<UpdateFn>& fns, const std::vector<cudaStream_t>& caps, int outer_iters,
                cudaStream_t st);
// single-slice split Bregman in phases (solve.cu)
struct Sb1Run;
int sb1_prepare(ct_matrix* M, Workspace& w, const ct_sb_params* Sp, const float* f, const float* u, Sb1Run** out,
                cudaStream_t st);
int sb1_update(Sb1Run* r, cudaStream_t s);
int sb1_finish(Sb1Run* r, float* u, ct_sb_stats* stats, cudaStream_t st);
void sb1_free(Sb1Run* r);
// What the persistent ragged-batch kernel (ragged.cu) takes from a prepared
// single-slice run: the operator's plan and the solver parameters.
struct Sb1Desc {
    ct_matrix* M;
    Workspace* w;
    OpEpilogue base;   // the plan's epilogue (coefficients, gate, data term, CG scalars)
    ValKind vk;
    bool exact;        // A^T A through the sparse products (no surrogate, no refresh)
    double gamma;      // shrink threshold 1 / lambda
    double stop_tol;   // Sec. 4 stopping rule
    int inner;         // CG steps per update
};
void sb1_describe(const Sb1Run* r, Sb1Desc* d);
// ragged.cu: every prepared single-slice run's updates as one persistent
// launch per update; *used = false when a run is outside its scope.
int ragged_persistent(const std::vector<Sb1Run*>& runs, int outer, cudaStream_t st, cudaStream_t cap, bool* used);
// bounded-wait limit (polls) of the persistent kernel and the held-dependency test switch
void set_wait_limit(long long polls, int hold);
int chambolle_pock(ct_matrix* M, const ct_cp_params* Cp, const float* g, float* u, int32_t batch,
                   ct_sb_stats* stats, cudaStream_t st);
int split_bregman_ragged(int32_t count, ct_matrix* const* A, const float* const* f, float* const* u,
                         const ct_sb_params* Sp, ct_sb_stats* stats, cudaStream_t st);
int split_bregman_batched(ct_matrix* M, const ct_sb_params* P, const float* f, float* u, int32_t B,
                          ct_sb_stats* stats, cudaStream_t st);

// noalloc.cu: commit the allocation-free entry point's scratch array on the
// current device (best effort)
void noalloc_reserve();

// fourier.cu: the Fourier-domain data term (Eqs. four_obj, fusedop)
int check_fourier_params(const ct_geometry& g, const ct_fourier_params& P);
int build_fourier(ct_matrix* M, const ct_fourier_params* P);
void free_fourier(ct_matrix* M);
int64_t fourier_stored_weights(const ct_matrix* M);
// Re(F^H F) in (double-float, tiled) fused with the CG operator epilogue
int launch_fourier_op_df(const ct_matrix* M, const OpEpilogue& ep, cudaStream_t st);
// out (double-float, tiled) = scale Re(F^H fhat), fhat the DFTs of the real sinogram f
int fourier_backproject_df(const ct_matrix* M, const float* f, float2* out, double scale, cudaStream_t st);
// point response s(d) = Re(F^H F e_c)[c + d] for |di|, |dj| <= r, FP64 [(2r+1)^2]
void fourier_point_response(const ct_matrix* M, int r, std::vector<double>& h);
// public products (FP32, row-major image, interleaved complex samples)
int fourier_forward(const ct_matrix* M, const float* x, float* y, cudaStream_t st);
int fourier_adjoint(const ct_matrix* M, const float* y, float* x, cudaStream_t st);
int fourier_normal(const ct_matrix* M, const float* x, float* out, cudaStream_t st);
int fourier_data(const ct_matrix* M, const float* f, float* fhat, cudaStream_t st);

}  // namespace ct
