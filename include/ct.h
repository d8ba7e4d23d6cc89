/*
 * ct.h -- C ABI of the GB300 sparse-operator CT reconstruction library (libct.so).
 *
 * Method: R. C. Barnard and R. Archibald, "Accelerating optimization-based
 * computed tomography via sparse matrix approximations" (arXiv 1705.07497).
 * The library evaluates the parallel-beam Radon transform restricted to the
 * measured angles, A = M R (Sec. 1, Eq. objmin), and its adjoint A^T as
 * precomputed sparse matrices (Sec. 3: geometry-dependent matrices are built
 * once, offline, and reused), and applies them inside conjugate-gradient
 * solves of
 *      (c_id I + c_ata A^T A + c_grad grad^T grad) u = rhs
 * which covers Eq. KKT (p = 2), Eq. PD_resolve (Chambolle-Pock resolvent)
 * and Eq. SB_solve (split Bregman), nested in anisotropic-TV split Bregman
 * (Sec. 4).  The sparse surrogate T of Sec. 3.2 (Eq. def_sparse_surr,
 * Eq. surr_SBupd) can replace A^T A.
 *
 * Conventions shared by every call
 *   image      N x N pixels of side 1, row-major: pixel (i, j) is element
 *              p = i*N + j and covers x in [j-N/2, j-N/2+1], y in [i-N/2, i-N/2+1].
 *   angles     theta_k = k*pi/n_angles_total, k = 0 .. n_angles_total-1; the row
 *              selector M keeps k % keep_every == 0 (kept angle k' = k/keep_every).
 *   detector   n_bins bins of width 1; bin b sits at s_b = b - (n_bins-1)/2.
 *   ray (k,b)  the line x cos(theta_k) + y sin(theta_k) = s_b; row q = k'*n_bins + b.
 *   A entries  exact intersection length of ray q with pixel p (Siddon
 *              lengths, computed in FP64 from a closed form); a ray lying on a
 *              pixel edge gives half its length to each of the two pixels;
 *              theta exactly 0 or pi/2 use exact direction cosines; lengths
 *              below 1e-12 are dropped.
 *   batches    a batch of B images is laid out [N*N][B] and a batch of B
 *              sinograms [rows][B]: the slice index is innermost.
 *   pointers   vector arguments are plain pointers to float32 data, owned by
 *              the caller.  Device pointers are used in place and the call is
 *              asynchronous on `cuda_stream` (a cudaStream_t; NULL = legacy
 *              default stream).  Host pointers (pageable or pinned) are
 *              staged through library-owned device buffers and the call
 *              returns after the results have been copied back (synchronous).
 *              All vector arguments of one call must be of the same kind.
 *   errors     every int-returning call returns CT_OK (0) or a negative
 *              CT_ERR_* code; nothing aborts or exits.  ct_last_error()
 *              returns a per-thread message for the last failure.
 *   threads    a matrix handle owns workspace used by ct_cg_solve and
 *              ct_split_bregman; concurrent solver calls on one handle must be
 *              serialised by the caller (same stream, or external ordering).
 */
#ifndef CT_H
#define CT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CT_OK = 0,
    CT_ERR_ARG = -1,         /* invalid argument, size or pointer               */
    CT_ERR_CUDA = -2,        /* a CUDA runtime call failed                       */
    CT_ERR_OOM = -3,         /* device or host allocation failed                 */
    CT_ERR_BREAKDOWN = -4,   /* CG saw p^T Op p <= 0 with a nonzero residual     */
    CT_ERR_NONFINITE = -5,   /* NaN or Inf met in a residual, dot or update      */
    CT_ERR_TIMEOUT = -6,     /* a bounded device-side wait expired (the persistent
                              * ragged-batch kernel of ct_split_bregman_ragged)  */
    CT_ERR_UNSUPPORTED = -7  /* option not available for this matrix / build     */
};

/* Matrix storage flags for ct_build_matrix (Sec. 3: precomputed sparse form). */
enum {
    CT_VAL_FP32 = 0,          /* FP32 values                                      */
    CT_VAL_FP16_ROWSCALE = 1, /* A = diag(s) Q: Q in FP16 (|Q| <= 1), s FP32 per
                                 row; A^T is applied as Q^T (s .* y), so the
                                 quantised normal operator stays symmetric     */
    CT_KEEP_FP32_COPY = 4,    /* with FP16 storage, also keep FP32 values for
                                 residual refreshes (ct_cg_params.refresh_every) */
    CT_F64_FP64_PIPE = 8      /* ct_forward_f64, ct_adjoint_f64 and ct_normal_f64
                                 gather and accumulate in FP64 (one FP64 FMA per
                                 entry) instead of the default double-float
                                 kernels on the FP32 pipes; several times slower
                                 on this part, whose FP64 pipe is narrow        */
};

typedef struct {
    int32_t n;              /* image size N (N x N pixels of side 1)              */
    int32_t n_angles_total; /* theta_k = k*pi/n_angles_total                      */
    int32_t keep_every;     /* M keeps k % keep_every == 0 (Sec. 1)               */
    int32_t n_bins;         /* detector bins of width 1, centred                  */
} ct_geometry;

typedef struct ct_matrix *ct_matrix_t; /* opaque, library-owned, device-resident */

/* Builds A = M R and A^T for geometry *g on the current CUDA device.  The
 * device form is internal: both matrices are stored in sliced ELL (slices of
 * 32 rows, 8-entry chunks per row, padding entries of value 0); A's columns
 * index a tiled image layout and A^T's rows follow it, with 16-bit column
 * indices local to each image tile's band of detector bins.  Both matrices
 * are computed from the same closed-form chord length, so A^T holds exactly
 * the values of A; ct_matrix_export returns plain CSR.
 * Errors: CT_ERR_ARG (n <= 0, n*n >= 2^31, counts <= 0, NULL out),
 * CT_ERR_UNSUPPORTED (more band slots per image tile than 16-bit indices
 * address: about 3000 kept angles), CT_ERR_OOM, CT_ERR_CUDA.
 * *out receives the handle (NULL on failure). */
int ct_build_matrix(const ct_geometry *g, uint32_t flags, ct_matrix_t *out);

/* rows = n_kept*n_bins, cols = N*N, nnz = number of stored nonzeros (no
 * padding).  Any output pointer may be NULL. */
int ct_matrix_info(ct_matrix_t A, int64_t *rows, int64_t *cols, int64_t *nnz);

/* Frees the handle, its matrices, workspace and captured graphs (NULL is a no-op). */
void ct_destroy_matrix(ct_matrix_t A);

/* y[rows][batch] = A x[N*N][batch]  (Sec. 1: the data term's M R).
 * With FP16 storage: y = s .* (Q x).  batch >= 1. */
int ct_forward(ct_matrix_t A, const float *x, float *y, int32_t batch, void *cuda_stream);

/* x[N*N][batch] = A^T y[rows][batch]  (the adjoint R* M* of Eq. KKT).
 * With FP16 storage: x = Q^T (s .* y). */
int ct_adjoint(ct_matrix_t A, const float *y, float *x, int32_t batch, void *cuda_stream);

/* FP64-vector forms of ct_forward / ct_adjoint for callers that keep their
 * vectors in FP64 (the differentiable reconstruction of the Python layer).
 * Same layout and batching; device pointers only (CT_ERR_ARG otherwise).  The
 * matrix values are those of the storage form.  Each FP64 input value is
 * split into a double-float pair (hi, lo) = (fl32(v), fl32(v - hi)), which
 * holds it to 2^-48 relative; the product runs in the solvers' double-float
 * kernels (error-free products, compensated sums) and each output pair is
 * summed back to FP64: about 1e-14 relative error per output, which is what
 * the derivatives of the unrolled reconstruction need.  A handle built with
 * CT_F64_FP64_PIPE gathers and accumulates in FP64 instead (one FP64 FMA per
 * entry).  Uses workspace buffers of the handle, allocated on first use. */
int ct_forward_f64(ct_matrix_t A, const double *x, double *y, int32_t batch, void *cuda_stream);
int ct_adjoint_f64(ct_matrix_t A, const double *y, double *x, int32_t batch, void *cuda_stream);

/* out = alpha A^T A x + lambda grad^T grad x: the operator of Eq. SB_solve
 * (with "+ lambda K*K", K = grad) on FP64 vectors [N*N][batch] in the
 * caller's row-major image order (forward differences, last difference
 * zero).  Two FP64-vector products (as ct_forward_f64 / ct_adjoint_f64) and
 * one fused stencil pass; the operator is symmetric, so it is also its own
 * derivative (the differentiable reconstruction's backward pass uses it).
 * Device pointers only; x and out must not overlap.  Asynchronous.
 * Errors: CT_ERR_ARG, CT_ERR_UNSUPPORTED (Fourier handle), CT_ERR_CUDA. */
int ct_normal_f64(ct_matrix_t A, double alpha, double lambda, const double *x, double *out, int32_t batch,
                  void *cuda_stream);

typedef struct {
    double c_id, c_ata, c_grad; /* Op = c_id I + c_ata A^T A (or T) + c_grad grad^T grad.
                                   SB (Eq. SB_solve): (0, alpha, lambda);
                                   CP resolvent (Eq. PD_resolve): (1, tau*alpha, 0);
                                   p = 2 normal equations (Eq. KKT): (0, alpha, 1). */
    int32_t max_iters;          /* CG steps (Sec. 4: a small fixed count)              */
    double rel_tol;             /* also stop once ||r|| <= rel_tol ||rhs||; 0 = off    */
    int32_t surrogate_r;        /* 0: exact A^T A; > 0: surrogate T of radius r (Sec. 3.2) */
    int32_t refresh_every;      /* FP16 storage: recompute r = rhs - Op(u) with the FP32
                                   matrices every k steps (needs CT_KEEP_FP32_COPY); 0 = off */
    int32_t surrogate_square;   /* 0: disc window |d|_2 <= r; 1: square |d|_inf <= r */
} ct_cg_params;

typedef struct {
    int32_t iters;        /* CG steps taken (max over the batch)                   */
    double final_rel_res; /* ||r||/||rhs|| of the recursively updated residual
                             (max over the batch)                                  */
    int32_t status;       /* CT_OK, CT_ERR_BREAKDOWN or CT_ERR_NONFINITE           */
} ct_cg_stats;

/* Solves Op u = rhs per slice with conjugate gradients (Sec. 2: no closed-form
 * solution exists), warm-started from u.  rhs, u: [N*N][batch]; u is
 * overwritten with the iterate.  FP32 vectors, FP64 dot products.  stats
 * (host pointer) may be NULL; when given, the call synchronises the stream
 * to fill it and returns its status.  Without stats a breakdown is reported
 * only through a later call's status. */
int ct_cg_solve(ct_matrix_t A, const ct_cg_params *params, const float *rhs, float *u,
                int32_t batch, ct_cg_stats *stats, void *cuda_stream);

typedef struct {
    double alpha, lambda;   /* Eq. objmin's alpha; split-Bregman penalty lambda     */
    int32_t outer_iters;    /* Bregman updates                                       */
    int32_t inner_cg_iters; /* CG steps per update (warm-started)                    */
    double stop_rel_update; /* Sec. 4: stop once ||u^{k+1}-u^k||_1 < tol * first; 0 = off */
    int32_t surrogate_r;    /* 0: exact A^T A; > 0: surrogate T (Eq. surr_SBupd)    */
    int32_t refresh_every;  /* as in ct_cg_params                                    */
    int32_t surrogate_square;
    double cg_rel_tol;      /* each inner solve also stops once ||r|| <= cg_rel_tol ||rhs||
                               (inner_cg_iters is then the cap); 0 = the fixed count of
                               Sec. 4.  A tight tolerance makes the reconstruction a
                               function of the problem alone: a fixed count of CG steps
                               amplifies rounding differences over many updates       */
} ct_sb_params;

typedef struct {
    int32_t outer_done;     /* Bregman updates performed (min over the batch)       */
    double first_update_l1; /* ||u^1 - u^0||_1 (slice 0)                            */
    double last_update_l1;  /* ||u^K - u^{K-1}||_1 (slice 0)                        */
    int32_t status;
} ct_sb_stats;

/* Anisotropic-TV split Bregman for min alpha/2 ||A u - f||^2 + ||grad u||_1
 * (Eq. objmin with p = 1, K = grad; Sec. 4), one independent problem per slice:
 *   rhs = alpha A^T f + lambda grad^T (d - b)
 *   u   = CG_{inner}(alpha A^T A (or T) + lambda grad^T grad, rhs, warm start u)
 *   d   = shrink(grad u + b, 1/lambda);  b = b + grad u - d
 * with d = b = 0 at the start.  f: [rows][batch] measured data (already
 * restricted by M); u: [N*N][batch], in = initial guess, out = reconstruction.
 * stats may be NULL (then the call does not synchronise). */
int ct_split_bregman(ct_matrix_t A, const ct_sb_params *params, const float *f, float *u,
                     int32_t batch, ct_sb_stats *stats, void *cuda_stream);

/* Chambolle-Pock primal-dual method (the method Sec. 2 cites; Chambolle and
 * Pock 2011, Algorithm 1) for min alpha/2 ||A u - g||^2 + ||grad u||_1 (Eq.
 * objmin with p = 1, K = grad, anisotropic TV):
 *   p    = clip(p + sigma grad ubar, -1, 1)                   (dual, per component)
 *   u    = (I + tau alpha A^T A)^{-1} (u - tau grad^T p + tau alpha A^T g)
 *                                   (Eq. PD_resolve, inner_cg_iters CG steps from u)
 *   ubar = u + theta (u - u_old)
 * with ubar = u (the initial guess) and p = 0 at the start.  Converges for
 * sigma tau ||grad||^2 < 1, ||grad||^2 <= 8.  g: [rows] measured data; u:
 * [N*N] in = initial guess, out = reconstruction.  batch must be 1.  stats
 * (NULL or one entry): updates done and the L1 size of the first and last
 * update; the call then synchronises.  Errors: CT_ERR_ARG (tau, sigma <= 0,
 * alpha < 0, theta outside [0, 1], negative counts), CT_ERR_UNSUPPORTED
 * (batch != 1), CT_ERR_BREAKDOWN / CT_ERR_NONFINITE from a resolvent solve. */
typedef struct {
    double alpha;           /* data weight                                     */
    double tau, sigma;      /* primal and dual step sizes                      */
    double theta;           /* extrapolation, 1 in Algorithm 1                 */
    int32_t outer_iters;    /* primal-dual updates                             */
    int32_t inner_cg_iters; /* CG steps per resolvent                          */
} ct_cp_params;

int ct_chambolle_pock(ct_matrix_t A, const ct_cp_params *params, const float *g, float *u, int32_t batch,
                      ct_sb_stats *stats, void *cuda_stream);

/* Ragged batch: `count` independent split-Bregman problems of possibly
 * different geometries in one call (Sec. 4's reconstruction, many slices and
 * scanners at once).  Problem i uses matrix A[i] (its geometry), data f[i]
 * ([rows_i], device pointer) and image u[i] ([N_i*N_i], device pointer; in =
 * initial guess, out = reconstruction); every problem runs with the same
 * params.  When every handle serves at most eight of the problems and the
 * operator is the exact one (surrogate_r = 0, refresh_every = 0), each
 * problem runs as a single-slice solve and one Bregman update of all of them
 * is ONE persistent cooperative kernel launch: its CTAs take work items
 * (a few 32-ray slices, an image tile or a run of pixels of one phase of one
 * problem) from a device queue that interleaves the problems phase by phase,
 * and an item waits, with a bounded spin, until the previous phase of its
 * problem is complete; the launch is captured into a CUDA graph that is
 * replayed outer_iters times.  A wait that runs out sets CT_ERR_TIMEOUT and
 * makes every CTA stop (see ct_set_wait_limit).  Otherwise problems that
 * share a handle are solved together as one batch of that handle (SpMM), the
 * groups' Bregman updates are captured in one CUDA graph, each group on its
 * own stream, and the graph is replayed outer_iters times.  The call
 * synchronises cuda_stream when it takes the persistent form.  The u[i] must not overlap
 * each other or any f[j].  stats: NULL, or an array of `count` entries, one
 * per problem (then the call synchronises on cuda_stream).  Handles must live
 * on the current device; calls sharing a handle must be serialised like any
 * solver call.  Errors: CT_ERR_ARG (count < 1, NULL arrays or pointers, host
 * pointers, bad params), CT_ERR_OOM, CT_ERR_CUDA, CT_ERR_TIMEOUT (a bounded
 * wait of the persistent kernel expired; the problems' images are then not
 * valid), and per problem CT_ERR_BREAKDOWN / CT_ERR_NONFINITE (the first one
 * met is returned). */
int ct_split_bregman_ragged(int32_t count, const ct_matrix_t *A, const float *const *f, float *const *u,
                            const ct_sb_params *params, ct_sb_stats *stats, void *cuda_stream);

/* Launch tuning of the batched products (no counterpart in the paper).  The
 * batched sparse products (batch >= 2) come in variants that differ only in
 * how many staged matrix entries each lane keeps in flight (4, 8, or 16 for
 * batches below 64 slices, where a lane takes one slice; the fused solver
 * kernels take 8 for 16); they compute bit-identical results.  By default
 * the first batched solve, or the first batched ct_forward_f64 /
 * ct_normal_f64, with a given batch size on a handle times the variants on
 * its own data (a few launches of the forward product, synchronising the
 * stream once, never inside a stream capture) and keeps the fastest.
 * ct_set_spmm_unroll pins the choice for a batch size (4, 8 or 16; 0 returns
 * it to automatic);
 * ct_get_spmm_unroll reports it (0 = not chosen yet).
 * Errors: CT_ERR_ARG (batch < 2, other unroll values, NULL output). */
int ct_set_spmm_unroll(ct_matrix_t A, int32_t batch, int32_t unroll);
int ct_get_spmm_unroll(ct_matrix_t A, int32_t batch, int32_t *unroll);

/* Bounded waits of the persistent ragged-batch kernel (no counterpart in the
 * paper).  Every wait of that kernel polls at most `polls` times (about
 * 128 ns or more apart) and then gives up with CT_ERR_TIMEOUT; polls <= 0
 * restores the default (about a second).  hold_first != 0 makes the first
 * phase of every problem wait for a flag that nothing ever sets, so that the
 * next ct_split_bregman_ragged call in persistent form runs out of its waits
 * and returns CT_ERR_TIMEOUT without touching the images: this exercises the
 * timeout path on a GPU without faulting it.  Process-wide; takes effect at
 * the next call.  Always returns CT_OK. */
int ct_set_wait_limit(int64_t polls, int32_t hold_first);

/* Launch shapes of the sparse products (no counterpart in the paper).  Each
 * product comes in launch shapes that all compute the same bits (every row is
 * summed in the same order whatever the shape); only speed depends on the
 * choice.  Fields (0 = not chosen yet / automatic):
 *   fwd_warps    one slice, y = A x: warps per block, 4 or 8 (a warp takes
 *                four neighbouring rays of a 32-ray slice)
 *   fwd_unroll   one slice, y = A x: 8-entry chunks each lane keeps in flight,
 *                2, 4, 8 or 16
 *   op_ctas      one slice, the A^T kernel fused with the CG operator: CTAs
 *                per SM its registers are sized for, 7, 4 or 3 (3: each lane
 *                also copies its next two matrix chunks into shared memory
 *                ahead of use); 5 or 3 when the sinogram band is staged in
 *                angle chunks (above about 180 kept angles)
 *   op_pixels    one slice, the same kernel: pixel rows per lane, 1, or 2
 *                (four warps per image tile, seven CTAs per SM; single-chunk
 *                bands only, with op_ctas 0 or 7)
 *   spmm_unroll  batches of 2 or more: staged entries in flight, 4, 8 or 16
 * By default the first solve on a handle (batch 1: ct_cg_solve,
 * ct_split_bregman, ct_chambolle_pock, and the single-slice groups of
 * ct_split_bregman_ragged; batch B: the batched solves) times the candidates
 * on the handle's own matrices, never inside a stream capture, and keeps the
 * fastest; batch-1 choices are also cached for the process by geometry and
 * storage flags, so later handles of the same geometry take them untimed.
 * ct_tune runs that search now (synchronising cuda_stream); ct_set_tuning pins
 * fields for a batch size (0 returns one to automatic); ct_get_tuning reports
 * them.  Fields of the other batch kind must be 0.  Errors: CT_ERR_ARG (batch
 * < 1, values outside the lists, NULL pointers), CT_ERR_UNSUPPORTED (Fourier
 * handle), CT_ERR_CUDA. */
typedef struct {
    int32_t fwd_warps;
    int32_t fwd_unroll;
    int32_t op_ctas;
    int32_t op_pixels;
    int32_t spmm_unroll;
} ct_tuning;

int ct_get_tuning(ct_matrix_t A, int32_t batch, ct_tuning *t);
int ct_set_tuning(ct_matrix_t A, int32_t batch, const ct_tuning *t);
int ct_tune(ct_matrix_t A, int32_t batch, void *cuda_stream);

/* Launch timing of the kernels of one CG step (measurement only; the paper's
 * Sec. 4 times whole reconstructions).  On the handle's single-slice
 * workspace, each kernel of a CG step on Op = c_ata A^T A + c_grad grad^T grad
 * (Eq. SB_solve with alpha = c_ata, lambda = c_grad) is launched exactly as
 * the solver launches it (the same template instance and launch shape),
 * 3 times untimed and then `reps` times back to back between two CUDA events
 * on cuda_stream; ms[k] (host array of 4) receives the mean milliseconds
 * per launch of:
 *   ms[0]  y = A p               (double-float vectors)
 *   ms[1]  q = Op(p), p.q        (A^T y fused with the operator epilogue and
 *                                 the grid-wide dot product)
 *   ms[2]  u += alpha p, r -= alpha q, r.r
 *   ms[3]  p = r + beta p
 * The workspace's vectors are overwritten (p = r = 1, u = q = 0 first); the
 * call synchronises.  Errors: CT_ERR_ARG (reps < 1, NULL ms),
 * CT_ERR_UNSUPPORTED (Fourier handle), CT_ERR_OOM, CT_ERR_CUDA. */
int ct_time_cg_kernels(ct_matrix_t A, double c_ata, double c_grad, int32_t reps, double *ms, void *cuda_stream);

/* Allocation-free variant of ct_cg_solve.  The paper has no counterpart.
 *
 * Some callers cannot allocate device memory at the moment they need a solve:
 * a real-time reconstruction loop that must not stall on an allocation (which
 * can synchronise the device), or a process whose device memory has already
 * been taken by another allocator, so that a fresh cudaMalloc would fail.
 * This entry point does the same single-slice CG solve as ct_cg_solve
 * (batch 1, exact operator: surrogate_r must be 0) but never allocates: its
 * vectors, reduction buffers and CG scalars live in one fixed scratch array
 * of CT_NOALLOC_SCRATCH_BYTES that is part of libct.so's device image.
 *   - Every GPU that loads the library holds this array until the process exits.
 *   - Problems that need more scratch than the limit (about 40 bytes per pixel
 *     plus 8 per sinogram sample; N = 512 with 130,500 rays fits) are rejected
 *     with CT_ERR_ARG and a message giving the size needed.
 *   - rhs and u must be device pointers (host staging would allocate).
 *   - The runtime backs the array on a device when it first loads the
 *     library's device code there.  ct_build_matrix and ct_build_fourier do
 *     that on the handle's device (they look up the array's address with
 *     cudaGetSymbolAddress), so the array is committed while allocating is
 *     still allowed.  If the device had no room then, the first call of this
 *     entry point on that device tries again and returns CT_ERR_OOM when it
 *     still cannot; make that first call before any stream capture.  Every
 *     call looks the address up again (with the handle's device current), so
 *     no stale address survives a device reset.
 *   - All calls share the one array and it keeps the last call's contents:
 *     the call clears what must start at zero itself, but calls whose work
 *     overlaps on the GPU (other streams, other threads) race on it; serialise
 *     them.
 * Arguments, results and errors are otherwise those of ct_cg_solve. */
#define CT_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int ct_cg_solve_noalloc(ct_matrix_t A, const ct_cg_params *params, const float *rhs, float *u,
                        ct_cg_stats *stats, void *cuda_stream);

/* Copies A (which = 0) or A^T (which = 1) to host memory as unpadded CSR:
 * row_ptr[rows+1] (int64), cols[nnz] (int32), vals[nnz] (FP32; with FP16
 * storage, the dequantised s_q * Q_qp).  Pass NULL arrays to query sizes
 * through ct_matrix_info.  Synchronous. */
int ct_matrix_export(ct_matrix_t A, int32_t which, int64_t *row_ptr, int32_t *cols, float *vals);

/* Copies the FP16 storage form to host memory: q_bits[nnz] (IEEE binary16
 * bit patterns of Q in the row order of A) and scale[rows] (s, FP32).
 * CT_ERR_UNSUPPORTED without CT_VAL_FP16_ROWSCALE.  Synchronous. */
int ct_matrix_export_fp16(ct_matrix_t A, uint16_t *q_bits, float *scale);

/* Surrogate stencil of Sec. 3.2: s(d) = (A^T A e_c)[c + d] for c = (N/2, N/2)
 * (0-based) and offsets d = (di, dj) in the window (disc |d|_2 <= r, or square
 * when square != 0), averaged with s(-d) so that T is symmetric; computed in
 * FP64.  Writes up to `capacity` taps (di[], dj[], val[], host arrays) and the
 * number of taps to *count.  Synchronous.
 * For the Siddon operator the point response decays like 1/|d| (a point
 * back-projects along every kept angle), so the window keeps a small part of
 * the response of A^T A to smooth images, and a surrogate solve returns an
 * image whose smooth part is too large by about sum(h) / sum(s), where h is
 * the whole point response and s the window's taps (about 290 for r = 1 at
 * N = 512 with 180 angles); small windows can also make the surrogate system
 * indefinite, which CG reports as CT_ERR_BREAKDOWN. */
int ct_surrogate_stencil(ct_matrix_t A, int32_t r, int32_t square, int32_t capacity,
                         int32_t *di, int32_t *dj, double *val, int32_t *count);

/* ---------------------------------------------------------------------------
 * Fourier-domain data term (Sec. 2, Eqs. four_obj, SBFFT) evaluated by Gaussian
 * gridding (Sec. 3.1) with the fused matrix B* B (Eq. fusedop).
 *
 * By the Fourier slice theorem the 1-D DFT of the projection at angle theta_k
 * samples the image's 2-D transform on the line rho (cos theta_k, sin theta_k).
 *   samples   J = n_kept * n_bins, sample j = k'*n_bins + m at
 *             omega_j = rho_m (cos theta_k, sin theta_k),
 *             rho_m = 2 pi (m - floor(n_bins/2)) / n_bins.
 *   F         (F x)_j = n_bins^{-1/2} sum_p x_p exp(-i omega_j . c_p), c_p the
 *             centre of pixel p: (j - N/2 + 1/2, i - N/2 + 1/2).
 *   data      fhat_j = n_bins^{-1/2} sum_b f_{k',b} exp(-i rho_m s_b), the DFT
 *             of each measured projection; the scaling makes ||F x - fhat||
 *             the sinogram residual of point-sampled pixels, so alpha and
 *             lambda keep their meaning.
 *   normal    Re(F^H F) (real images); right-hand side Re(F^H fhat).
 * F is evaluated as Greengard and Lee's gridding: deconvolution by
 * E(k) = sqrt(pi/tau) exp(k^2 tau) per dimension, zero padding to a 2N x 2N
 * grid, FFT, and Gaussian weights exp(-(w - 2 pi m / 2N)^2 / (4 tau)) over the
 * 2 m_sp + 1 grid points per dimension nearest each sample (|m - m_j| <= m_sp,
 * m_j = floor(w 2N / 2 pi), periodic).  With G those weights (J x 4N^2),
 * Re(F^H F) = E Z^T FFT^H (G^T G) FFT Z E / (16 N^4 n_bins); convolution
 * fusing stores C = G^T G, whose nonzeros lie on the (4 m_sp + 1)^2 periodic
 * offsets |d| <= 2 m_sp, so that one normal-operator product is two FFTs,
 * one product with C and two diagonal scalings.  Accuracy about 2, 6 and 12
 * digits at m_sp = 2, 6, 12 with tau = m_sp / N^2.  The grid and sample
 * vectors, the FFT twiddles and the pixel scaling are double-float; the
 * weights and C are FP32 (a symmetric perturbation of about 1e-7 relative).
 *
 * The handle returned by ct_build_fourier works with ct_matrix_info
 * (rows = J, cols = N*N, nnz = stored weights: C's (4 m_sp + 1)^2 * 4N^2
 * diagonal entries, or J (2 m_sp + 1)^2 for CT_FOURIER_GRIDDING),
 * ct_destroy_matrix, ct_surrogate_stencil (the stencil of the Fourier normal
 * operator, whose point response is translation invariant: s(d) =
 * n_bins^{-1} sum_j cos(omega_j . d), FP64), and with ct_cg_solve,
 * ct_split_bregman and ct_chambolle_pock at batch 1, where c_ata multiplies
 * Re(F^H F) and the data vectors f, g stay real sinograms [n_kept][n_bins]
 * (transformed to fhat inside the call).  Every other call returns
 * CT_ERR_UNSUPPORTED for it.  N must be a power of two in [16, 2048].
 * The products and solves use the handle's grid and sample buffers, so calls
 * on one handle must be serialised (one stream, or external ordering). */
enum {
    CT_FOURIER_FUSED = 0,    /* precomputed C = G^T G (convolution fusing, Eq. fusedop) */
    CT_FOURIER_GRIDDING = 1  /* interpolate with G, then spread with G^T, each product */
};

typedef struct {
    int32_t m_sp;  /* window half-width, 1 .. 12 (2 m_sp + 1 <= 2N)                 */
    double tau;    /* Gaussian parameter; 0 selects m_sp / N^2                       */
    int32_t mode;  /* CT_FOURIER_FUSED or CT_FOURIER_GRIDDING                        */
} ct_fourier_params;

/* Builds the samples, weights and (fused mode) C on the current device.
 * Errors: CT_ERR_ARG for bad sizes or parameters, CT_ERR_UNSUPPORTED for N not
 * a power of two in [16, 2048], CT_ERR_OOM, CT_ERR_CUDA. */
int ct_build_fourier(const ct_geometry *g, const ct_fourier_params *params, ct_matrix_t *out);

/* y = F x: x[N*N] real image (row-major), y[2*J] complex samples (re, im
 * interleaved).  Device pointers only (CT_ERR_ARG otherwise); asynchronous. */
int ct_fourier_forward(ct_matrix_t F, const float *x, float *y, void *cuda_stream);

/* x = Re(F^H y): y[2*J] complex, x[N*N] real.  Device pointers; asynchronous. */
int ct_fourier_adjoint(ct_matrix_t F, const float *y, float *x, void *cuda_stream);

/* out = Re(F^H F x) through the handle's mode (fused C or gridding pair).
 * Device pointers; asynchronous. */
int ct_fourier_normal(ct_matrix_t F, const float *x, float *out, void *cuda_stream);

/* fhat = the DFTs of the projections: f[n_kept*n_bins] real sinogram,
 * fhat[2*J] complex.  Device pointers; asynchronous. */
int ct_fourier_data(ct_matrix_t F, const float *f, float *fhat, void *cuda_stream);

/* Short description of a status code. */
const char *ct_status_string(int status);

/* Message of the last failure on the calling thread ("" if none). */
const char *ct_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CT_H */
