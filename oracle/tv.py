"""FP64 oracle of the solvers: gradient, CG, split Bregman, surrogate T, resolvent.

Test infrastructure only (see the package docstring).

Images are 2-D arrays of shape (ny, nx) stored row-major, so pixel (i, j) is
entry p = i * nx + j of the flattened vector that A acts on.  ``A`` is any
object with ``@`` and ``.T`` (a scipy sparse matrix in practice).

Readings taken where the paper is silent or garbled:
  * K = grad, anisotropic TV (Sec. 4): forward differences with a zero last
    difference (Neumann boundary); K* K = grad^T grad.
  * Eq. SB_solve (and Eqs. SBFFT, SB_update, surr_SBupd) print the operator
    as alpha R*M*MR "-" lambda K*K.  With K = grad, K*K is positive
    semidefinite, so the minus would make the system indefinite; the split
    Bregman method of Goldstein and Osher solves alpha A^T A + lambda K*K.
    The sign is read as "+".
  * The "v" of Eq. SB_solve is d - b (the split variable minus the Bregman
    variable of Goldstein-Osher).
  * Inexact updates (Sec. 4: a fixed, small number of CG steps) warm-start CG
    from the previous iterate.
  * The size of a Bregman update (Sec. 4's stopping rule) is ||u^{k+1}-u^k||_1.
  * The surrogate's point response is taken of the normal operator actually
    used, A^T A, at pixel (N/2, N/2) (0-based); its taps inside the disc
    |d| <= r are averaged with their mirror images, s(d) <- (s(d)+s(-d))/2, so
    that T is symmetric; translates falling outside the image are dropped
    (Sec. 3.2: the object is assumed to stay r pixels away from the edges).
"""

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# K = grad (anisotropic TV, Sec. 4) and its adjoint
# --------------------------------------------------------------------------
def grad(u):
    """Forward differences (gx, gy) of an image u of shape (ny, nx).

    gx[i, j] = u[i, j+1] - u[i, j] for j < nx-1, else 0;
    gy[i, j] = u[i+1, j] - u[i, j] for i < ny-1, else 0.
    """
    gx = np.zeros_like(u)
    gy = np.zeros_like(u)
    gx[:, :-1] = u[:, 1:] - u[:, :-1]
    gy[:-1, :] = u[1:, :] - u[:-1, :]
    return gx, gy


def grad_adj(wx, wy):
    """Adjoint of ``grad``: <grad u, w> = <u, grad_adj(w)>.

    (grad_x^T w)[i, j] = w[i, j-1] [j >= 1] - w[i, j] [j <= nx-2], and the
    same along i for the y component.
    """
    out = np.zeros_like(wx)
    out[:, 1:] += wx[:, :-1]
    out[:, :-1] -= wx[:, :-1]
    out[1:, :] += wy[:-1, :]
    out[:-1, :] -= wy[:-1, :]
    return out


def shrink(x, gamma):
    """Soft thresholding sign(x) max(|x| - gamma, 0).

    Written as x - gamma sign(x) where |x| > gamma, else 0, with the branch
    decided on the real part: the same values for real x, and the analytic
    continuation of the active branch for complex x (complex-step
    differentiation evaluates the oracle at f + i h d)."""
    xr = np.real(x)
    return np.where(np.abs(xr) > gamma, x - gamma * np.sign(xr), 0.0 * x)


# --------------------------------------------------------------------------
# The operator of Eqs. KKT / PD_resolve / SB_solve
# --------------------------------------------------------------------------
def make_operator(A, shape, c_id, c_ata, c_grad, normal=None):
    """Op(x) = c_id x + c_ata N(x) + c_grad grad^T grad x on flattened images.

    N = A^T A by default (Eqs. KKT, PD_resolve, SB_solve) or a surrogate
    (Eq. surr_SBupd) when ``normal`` is given.
    SB: (c_id, c_ata, c_grad) = (0, alpha, lambda); Chambolle-Pock resolvent:
    (1, tau alpha, 0); p = 2 normal equations: (0, alpha, 1).
    """
    if normal is None:
        def normal(x):
            return A.T @ (A @ x)

    def op(x):
        y = np.zeros_like(x)
        if c_id != 0.0:
            y += c_id * x
        if c_ata != 0.0:
            y += c_ata * normal(x)
        if c_grad != 0.0:
            gx, gy = grad(x.reshape(shape))
            y += c_grad * grad_adj(gx, gy).ravel()
        return y

    return op


class Breakdown(ArithmeticError):
    """p^T Op p <= 0 with a nonzero residual: the operator is not SPD."""


def cg(op, rhs, u0, iters, rel_tol=0.0, refresh_every=0, refresh_op=None):
    """Conjugate gradients (Hestenes-Stiefel) for Op u = rhs, warm-started at u0.

    Sec. 2: the systems have no closed-form solution, so an iterative solver
    is used.  Runs ``iters`` steps, or fewer if the residual is exactly zero
    or ||r|| <= rel_tol ||rhs||.  Returns (u, stats).

    Residual replacement (the FP16-storage form's refresh, not in the paper):
    with refresh_every = k > 0, after every k-th step that is not the last
    one the recursively updated residual is replaced by rhs - refresh_op(u)
    (refresh_op defaults to op: the FP32 operator when op is the quantised
    one), and r.r with it; the search direction is kept (no restart).
    """
    # Complex inputs (complex-step differentiation) keep their dtype; the
    # dot products are plain sums of products and every decision below is
    # taken on real parts, so real inputs follow exactly the real algorithm.
    u = np.array(u0, dtype=np.result_type(u0, rhs, np.float64), copy=True)
    r = rhs - op(u)
    p = r.copy()
    rr = r @ r
    rhs_norm = float(np.sqrt(np.real(rhs @ rhs)))
    done = 0
    for _ in range(iters):
        if np.real(rr) == 0.0:
            break
        if rel_tol > 0.0 and np.sqrt(np.real(rr)) <= rel_tol * rhs_norm:
            break
        q = op(p)
        pq = p @ q
        if not np.real(pq) > 0.0:
            raise Breakdown("p^T Op p = %r" % pq)
        a = rr / pq
        u = u + a * p
        r = r - a * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        done += 1
        if refresh_every > 0 and done % refresh_every == 0 and done < iters:
            r = rhs - (op if refresh_op is None else refresh_op)(u)
            rr = r @ r
    rel = float(np.sqrt(np.real(rr))) / rhs_norm if rhs_norm > 0 else 0.0
    return u, {"iters": done, "rel_res": rel}


# --------------------------------------------------------------------------
# Split Bregman for min alpha/2 ||A u - f||^2 + ||grad u||_1 (Sec. 2, Sec. 4)
# --------------------------------------------------------------------------
def split_bregman(A, f, shape, alpha, lam, outer, inner, u0=None, normal=None,
                  stop_rel_update=0.0, cg_tol=0.0, state=None, refresh_every=0, refresh_A=None):
    """Anisotropic-TV split Bregman with inexact CG solves of Eq. SB_solve.

    Each outer step:
      rhs     = alpha A^T f + lambda grad^T (d - b)
      u       = CG(alpha N + lambda grad^T grad, rhs, warm start u, ``inner``)
      g       = grad u
      d       = shrink(g + b, 1/lambda)        (componentwise)
      b       = b + g - d
      update  = ||u_new - u_old||_1
    N = A^T A, or the surrogate T (Eq. surr_SBupd) when ``normal`` is given;
    the right-hand side keeps the exact alpha A^T f in both cases.
    Stops after ``outer`` steps, or once update < stop_rel_update * first
    update (Sec. 4's rule).  ``state`` = (u, dx, dy, bx, by) resumes a run.
    ``refresh_every`` / ``refresh_A``: every inner CG replaces its residual
    every k steps with the one of alpha refresh_A^T refresh_A + lambda
    grad^T grad (the FP32 matrix of the FP16-storage form; see ``cg``).
    """
    ny, nx = shape
    if state is not None:
        u, dx, dy, bx, by = (np.array(a, dtype=np.result_type(a, np.float64), copy=True) for a in state)
        u = u.ravel()
    else:
        u = np.zeros(ny * nx) if u0 is None else np.array(u0, dtype=np.float64).ravel().copy()
        dx = np.zeros(shape)
        dy = np.zeros(shape)
        bx = np.zeros(shape)
        by = np.zeros(shape)
    op = make_operator(A, shape, 0.0, alpha, lam, normal=normal)
    op_refresh = None if refresh_A is None else make_operator(refresh_A, shape, 0.0, alpha, lam)
    atf = alpha * (A.T @ f)
    updates = []
    k = 0
    for k in range(outer):
        rhs = atf + lam * grad_adj(dx - bx, dy - by).ravel()
        u_old = u
        u, _ = cg(op, rhs, u_old, inner, rel_tol=cg_tol, refresh_every=refresh_every, refresh_op=op_refresh)
        gx, gy = grad(u.reshape(shape))
        dx = shrink(gx + bx, 1.0 / lam)
        dy = shrink(gy + by, 1.0 / lam)
        bx = bx + gx - dx
        by = by + gy - dy
        updates.append(float(np.abs(u - u_old).sum()))
        if stop_rel_update > 0.0 and updates[-1] < stop_rel_update * updates[0]:
            k += 1
            break
    else:
        k = outer
    return {
        "u": u.reshape(shape),
        "dx": dx, "dy": dy, "bx": bx, "by": by,
        "updates": updates,
        "outer_done": k,
    }


def tv_objective(A, f, u, alpha):
    """alpha/2 ||A u - f||^2 + ||grad_x u||_1 + ||grad_y u||_1 (Eq. objmin, p=1)."""
    gx, gy = grad(u)
    res = A @ u.ravel() - f
    return 0.5 * alpha * float(res @ res) + float(np.abs(gx).sum() + np.abs(gy).sum())


# --------------------------------------------------------------------------
# Chambolle-Pock resolvent, Eq. PD_resolve
# --------------------------------------------------------------------------
def resolvent(A, shape, tau, alpha, u_tilde, g, iters, u0=None):
    """Solves (I + tau alpha A^T A) u = u_tilde + tau alpha A^T g by CG."""
    rhs = u_tilde.ravel() + tau * alpha * (A.T @ g)
    op = make_operator(A, shape, 1.0, tau * alpha, 0.0)
    start = u_tilde.ravel() if u0 is None else u0.ravel()
    return cg(op, rhs, start, iters)


def chambolle_pock(A, g, shape, alpha, tau, sigma, outer, inner, theta=1.0, u0=None):
    """Primal-dual method of Chambolle and Pock (cited in Sec. 2; their 2011
    paper, Algorithm 1) for min_u alpha/2 ||A u - g||^2 + ||grad u||_1
    (anisotropic TV).  With K = grad, F the l1 norm (F* the indicator of the
    box |p_x|, |p_y| <= 1, whose prox is the projection) and G the data term,
    whose prox is the resolvent of Eq. PD_resolve solved by `inner` CG steps
    warm-started at the previous iterate:
        p^{k+1}    = clip(p^k + sigma grad(ubar^k), -1, 1)
        u^{k+1}    = (I + tau alpha A^T A)^{-1} (u^k - tau grad^T p^{k+1} + tau alpha A^T g)
        ubar^{k+1} = u^{k+1} + theta (u^{k+1} - u^k)
    with u^0 = ubar^0 = u0 (else 0) and p^0 = 0; converges for
    sigma tau ||grad||^2 < 1 (||grad||^2 <= 8 here).  Returns u, the dual
    (px, py), the L1 size of every update and the number of updates."""
    ny, nx = shape
    u = np.zeros(ny * nx) if u0 is None else np.array(u0, dtype=np.float64).ravel().copy()
    ubar = u.copy()
    px = np.zeros(shape)
    py = np.zeros(shape)
    updates = []
    for _ in range(outer):
        gx, gy = grad(ubar.reshape(shape))
        px = np.clip(px + sigma * gx, -1.0, 1.0)
        py = np.clip(py + sigma * gy, -1.0, 1.0)
        ut = u - tau * grad_adj(px, py).ravel()
        u_new, _ = resolvent(A, shape, tau, alpha, ut, g, inner, u0=u)
        updates.append(float(np.abs(u_new - u).sum()))
        ubar = u_new + theta * (u_new - u)
        u = u_new
    return {"u": u.reshape(shape), "px": px, "py": py, "updates": updates, "outer_done": outer}


# --------------------------------------------------------------------------
# Sparse surrogate T, Sec. 3.2 (Eq. def_sparse_surr)
# --------------------------------------------------------------------------
def point_response(A, n):
    """h = A^T A applied to the unit image at pixel (N/2, N/2), as an N x N image."""
    e = np.zeros(n * n)
    e[(n // 2) * n + n // 2] = 1.0
    return (A.T @ (A @ e)).reshape(n, n)


def stencil_offsets(r, shape="disc"):
    """Offsets (di, dj) of the truncation window |(di, dj)| <= r.

    'disc' is the Euclidean reading of Sec. 3.2's |.| <= r (5 taps at r=1,
    29 at r=3); 'square' is the max-norm reading ((2r+1)^2 taps).
    """
    out = []
    for di in range(-r, r + 1):
        for dj in range(-r, r + 1):
            if shape == "disc" and di * di + dj * dj > r * r:
                continue
            out.append((di, dj))
    return out


def surrogate_stencil(h, r, shape="disc"):
    """Truncated point response s(d) = h[c + d] on the window, symmetrised."""
    n = h.shape[0]
    c = n // 2
    taps = {}
    for di, dj in stencil_offsets(r, shape):
        taps[(di, dj)] = 0.5 * (h[c + di, c + dj] + h[c - di, c - dj])
    return taps


def surrogate_matrix(taps, n):
    """T = sum over translates T^{k,l} (Eq. def_sparse_surr), assembled.

    The translate for source pixel p' = c + (k, l) is the truncated point
    response moved to p'; it becomes column p' of T.  Entries that would fall
    outside the image are dropped (no periodic wrap).
    """
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    src = (ii * n + jj).ravel()
    for (di, dj), v in taps.items():
        ti, tj = (ii + di).ravel(), (jj + dj).ravel()
        ok = (ti >= 0) & (ti < n) & (tj >= 0) & (tj < n)
        rows.append(ti[ok] * n + tj[ok])
        cols.append(src[ok])
        vals.append(np.full(ok.sum(), v))
    return sp.csr_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n * n, n * n)
    )
