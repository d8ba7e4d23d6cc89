"""Pins of the FP64 solver oracle: gradient, CG, split Bregman, surrogate T.

Each pin checks the oracle against an independent construction or a
mathematical fact: Kronecker-product difference matrices, a dense Cholesky
solve, the Krylov-subspace optimality of CG iterates, the 1-D TV optimality
certificate, KKT conditions of the TV problem, and the sum-of-translates
definition of T (Sec. 3.2, Eq. def_sparse_surr) against a library
correlation.
"""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.signal as ssig
import scipy.sparse as sp

from oracle import radon, tv
from paper_1705_07497_gb300 import inputs


def _diff_matrix(n):
    """1-D forward difference with a zero last row (Neumann)."""
    D = sp.lil_matrix((n, n))
    for j in range(n - 1):
        D[j, j] = -1.0
        D[j, j + 1] = 1.0
    return D.tocsr()


def _grad_matrices(ny, nx):
    Gx = sp.kron(sp.identity(ny), _diff_matrix(nx))
    Gy = sp.kron(_diff_matrix(ny), sp.identity(nx))
    return Gx.tocsr(), Gy.tocsr()


def test_grad_matches_kronecker_construction():
    ny, nx = 7, 9
    u = inputs.random_vector(ny * nx, 5).reshape(ny, nx)
    w = inputs.random_vector(2 * ny * nx, 6).reshape(2, ny, nx)
    Gx, Gy = _grad_matrices(ny, nx)
    gx, gy = tv.grad(u)
    np.testing.assert_allclose(gx.ravel(), Gx @ u.ravel(), atol=1e-15)
    np.testing.assert_allclose(gy.ravel(), Gy @ u.ravel(), atol=1e-15)
    got = tv.grad_adj(w[0], w[1]).ravel()
    np.testing.assert_allclose(got, Gx.T @ w[0].ravel() + Gy.T @ w[1].ravel(), atol=1e-14)


def test_grad_adjoint_identity():
    u = inputs.random_vector(64 * 64, 7).reshape(64, 64)
    w = inputs.random_vector(2 * 64 * 64, 8).reshape(2, 64, 64)
    gx, gy = tv.grad(u)
    lhs = float((gx * w[0]).sum() + (gy * w[1]).sum())
    rhs = float((u * tv.grad_adj(w[0], w[1])).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _small_problem(n=16, nt=24, keep=1):
    A = radon.siddon_matrix(n, nt, keep, inputs.n_bins_for(n))
    return A


def _dense_op(A, n, c_id, c_ata, c_grad):
    Gx, Gy = _grad_matrices(n, n)
    Ad = A.toarray()
    L = (Gx.T @ Gx + Gy.T @ Gy).toarray()
    return c_id * np.eye(n * n) + c_ata * Ad.T @ Ad + c_grad * L


def test_cg_converges_to_dense_cholesky_solve():
    n = 16
    A = _small_problem(n)
    M = _dense_op(A, n, 0.0, 1.0, 0.5)
    rhs = inputs.random_vector(n * n, 9)
    Lc = np.linalg.cholesky(M)
    want = sla.solve_triangular(Lc.T, sla.solve_triangular(Lc, rhs, lower=True), lower=False)
    op = tv.make_operator(A, (n, n), 0.0, 1.0, 0.5)
    got, st = tv.cg(op, rhs, np.zeros(n * n), 2000, rel_tol=1e-13)
    assert st["rel_res"] <= 1e-13
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_cg_iterate_minimises_energy_over_krylov_space(k):
    """After k steps from x0, CG's iterate minimises the Op-energy of the
    error over x0 + span{r0, Op r0, ..., Op^{k-1} r0}."""
    n = 16
    A = _small_problem(n)
    M = _dense_op(A, n, 0.0, 1.0, 0.3)
    rhs = inputs.random_vector(n * n, 10)
    x0 = inputs.random_vector(n * n, 11)
    r0 = rhs - M @ x0
    V = [r0]
    for _ in range(k - 1):
        V.append(M @ V[-1])
    Qb, _ = np.linalg.qr(np.stack(V, axis=1))
    y = np.linalg.solve(Qb.T @ M @ Qb, Qb.T @ r0)
    want = x0 + Qb @ y
    op = tv.make_operator(A, (n, n), 0.0, 1.0, 0.3)
    got, st = tv.cg(op, rhs, x0, k)
    assert st["iters"] == k
    assert np.linalg.norm(got - want) <= 1e-8 * np.linalg.norm(want)


def test_cg_refresh_beyond_the_last_step_is_plain_cg():
    """A refresh period at or past the step count never replaces the residual:
    the iterate is plain CG's, to the last bit."""
    n = 16
    A = _small_problem(n)
    op = tv.make_operator(A, (n, n), 0.0, 1.0, 0.3)
    op2 = tv.make_operator(A, (n, n), 0.0, 1.1, 0.3)
    rhs = inputs.random_vector(n * n, 12)
    x0 = inputs.random_vector(n * n, 13)
    plain, _ = tv.cg(op, rhs, x0, 8)
    for k in (8, 9, 100):
        got, _ = tv.cg(op, rhs, x0, 8, refresh_every=k, refresh_op=op2)
        np.testing.assert_array_equal(got, plain)


def test_cg_refresh_with_the_same_operator_only_rounds():
    """Replacing the recursive residual by the true one of the same operator
    changes nothing in exact arithmetic (the two residuals are equal), so the
    iterate agrees with plain CG to rounding while CG is far from converged
    (a few steps: a fixed CG step count amplifies rounding as it grows)."""
    n = 16
    A = _small_problem(n)
    op = tv.make_operator(A, (n, n), 0.0, 1.0, 0.3)
    rhs = inputs.random_vector(n * n, 14)
    plain, st = tv.cg(op, rhs, np.zeros(n * n), 6)
    assert st["rel_res"] > 1e-2
    for k in (1, 2, 5):
        got, _ = tv.cg(op, rhs, np.zeros(n * n), 6, refresh_every=k)
        assert np.linalg.norm(got - plain) <= 1e-13 * np.linalg.norm(plain)


def test_cg_refresh_by_hand():
    """Three steps by hand for Op = diag(1, 2, 4), rhs = (1, 1, 1), u0 = 0,
    with the residual replaced after step 2 by that of B = diag(1, 2, 5):
    step 1: alpha = 3/7, u1 = (3, 3, 3)/7, r1 = (4, 1, -5)/7, p1 = (6, 3, -3)/7;
    step 2: alpha = 7/15, u2 = (29, 22, 8)/35, recursive r2 = (6, -9, 3)/35,
    beta = 3/25, p2 = (48, -36, 6)/175; refresh: r2 = rhs - B u2 =
    (6, -9, -5)/35, r.r = 142/1225; step 3: p2.Op p2 = 5040/30625,
    alpha = 355/504, u3 = (751/735, 237/490, 743/2940).  Plain CG ends at the
    solution (1, 1/2, 1/4); a refresh after step 1 instead would end at
    (38949/30149, 24897/60298, 15123/60298)."""
    d = np.array([1.0, 2.0, 4.0])
    b = np.array([1.0, 2.0, 5.0])
    got, st = tv.cg(lambda x: d * x, np.ones(3), np.zeros(3), 3, refresh_every=2, refresh_op=lambda x: b * x)
    assert st["iters"] == 3
    np.testing.assert_allclose(got, [751 / 735, 237 / 490, 743 / 2940], rtol=1e-14, atol=0)
    plain, _ = tv.cg(lambda x: d * x, np.ones(3), np.zeros(3), 3)
    np.testing.assert_allclose(plain, [1.0, 0.5, 0.25], rtol=1e-14, atol=0)


def test_sb_refresh_uses_the_refresh_matrix_in_every_inner_solve():
    """Split Bregman with a refresh matrix equal to A is split Bregman without
    one, to rounding; with a different refresh matrix it moves."""
    n = 16
    A = _small_problem(n)
    truth = inputs.ellipse_phantom(n, 2)
    f = A @ truth.ravel()
    plain = tv.split_bregman(A, f, (n, n), 1.0, 0.1, 4, 6)["u"]
    same = tv.split_bregman(A, f, (n, n), 1.0, 0.1, 4, 6, refresh_every=2, refresh_A=A)["u"]
    assert np.linalg.norm(same - plain) <= 1e-10 * np.linalg.norm(plain)
    other = tv.split_bregman(A, f, (n, n), 1.0, 0.1, 4, 6, refresh_every=2, refresh_A=1.01 * A)["u"]
    assert np.linalg.norm(other - plain) >= 1e-4 * np.linalg.norm(plain)


def test_sb_1d_tv_denoising_satisfies_optimality_certificate():
    """A = I on an n x 1 image: SB must reach the 1-D TV-denoising minimiser of
    alpha/2 ||u - f||^2 + sum |u_{k+1} - u_k|.  Its certificate is
    z_k = alpha sum_{i<=k} (u_i - f_i), with |z_k| <= 1, z_k = sign(u_{k+1}-u_k)
    wherever u jumps, and sum_i (u_i - f_i) = 0."""
    n, alpha = 40, 2.0
    rng = np.random.Generator(np.random.PCG64(12))
    f = np.repeat(rng.uniform(0, 3, 5), 8) + 0.4 * rng.standard_normal(n)
    A = sp.identity(n, format="csr")
    res = tv.split_bregman(A, f, (n, 1), alpha, 0.5, outer=3000, inner=200, cg_tol=1e-14)
    u = res["u"].ravel()
    z = alpha * np.cumsum(u - f)
    assert abs(z[-1]) <= 1e-8
    z = z[:-1]
    du = np.diff(u)
    assert np.all(np.abs(z) <= 1.0 + 1e-7)
    jumps = np.abs(du) > 1e-8
    assert jumps.any() and not jumps.all()
    np.testing.assert_allclose(z[jumps], np.sign(du[jumps]), atol=1e-6)


def test_sb_constant_image_is_a_fixed_point():
    n = 16
    A = _small_problem(n)
    u_true = np.full((n, n), 0.7)
    f = A @ u_true.ravel()
    res = tv.split_bregman(A, f, (n, n), 1.0, 1.0, outer=5, inner=10, u0=u_true)
    np.testing.assert_allclose(res["u"], u_true, atol=1e-13)
    for key in ("dx", "dy", "bx", "by"):
        assert np.abs(res[key]).max() <= 1e-13


def test_sb_update_size_is_the_l1_norm_in_closed_form():
    """Sec. 4 measures each Bregman update by its L1 norm.  With A = I and
    constant data f = c on an n x 1 image, grad f = 0, so the first CG step
    from u = 0 lands exactly on u = f (step size 1/alpha) and the residual is
    zero: the first update is n |c| in L1 (sqrt(n) |c| in L2, n c if signed),
    and the second is 0."""
    n, c = 40, -0.5
    A = sp.identity(n, format="csr")
    res = tv.split_bregman(A, np.full(n, c), (n, 1), 2.0, 0.5, outer=2, inner=5)
    np.testing.assert_array_equal(res["u"].ravel(), np.full(n, c))
    assert res["updates"] == [n * abs(c), 0.0]


def test_stop_rule_ends_at_the_first_update_below_tol_times_the_first():
    """Sec. 4's stopping rule: the run ends after the first update whose L1
    size is below tol times the first update's (not the previous one's: the
    sizes here are not monotone), holding the uninterrupted run's iterate."""
    n = 16
    A = _small_problem(n)
    f = A @ inputs.ellipse_phantom(n, 17).ravel()
    full = tv.split_bregman(A, f, (n, n), 1.0, 0.5, outer=60, inner=5)
    U = np.array(full["updates"])
    tol = 0.05
    k = int(np.argmax(U < tol * U[0])) + 1
    assert 2 < k < 60 and np.any(np.diff(U[:k]) > 0)
    stop = tv.split_bregman(A, f, (n, n), 1.0, 0.5, outer=60, inner=5, stop_rel_update=tol)
    assert stop["outer_done"] == k and len(stop["updates"]) == k
    part = tv.split_bregman(A, f, (n, n), 1.0, 0.5, outer=k, inner=5)
    np.testing.assert_array_equal(stop["u"], part["u"])


def test_tv_objective_in_closed_form():
    """Eq. objmin with p = 1, K = grad (anisotropic), on a 2 x 2 image with
    A = I, f = 1 and alpha = 2: the residual u - f = (0, 2, -1, -3) gives
    (2/2) 14 = 14, the differences 3-1, -2-0 (along x) and 0-1, -2-3 (along
    y) give 2 + 2 + 1 + 5 = 10."""
    A = sp.identity(4, format="csr")
    u = np.array([[1.0, 3.0], [0.0, -2.0]])
    assert tv.tv_objective(A, np.ones(4), u, 2.0) == 24.0


def test_sb_limit_satisfies_tv_kkt_conditions():
    """At convergence z = lambda b certifies optimality of u for
    min alpha/2 ||A u - f||^2 + ||grad u||_1: |z| <= 1, z = sign(grad u) where
    grad u != 0, alpha A^T (A u - f) + grad^T z = 0; and u beats nearby points."""
    n, alpha, lam = 8, 0.3, 2.0
    A = radon.siddon_matrix(n, 12, 1, inputs.n_bins_for(n))
    truth = inputs.ellipse_phantom(n, 3)
    f = A @ truth.ravel() + 0.3 * inputs.standard_normal(A.shape[0], 4)
    res = tv.split_bregman(A, f, (n, n), alpha, lam, outer=1500, inner=300, cg_tol=1e-14)
    u = res["u"]
    assert res["updates"][-1] <= 1e-10 * res["updates"][0]
    zx, zy = lam * res["bx"], lam * res["by"]
    gx, gy = tv.grad(u)
    assert max(np.abs(zx).max(), np.abs(zy).max()) <= 1.0 + 1e-8
    for g, z in ((gx, zx), (gy, zy)):
        nz = np.abs(g) > 1e-7
        np.testing.assert_allclose(z[nz], np.sign(g[nz]), atol=1e-6)
    stat = alpha * (A.T @ (A @ u.ravel() - f)) + tv.grad_adj(zx, zy).ravel()
    assert np.abs(stat).max() <= 1e-7
    F0 = tv.tv_objective(A, f, u, alpha)
    rng = np.random.Generator(np.random.PCG64(13))
    for eps in (1e-3, 1e-5):
        for _ in range(20):
            v = rng.standard_normal(u.shape)
            assert tv.tv_objective(A, f, u + eps * v, alpha) >= F0 - 1e-12 * abs(F0)


def test_resolvent_identity_case_and_dense_solve():
    n = 16
    A = _small_problem(n)
    ut = inputs.random_vector(n * n, 14).reshape(n, n)
    g = inputs.random_vector(A.shape[0], 15)
    # tau alpha = 0: the resolvent is the identity, the solution is u_tilde
    u, _ = tv.resolvent(A, (n, n), 0.0, 1.0, ut, g, 3, u0=np.zeros(n * n))
    np.testing.assert_allclose(u, ut.ravel(), atol=1e-14)
    tau, alpha = 0.02, 1.0
    u, st = tv.resolvent(A, (n, n), tau, alpha, ut, g, 500)
    M = _dense_op(A, n, 1.0, tau * alpha, 0.0)
    want = np.linalg.solve(M, ut.ravel() + tau * alpha * (A.T @ g))
    assert np.linalg.norm(u - want) <= 1e-9 * np.linalg.norm(want)


@pytest.mark.parametrize("r,shape,ntaps", [(1, "disc", 5), (3, "disc", 29), (2, "square", 25)])
def test_surrogate_matrix_is_sum_of_translates(r, shape, ntaps):
    n = 32
    A = radon.siddon_matrix(n, 40, 1, inputs.n_bins_for(n))
    h = tv.point_response(A, n)
    taps = tv.surrogate_stencil(h, r, shape)
    assert len(taps) == ntaps
    T = tv.surrogate_matrix(taps, n)
    # symmetric to the last bit
    assert (T - T.T).count_nonzero() == 0
    # column c holds the truncated, symmetrised point response
    c = (n // 2) * n + n // 2
    col = T[:, c].toarray().ravel().reshape(n, n)
    for (di, dj), v in taps.items():
        assert col[n // 2 + di, n // 2 + dj] == v
        assert v == 0.5 * (h[n // 2 + di, n // 2 + dj] + h[n // 2 - di, n // 2 - dj])
    assert np.count_nonzero(col) <= ntaps
    # T u equals a zero-padded correlation with the stencil (independent library path)
    K = np.zeros((2 * r + 1, 2 * r + 1))
    for (di, dj), v in taps.items():
        K[r + di, r + dj] = v
    u = inputs.random_vector(n * n, 16).reshape(n, n)
    want = ssig.correlate2d(u, K[::-1, ::-1], mode="same", boundary="fill")
    np.testing.assert_allclose((T @ u.ravel()).reshape(n, n), want, atol=1e-11)


def test_point_response_is_column_of_normal_matrix():
    n = 16
    A = _small_problem(n)
    h = tv.point_response(A, n)
    Ad = A.toarray()
    np.testing.assert_allclose(h.ravel(), (Ad.T @ Ad)[:, (n // 2) * n + n // 2], atol=1e-13)


def test_surrogate_reconstruction_is_less_accurate_and_improves_with_r():
    """Sec. 4 (Tables of fixed-iteration error, and the r = 3 remark): after a
    fixed number of updates the surrogate reconstruction is further from the
    exact-operator one, and a larger r brings it closer."""
    n = 64
    A = radon.siddon_matrix(n, 90, 3, 91)
    truth = inputs.ellipse_phantom(n, 0)
    f = A @ truth.ravel()
    exact = tv.split_bregman(A, f, (n, n), 1.0, 1.0, outer=20, inner=10)["u"]
    h = tv.point_response(A, n)
    errs = []
    for r in (1, 3):
        T = tv.surrogate_matrix(tv.surrogate_stencil(h, r), n)
        u = tv.split_bregman(A, f, (n, n), 1.0, 1.0, outer=20, inner=10, normal=lambda x: T @ x)["u"]
        errs.append(np.abs(u - truth).sum() / np.abs(truth).sum())
    err_exact = np.abs(exact - truth).sum() / np.abs(truth).sum()
    assert errs[0] > err_exact and errs[1] > err_exact
    assert errs[1] < errs[0]


@pytest.mark.parametrize("r", [1, 3])
def test_surrogate_image_mass_follows_the_dropped_response(r):
    """Why the surrogate misses in this setting: summing the surrogate system
    over all pixels (1^T grad^T = 0) gives sum(s) * sum(u) ~ sum over pixels of
    (A^T A 1) times the phantom ~ sum(h) * sum(truth) for an object away from
    the edges, so the reconstruction's mass is sum(h) / sum(s) times the
    phantom's (h the whole point response, s the window's taps)."""
    n = 64
    A = radon.siddon_matrix(n, 90, 3, 91)
    truth = inputs.ellipse_phantom(n, 0)
    f = A @ truth.ravel()
    h = tv.point_response(A, n)
    taps = tv.surrogate_stencil(h, r)
    T = tv.surrogate_matrix(taps, n)
    u = tv.split_bregman(A, f, (n, n), 1.0, 1.0, 20, 10, normal=lambda x: T @ x)["u"]
    ratio = h.sum() / sum(taps.values())
    assert ratio > 10.0
    assert abs(u.sum() / truth.sum() / ratio - 1.0) <= 0.1


def _complex_step(A, f, shape, alpha, lam, outer, inner, w, d, h=1e-30):
    u = tv.split_bregman(A, f + 1j * h * d, shape, alpha, lam, outer, inner)["u"].ravel()
    return float(np.imag(w @ u)) / h


def test_complex_step_derivative_matches_finite_differences():
    """Complex-step differentiation of the oracle's unrolled split Bregman
    (used as the FP64 derivative reference at sizes where real differences
    drown in rounding) agrees with central differences on a small case, and
    its real part is the unperturbed reconstruction."""
    n = 24
    A = radon.siddon_matrix(n, 30, 1, inputs.n_bins_for(n))
    f = A @ inputs.ellipse_phantom(n, 11).ravel() + 0.05 * inputs.standard_normal(A.shape[0], 12)
    w = inputs.random_vector(n * n, 13)
    rng = np.random.Generator(np.random.PCG64(14))
    for _ in range(4):
        d = rng.standard_normal(f.size)
        cs = _complex_step(A, f, (n, n), 1.0, 1.0, 4, 5, w, d)
        L = lambda h: float(w @ tv.split_bregman(A, f + h * d, (n, n), 1.0, 1.0, 4, 5)["u"].ravel())
        fd = [(L(h) - L(-h)) / (2 * h) for h in (1e-5, 5e-6)]
        if abs(fd[0] - fd[1]) > 1e-6 * abs(fd[1]):
            continue  # the segment crosses a shrink kink
        assert abs(cs - fd[1]) <= 1e-6 * abs(fd[1])
    u_c = tv.split_bregman(A, f + 1j * 1e-30 * d, (n, n), 1.0, 1.0, 4, 5)["u"]
    u_r = tv.split_bregman(A, f, (n, n), 1.0, 1.0, 4, 5)["u"]
    np.testing.assert_allclose(np.real(u_c), u_r, rtol=0, atol=1e-12 * np.abs(u_r).max())


def test_complex_step_of_linear_solve_is_exact():
    """The p = 2 normal equations: CG run to convergence is linear in the rhs,
    so the complex-step derivative equals the solve applied to the direction."""
    n = 12
    A = radon.siddon_matrix(n, 16, 1, inputs.n_bins_for(n))
    op = tv.make_operator(A, (n, n), 0.0, 1.0, 1.0)
    rhs = inputs.random_vector(n * n, 15)
    d = inputs.random_vector(n * n, 16)
    u_c, _ = tv.cg(op, rhs + 1j * 1e-30 * d, np.zeros(n * n), 400, rel_tol=1e-14)
    want, _ = tv.cg(op, d, np.zeros(n * n), 400, rel_tol=1e-14)
    np.testing.assert_allclose(np.imag(u_c) / 1e-30, want, rtol=0, atol=1e-8 * np.abs(want).max())


def test_chambolle_pock_reaches_the_split_bregman_minimiser_with_a_kkt_certificate():
    """Chambolle-Pock (dual projection, resolvent of Eq. PD_resolve, theta = 1)
    and split Bregman are different algorithms for the same objective
    alpha/2 ||A u - f||^2 + ||grad u||_1: both limits must coincide, and CP's
    dual p must certify optimality (|p| <= 1, p = sign(grad u) where
    grad u != 0, alpha A^T (A u - f) + grad^T p = 0)."""
    n, alpha, lam = 8, 0.3, 2.0
    A = radon.siddon_matrix(n, 12, 1, inputs.n_bins_for(n))
    truth = inputs.ellipse_phantom(n, 3)
    f = A @ truth.ravel() + 0.3 * inputs.standard_normal(A.shape[0], 4)
    sb = tv.split_bregman(A, f, (n, n), alpha, lam, outer=1500, inner=300, cg_tol=1e-14)
    step = 0.99 / np.sqrt(8.0)
    cp = tv.chambolle_pock(A, f, (n, n), alpha, step, step, outer=2000, inner=100)
    u = cp["u"]
    assert np.linalg.norm(u - sb["u"]) <= 1e-8 * np.linalg.norm(sb["u"])
    px, py = cp["px"], cp["py"]
    assert max(np.abs(px).max(), np.abs(py).max()) <= 1.0
    gx, gy = tv.grad(u)
    for g, p in ((gx, px), (gy, py)):
        nz = np.abs(g) > 1e-7
        assert nz.any()
        np.testing.assert_allclose(p[nz], np.sign(g[nz]), atol=1e-6)
    stat = alpha * (A.T @ (A @ u.ravel() - f)) + tv.grad_adj(px, py).ravel()
    assert np.abs(stat).max() <= 1e-7


def test_chambolle_pock_two_steps_in_closed_form():
    """Two primal-dual steps by hand on a 1 x 2 image with A = I, g = (0, 1),
    alpha = 1, tau = sigma = 1/2 (each resolvent is (3/2) u = rhs, exact after
    one CG step): u1 = (0, 1/3), extrapolated ubar1 = (0, 2/3), dual
    p_x = clip(sigma 2/3) = 1/3, grad^T p = (-1/3, 1/3), u2 = ((1/6, 1/6) +
    (0, 1/2)) / (3/2) = (1/9, 4/9).  Without the extrapolation u2 would be
    (1/18, 1/2)."""
    r = tv.chambolle_pock(sp.identity(2, format="csr"), np.array([0.0, 1.0]), (1, 2), 1.0, 0.5, 0.5, 2, 3)
    np.testing.assert_allclose(r["u"].ravel(), [1.0 / 9.0, 4.0 / 9.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r["px"].ravel(), [1.0 / 3.0, 0.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r["updates"], [1.0 / 3.0, 2.0 / 9.0], rtol=1e-15)


def test_chambolle_pock_constant_image_is_a_fixed_point():
    n = 16
    A = _small_problem(n)
    u_true = np.full((n, n), 0.7)
    f = A @ u_true.ravel()
    res = tv.chambolle_pock(A, f, (n, n), 1.0, 0.3, 0.3, outer=5, inner=10, u0=u_true)
    np.testing.assert_allclose(res["u"], u_true, atol=1e-13)
    assert np.abs(res["px"]).max() == 0.0 and np.abs(res["py"]).max() == 0.0
