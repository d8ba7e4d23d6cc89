"""Pins of the Fourier-domain oracle (Sec. 2, Eq. four_obj; Sec. 3.1, Eq.
fusedop) against the definitions, a library FFT and the accuracy the paper
states for Gaussian gridding."""

import math
import os

import numpy as np
import pytest

from oracle import fourier as fo
from oracle import radon, tv

GEOMS = [(16, 24, 1, 23), (32, 40, 2, 46)]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gridding_accuracy.txt")


def _stated_accuracy():
    """(m_sp, bound) rows of the paper's accuracy statement (tests/golden)."""
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                m_sp, digits, bound = line.split()
                assert float(bound) <= 50.0 * 10.0 ** -int(digits)
                rows.append((int(m_sp), float(bound)))
    return rows


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("geom", GEOMS)
@pytest.mark.parametrize("m_sp,bound", [(2, 3e-2)] + _stated_accuracy())
def test_gridding_meets_the_stated_accuracy(geom, m_sp, bound):
    """Sec. 3.1: M_sp = 6, tau = 6/N^2 gives 6 digits, M_sp = 12, tau = 12/N^2
    gives 12 (tests/golden/gridding_accuracy.txt); forward, adjoint and the
    fused normal operator against the brute nonuniform DFT (M_sp = 2, which
    the paper does not rate: about two digits)."""
    n = geom[0]
    rng = np.random.default_rng(7)
    F = fo.nudft_matrix(*geom)
    mu = rng.standard_normal(n * n)
    c = rng.standard_normal(F.shape[0]) + 1j * rng.standard_normal(F.shape[0])
    g = fo.Gridding(*geom, m_sp)
    assert _rel(g.forward(mu), F @ mu) <= bound
    assert _rel(g.adjoint(c), np.real(F.conj().T @ c)) <= bound
    assert _rel(g.normal_fused(mu), np.real(F.conj().T @ (F @ mu))) <= bound


def test_accuracy_grows_with_the_window():
    geom = GEOMS[0]
    n = geom[0]
    F = fo.nudft_matrix(*geom)
    mu = np.random.default_rng(8).standard_normal(n * n)
    errs = [_rel(fo.Gridding(*geom, m).forward(mu), F @ mu) for m in (2, 4, 6, 8, 12)]
    assert all(b < a for a, b in zip(errs, errs[1:]))


@pytest.mark.parametrize("geom", GEOMS)
def test_type1_is_the_adjoint_of_type2(geom):
    n = geom[0]
    rng = np.random.default_rng(9)
    g = fo.Gridding(*geom, 4)
    mu = rng.standard_normal(n * n)
    c = rng.standard_normal(len(g.wx)) + 1j * rng.standard_normal(len(g.wx))
    lhs = np.real(np.vdot(c, g.forward(mu)))
    rhs = float(mu @ g.adjoint(c))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(mu) * np.linalg.norm(c)


@pytest.mark.parametrize("geom", GEOMS)
def test_fused_matrix_reproduces_the_two_gridding_steps(geom):
    """Convolution fusing changes the association only: C = G^T G applied
    between the FFTs equals interpolation followed by spreading."""
    n = geom[0]
    g = fo.Gridding(*geom, 6)
    mu = np.random.default_rng(10).standard_normal(n * n)
    assert _rel(g.normal_fused(mu), g.normal(mu)) <= 1e-13


def test_fused_matrix_structure():
    """C is symmetric and its entries lie on the periodic offsets |d| <= 2 M_sp."""
    g = fo.Gridding(16, 24, 1, 23, 2)
    C = g.fused_matrix().tocoo()
    assert abs(C - C.T).max() <= 1e-15 * abs(C).max()
    m_r = g.m_r

    def wrap(d):
        return np.minimum(d % m_r, (-d) % m_r)

    dx = wrap((C.col % m_r) - (C.row % m_r))
    dy = wrap((C.col // m_r) - (C.row // m_r))
    assert dx.max() <= 2 * g.m_sp and dy.max() <= 2 * g.m_sp


@pytest.mark.parametrize("n_bins", [23, 24])
def test_sinogram_dft_is_a_shifted_library_fft(n_bins):
    """fhat = n^{-1/2} sum_b f_b exp(-i rho_m s_b) is numpy's FFT with the
    frequency index shifted by floor(n/2) and the phase of the bin centring."""
    rng = np.random.default_rng(11)
    f = rng.standard_normal((5, n_bins))
    got = fo.sinogram_dft(f, 5, n_bins).reshape(5, n_bins)
    X = np.fft.fft(f, axis=1)
    h = n_bins // 2
    m = np.arange(n_bins) - h
    want = X[:, m % n_bins] * np.exp(1j * math.pi * m * (n_bins - 1) / n_bins) / math.sqrt(n_bins)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_data_transform_and_operator_agree_on_a_pixel():
    """With an even number of bins the bin centres at theta = 0 and pi/2 are
    the pixel centres: a pixel's projection there is one unit bin, and the DFT
    of that sinogram row equals the operator's column on those samples."""
    n, n_total, ke, nb = 8, 4, 1, 12
    F = fo.nudft_matrix(n, n_total, ke, nb)
    A = radon.siddon_matrix(n, n_total, ke, nb).toarray()
    for p in (0, 19, 45, 63):
        e = np.zeros(n * n)
        e[p] = 1.0
        sino = A @ e
        fh = fo.sinogram_dft(sino, n_total, nb).reshape(n_total, nb)
        col = (F @ e).reshape(n_total, nb)
        for k in (0, 2):  # theta = 0 and pi/2
            assert np.allclose(sino.reshape(n_total, nb)[k].sum(), 1.0)
            assert np.abs(fh[k] - col[k]).max() <= 1e-13


def test_point_response_is_the_normal_operator_column():
    """The closed form n_bins^-1 sum_j cos(omega_j . d) is column c of
    Re(F^H F), and the exact system's normal operator applied to the unit
    image at c (off the image centre, so a point reflection of the image
    would show) gives that column."""
    n, geom = 16, (16, 24, 1, 23)
    F = fo.nudft_matrix(*geom)
    c = (n // 2) * n + n // 2
    col = np.real(F.conj().T @ F[:, c]).reshape(n, n)
    h = fo.point_response(*geom, 3)
    win = (slice(n // 2 - 3, n // 2 + 4), slice(n // 2 - 3, n // 2 + 4))
    assert np.abs(h - col[win]).max() <= 1e-13
    e = np.zeros(n * n)
    e[c] = 1.0
    got = fo.FourierSystem(*geom).normal(e).reshape(n, n)
    assert np.abs(h - got[win]).max() <= 1e-13


def test_exact_system_adjoint_identity():
    """Re <F mu, c> = <mu, Re(F^H c)> for a real image mu and complex c."""
    geom = (16, 24, 1, 23)
    S = fo.FourierSystem(*geom)
    rng = np.random.default_rng(21)
    mu = rng.standard_normal(16 * 16)
    c = rng.standard_normal(24 * 23) + 1j * rng.standard_normal(24 * 23)
    lhs = float(np.real(np.vdot(c, S @ mu)))
    rhs = float(mu @ (S.T @ c))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_cg_on_the_fourier_system_solves_the_dense_normal_equations():
    """CG on alpha Re(F^H F) + lambda grad^T grad (the system of Eq. SBFFT
    with the sign read as +), with the gridded operator at M_sp = 12, against
    a dense solve built from the brute-force F."""
    geom = (16, 24, 1, 23)
    n = geom[0]
    shape = (n, n)
    rng = np.random.default_rng(12)
    rhs = rng.standard_normal(n * n)
    g = fo.Gridding(*geom, 12)
    op = tv.make_operator(None, shape, 0.0, 1.0, 0.5, normal=g.normal_fused)
    u, st = tv.cg(op, rhs, np.zeros(n * n), 400, rel_tol=1e-13)
    F = fo.nudft_matrix(*geom)
    L = np.zeros((n * n, n * n))
    for q in range(n * n):
        e = np.zeros(n * n)
        e[q] = 1.0
        gx, gy = tv.grad(e.reshape(shape))
        L[:, q] = tv.grad_adj(gx, gy).ravel()
    dense = np.real(F.conj().T @ F) + 0.5 * L
    assert _rel(u, np.linalg.solve(dense, rhs)) <= 1e-8


def test_fourier_split_bregman_runs_on_the_system():
    """The generic split-Bregman oracle on the Fourier system: gridded (M_sp =
    12) and exact operators give the same iterates to near the gridding
    accuracy over two updates (longer fixed-count runs amplify the 1e-11
    operator difference, as they amplify any rounding)."""
    geom = (16, 24, 1, 23)
    n = geom[0]
    A = radon.siddon_matrix(*geom)
    x = np.zeros((n, n))
    x[5:11, 3:12] = 1.0  # not symmetric about the image centre
    x[6, 9] = 2.0
    fhat = fo.sinogram_dft(A @ x.ravel(), 24, 23)
    exact = fo.FourierSystem(*geom)
    grid = fo.FourierSystem(*geom, gridding=fo.Gridding(*geom, 12))
    a = tv.split_bregman(exact, fhat, (n, n), 1.0, 1.0, 2, 5, normal=exact.normal)
    b = tv.split_bregman(grid, fhat, (n, n), 1.0, 1.0, 2, 5, normal=grid.normal)
    assert _rel(b["u"], a["u"]) <= 1e-9
    assert a["updates"][0] > 0


def _stencil_symbol_min(h, r, rr, square):
    """min over frequencies of the symmetrised truncated stencil plus the
    grad^T grad symbol (alpha = lambda = 1): the surrogate system's symbol."""
    w = np.linspace(-math.pi, math.pi, 257)
    WX, WY = np.meshgrid(w, w)
    sym = 4.0 - 2.0 * np.cos(WX) - 2.0 * np.cos(WY)
    for di in range(-rr, rr + 1):
        for dj in range(-rr, rr + 1):
            if square or di * di + dj * dj <= rr * rr:
                sym = sym + 0.5 * (h[r + di, r + dj] + h[r - di, r - dj]) * np.cos(WX * dj + WY * di)
    return float(sym.min())


def test_truncated_fourier_point_response_definiteness():
    """The Fourier normal operator's point response decays like 1/|d| (the
    polar samples crowd the origin), so truncating it can make the surrogate
    system indefinite: at N = 128 with N pi / 4 angles the disc of radius 1
    and the windows of radius 3 are indefinite, the 3 x 3 square and the disc
    of radius 2 are positive (the windows the experiment replay uses)."""
    h = fo.point_response(128, 101, 1, 182, 3)
    assert _stencil_symbol_min(h, 3, 1, False) < 0
    assert _stencil_symbol_min(h, 3, 3, False) < 0
    assert _stencil_symbol_min(h, 3, 3, True) < 0
    assert _stencil_symbol_min(h, 3, 1, True) > 0
    assert _stencil_symbol_min(h, 3, 2, False) > 0
