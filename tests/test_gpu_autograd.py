"""Differentiation: autograd Functions over A / A^T and the unrolled,
checkpointed split Bregman, checked against FP64 finite differences of the
oracle and against the oracle's reconstruction.

Finite differences: central differences of the FP64 oracle with Richardson
extrapolation at h = 2e-4 and 1e-4 (h = 1e-6 is dominated by the oracle's own
rounding on these workloads); directions whose two estimates disagree are
treated as crossing a shrink kink and skipped (at most a quarter of them).
"""

import functools

import numpy as np
import pytest

from oracle import radon, tv
from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


@functools.lru_cache(maxsize=None)
def oracle_A(*geom):
    return radon.siddon_matrix(*geom)


@functools.lru_cache(maxsize=None)
def gpu_A(*geom):
    return ct.Matrix(*geom)


def test_radon_functions_pass_gradcheck(dev):
    from paper_1705_07497_gb300.autograd import radon, radon_adjoint

    M = gpu_A(16, 12, 1, 23)
    x = torch.tensor(inputs.random_vector(M.cols * 2, 70).reshape(M.cols, 2), dtype=torch.float64,
                     device=dev, requires_grad=True)
    y = torch.tensor(inputs.random_vector(M.rows * 2, 71).reshape(M.rows, 2), dtype=torch.float64,
                     device=dev, requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: radon(M, t), (x,), eps=1e-6, atol=1e-8, rtol=1e-6)
    assert torch.autograd.gradcheck(lambda t: radon_adjoint(M, t), (y,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_f64_products_match_oracle(dev):
    geom = (64, 90, 3, 91)
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    for batch in (1, 3):
        x = inputs.random_vector(M.cols * batch, 72).reshape(M.cols, batch)
        y = torch.empty((M.rows, batch), dtype=torch.float64, device=dev)
        M.forward(torch.tensor(x, device=dev), y)
        want = ref @ x
        assert np.linalg.norm(y.cpu().numpy() - want) <= 1e-12 * np.linalg.norm(want)


def _sb_oracle(A, f, n, outer, inner):
    return tv.split_bregman(A, f, (n, n), 1.0, 1.0, outer, inner)["u"].ravel()


def _fd(A, f, n, outer, inner, w, d):
    def L(h):
        return float(w @ _sb_oracle(A, f + h * d, n, outer, inner))
    est = []
    for h in (2e-4, 1e-4):
        est.append((L(h) - L(-h)) / (2 * h))
    rich = (4 * est[1] - est[0]) / 3
    return rich, abs(est[0] - est[1]) / max(abs(rich), 1e-30)


def _check_gradient(dev, geom, seed, outer, inner, ndir, tol):
    from paper_1705_07497_gb300.autograd import split_bregman_unrolled

    n = geom[0]
    A = oracle_A(*geom)
    M = gpu_A(*geom)
    truth = inputs.ellipse_phantom(n, seed)
    f = inputs.gaussian_noisy(A @ truth.ravel(), 0.01, seed + 1)
    w = inputs.random_vector(n * n, seed + 2)
    ft = torch.tensor(f, dtype=torch.float64, device=dev, requires_grad=True)
    u = split_bregman_unrolled(M, ft, 1.0, 1.0, outer, inner)
    # forward parity with the oracle
    want = _sb_oracle(A, f, n, outer, inner)
    got = u.detach().cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-8 * np.linalg.norm(want)
    (torch.tensor(w, device=dev) * u).sum().backward()
    g = ft.grad.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(seed + 3))
    checked, skipped = 0, 0
    while checked < ndir:
        d = rng.standard_normal(f.size)
        fd, spread = _fd(A, f, n, outer, inner, w, d)
        if spread > 1e-3:
            skipped += 1
            assert skipped <= ndir // 4 + 1, "too many directions cross a shrink kink"
            continue
        ad = float(g @ d)
        assert abs(ad - fd) <= tol * abs(fd), (ad, fd)
        checked += 1


def test_unrolled_gradient_small(dev):
    _check_gradient(dev, (32, 40, 1, 46), 77, outer=5, inner=5, ndir=8, tol=1e-5)


def test_unrolled_gradient_256(dev):
    """256x256, 180 of 360 angles, 363 bins, 10 unrolled updates of 10 CG steps."""
    _check_gradient(dev, (256, 360, 2, 363), 3000, outer=10, inner=10, ndir=3, tol=1e-4)


def test_checkpointing_does_not_change_the_gradient(dev):
    from paper_1705_07497_gb300.autograd import split_bregman_unrolled

    geom = (64, 90, 3, 91)
    M = gpu_A(*geom)
    A = oracle_A(*geom)
    F = np.stack([A @ inputs.ellipse_phantom(64, s).ravel() for s in (1, 2, 3)], axis=1)
    grads = []
    for ck in (True, False):
        ft = torch.tensor(F, dtype=torch.float64, device=dev, requires_grad=True)
        u = split_bregman_unrolled(M, ft, 1.0, 0.5, 4, 5, use_checkpoint=ck)
        (u * u).sum().backward()
        grads.append(ft.grad.clone())
    assert torch.equal(grads[0], grads[1])


def test_batched_unrolled_16_slices(dev):
    """16 slices of 256x256 in one differentiable call; slice 5 against the oracle."""
    from paper_1705_07497_gb300.autograd import split_bregman_unrolled

    geom = (256, 360, 2, 363)
    M = gpu_A(*geom)
    A = oracle_A(*geom)
    F = np.stack([inputs.gaussian_noisy(A @ inputs.ellipse_phantom(256, 3000 + s).ravel(), 0.01, 3100 + s)
                  for s in range(16)], axis=1)
    ft = torch.tensor(F, dtype=torch.float64, device=dev, requires_grad=True)
    u = split_bregman_unrolled(M, ft, 1.0, 1.0, 10, 10)
    u.sum().backward()
    assert torch.isfinite(ft.grad).all()
    want = _sb_oracle(A, F[:, 5], 256, 10, 10)
    got = u[:, 5].detach().cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-8 * np.linalg.norm(want)
