"""Differentiation: autograd Functions over A / A^T and the unrolled,
checkpointed split Bregman, checked against FP64 derivatives of the oracle
and against the oracle's reconstruction.

Derivative references: on a small case, central differences of the FP64
oracle with Richardson extrapolation at h = 2e-4 and 1e-4 (directions whose
two estimates disagree cross a shrink kink and are skipped); at 256x256 real
differences drown in the oracle's own amplified rounding at every usable h,
so the reference there is the oracle's complex-step derivative
Im(L(f + i h d)) / h with h = 1e-30 (no subtractive cancellation, and the
real trajectory, hence every shrink decision, is the unperturbed one).
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
def oracle_A32(*geom):
    """The oracle's matrix with its values rounded to FP32: what the library stores."""
    A = oracle_A(*geom).copy()
    A.data = A.data.astype(np.float32).astype(np.float64)
    return A


@functools.lru_cache(maxsize=None)
def gpu_A(*geom, flags=0):
    return ct.Matrix(*geom, flags=flags)


# FP64-vector products: double-float on the FP32 pipes (default) or the FP64 pipe
F64_PATHS = [pytest.param(0, id="double-float"), pytest.param(ct.CT_F64_FP64_PIPE, id="fp64-pipe")]


@pytest.mark.parametrize("flags", F64_PATHS)
def test_radon_functions_pass_gradcheck(dev, flags):
    from paper_1705_07497_gb300.autograd import radon, radon_adjoint

    M = gpu_A(16, 12, 1, 23, flags=flags)
    x = torch.tensor(inputs.random_vector(M.cols * 2, 70).reshape(M.cols, 2), dtype=torch.float64,
                     device=dev, requires_grad=True)
    y = torch.tensor(inputs.random_vector(M.rows * 2, 71).reshape(M.rows, 2), dtype=torch.float64,
                     device=dev, requires_grad=True)
    # both maps are linear, so a central difference is exact up to rounding at
    # any step; a step of 1e-3 keeps the products' rounding (about 1e-14 of
    # the output in double-float) well below the tolerance once divided by it
    assert torch.autograd.gradcheck(lambda t: radon(M, t), (x,), eps=1e-3, atol=1e-8, rtol=1e-6)
    assert torch.autograd.gradcheck(lambda t: radon_adjoint(M, t), (y,), eps=1e-3, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("flags", F64_PATHS)
def test_f64_products_match_oracle(dev, flags):
    geom = (64, 90, 3, 91)
    ref = oracle_A32(*geom)
    M = gpu_A(*geom, flags=flags)
    for batch in (1, 3):
        x = inputs.random_vector(M.cols * batch, 72).reshape(M.cols, batch)
        y = torch.empty((M.rows, batch), dtype=torch.float64, device=dev)
        M.forward(torch.tensor(x, device=dev), y)
        want = ref @ x
        assert np.linalg.norm(y.cpu().numpy() - want) <= 1e-12 * np.linalg.norm(want)


def test_batched_f64_product_variants_are_bit_identical(dev):
    """Double-float FP64-vector products over 3 slices: every staged-entry
    unroll gives the same bits, and the first product tunes it."""
    geom = (64, 90, 3, 91)
    x = torch.tensor(inputs.random_vector(4096 * 3, 76).reshape(4096, 3), dtype=torch.float64, device=dev)
    ys = []
    for unroll in (4, 8, 16, 0):
        M = ct.Matrix(*geom)
        if unroll:
            M.set_spmm_unroll(3, unroll)
        y = torch.empty((M.rows, 3), dtype=torch.float64, device=dev)
        M.forward(x, y)
        xa = torch.empty_like(x)
        M.adjoint(y, xa)
        torch.cuda.synchronize()
        if not unroll:
            assert M.spmm_unroll(3) in (4, 8, 16)
        ys.append((y.cpu(), xa.cpu()))
        M.close()
    for y, xa in ys[1:]:
        assert torch.equal(y, ys[0][0]) and torch.equal(xa, ys[0][1])


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


def _check_gradient(dev, geom, seed, outer, inner, ndir, tol, fwd_tol=1e-8, flags=0):
    from paper_1705_07497_gb300.autograd import split_bregman_unrolled

    n = geom[0]
    A = oracle_A(*geom)
    M = gpu_A(*geom, flags=flags)
    truth = inputs.ellipse_phantom(n, seed)
    f = inputs.gaussian_noisy(A @ truth.ravel(), 0.01, seed + 1)
    w = inputs.random_vector(n * n, seed + 2)
    ft = torch.tensor(f, dtype=torch.float64, device=dev, requires_grad=True)
    u = split_bregman_unrolled(M, ft, 1.0, 1.0, outer, inner)
    # forward parity with the oracle on the stored (FP32-valued) matrix
    want = _sb_oracle(oracle_A32(*geom), f, n, outer, inner)
    got = u.detach().cpu().numpy()
    assert np.linalg.norm(got - want) <= fwd_tol * np.linalg.norm(want)
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


@pytest.mark.parametrize("flags", F64_PATHS)
def test_unrolled_gradient_small(dev, flags):
    _check_gradient(dev, (32, 40, 1, 46), 77, outer=5, inner=5, ndir=8, tol=1e-5, flags=flags)


def _complex_step(A, f, n, outer, inner, w, d, h=1e-30):
    """d/dt of w . u(f + t d) at t = 0 by the oracle's complex step."""
    uc = tv.split_bregman(A, f + 1j * h * d, (n, n), 1.0, 1.0, outer, inner)["u"].ravel()
    return float(np.imag(w @ uc)) / h


def test_unrolled_gradient_256_on_32_directions(dev):
    """256x256, 180 of 360 angles, 363 bins, 10 unrolled updates of 10 CG steps
    (the differentiable workload's size): the autograd gradient with respect
    to the data against the oracle's complex-step derivative on 32 seeded
    directions, for both FP64-vector product paths (double-float and FP64
    pipe).  The complex step follows the unperturbed trajectory, so it
    differentiates the branch of every shrink that the reconstruction takes,
    as autograd does; no direction crosses a kink (R-AD1) in this form."""
    from oracle import spmv
    from paper_1705_07497_gb300.autograd import split_bregman_unrolled

    geom = (256, 360, 2, 363)
    n = 256
    A = oracle_A(*geom)
    A32 = oracle_A32(*geom)
    f = inputs.gaussian_noisy(A @ inputs.ellipse_phantom(n, 3000).ravel(), 0.01, 3001)
    w = inputs.random_vector(n * n, 3002)
    # 10 x 10 CG steps at this size amplify rounding ~1e6-fold (an FP64
    # perturbation of 1e-15 moves the oracle by 1e-9), and the derivative far
    # more (FP64 autograd on the CPU meets the complex-step value to ~1e-5)
    want = _sb_oracle(A32, f, n, 10, 10)
    grads = {}
    for name, flags in (("double-float", 0), ("fp64-pipe", ct.CT_F64_FP64_PIPE)):
        M = gpu_A(*geom, flags=flags)
        ft = torch.tensor(f, dtype=torch.float64, device=dev, requires_grad=True)
        u = split_bregman_unrolled(M, ft, 1.0, 1.0, 10, 10)
        got = u.detach().cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-7 * np.linalg.norm(want), name
        (torch.tensor(w, device=dev) * u).sum().backward()
        grads[name] = ft.grad.cpu().numpy()
    At = spmv.ThreadedCSR(A32)
    rng = np.random.Generator(np.random.PCG64(3003))
    errs = {name: [] for name in grads}
    for _ in range(32):
        d = rng.standard_normal(f.size)
        cs = _complex_step(At, f, n, 10, 10, w, d)
        for name, g in grads.items():
            errs[name].append(abs(float(g @ d) - cs) / abs(cs))
    for name, e in errs.items():
        print("FP64 vectors (%s products), 32 directions: max relative error of the directional derivative %.2e"
              % (name, max(e)))
        assert max(e) <= 1e-4, (name, e)


def test_unrolled_gradient_error_of_the_fp32_path(dev):
    """The same reconstruction and gradient with FP32 vectors and products (the
    library's FP32 ct_forward / ct_adjoint): the error against the oracle's
    complex-step derivative is stated, not bounded tightly; a fixed count of
    CG steps amplifies FP32 rounding of the iteration vectors (R-P2)."""
    from oracle import spmv
    from paper_1705_07497_gb300.autograd import split_bregman_unrolled

    geom = (256, 360, 2, 363)
    n = 256
    A = oracle_A(*geom)
    A32 = oracle_A32(*geom)
    M = gpu_A(*geom)
    f = inputs.gaussian_noisy(A @ inputs.ellipse_phantom(n, 3000).ravel(), 0.01, 3001)
    w = inputs.random_vector(n * n, 3002)
    ft = torch.tensor(f, dtype=torch.float32, device=dev, requires_grad=True)
    u = split_bregman_unrolled(M, ft, 1.0, 1.0, 10, 10)
    want = _sb_oracle(A32, f, n, 10, 10)
    fwd_err = float(np.linalg.norm(u.detach().cpu().double().numpy() - want) / np.linalg.norm(want))
    (torch.tensor(w, dtype=torch.float32, device=dev) * u).sum().backward()
    g = ft.grad.double().cpu().numpy()
    At = spmv.ThreadedCSR(A32)
    rng = np.random.Generator(np.random.PCG64(3003))
    errs = []
    for _ in range(8):
        d = rng.standard_normal(f.size)
        cs = _complex_step(At, f, n, 10, 10, w, d)
        errs.append(abs(float(g @ d) - cs) / abs(cs))
    print("FP32 path: reconstruction %.2e, directional derivative max %.2e median %.2e (8 directions)"
          % (fwd_err, max(errs), float(np.median(errs))))
    assert np.isfinite(g).all() and fwd_err < 1.0


@pytest.mark.parametrize("flags", F64_PATHS)
def test_fused_normal_operator_matches_its_composition_and_gradcheck(dev, flags):
    from paper_1705_07497_gb300.autograd import NormalOp, grad2d, grad2d_adj, radon, radon_adjoint

    M = gpu_A(64, 90, 3, 91, flags=flags)
    x = torch.tensor(inputs.random_vector(M.cols * 3, 74).reshape(M.cols, 3), dtype=torch.float64, device=dev)
    got = NormalOp.apply(M, x, 0.7, 0.3)
    want = 0.7 * radon_adjoint(M, radon(M, x)) + 0.3 * grad2d_adj(*grad2d(x, 64), 64)
    assert torch.linalg.norm(got - want) <= 1e-13 * torch.linalg.norm(want)
    S = gpu_A(16, 12, 1, 23, flags=flags)
    xs = torch.tensor(inputs.random_vector(S.cols * 2, 75).reshape(S.cols, 2), dtype=torch.float64, device=dev,
                      requires_grad=True)
    # linear as well: the same step as for the products
    assert torch.autograd.gradcheck(lambda t: NormalOp.apply(S, t, 1.3, 0.4), (xs,), eps=1e-3, atol=1e-8, rtol=1e-6)


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
    want = _sb_oracle(oracle_A32(*geom), F[:, 5], 256, 10, 10)
    got = u[:, 5].detach().cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-7 * np.linalg.norm(want)
