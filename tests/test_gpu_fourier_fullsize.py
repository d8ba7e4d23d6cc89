"""The Fourier-domain term at the size the Fourier bench runs (512 x 512,
180 of 720 angles, 725 bins, M_sp = 6, fused): sampled outputs of F x against
the nonuniform DFT by its definition, the normal operator against the
oracle's gridding, and the first Bregman update against the oracle."""

import numpy as np
import pytest

from oracle import fourier as fo
from oracle import radon, tv
from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GEOM = (512, 720, 4, 725)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def F(dev):
    h = ct.FourierMatrix(*GEOM, m_sp=6, mode=ct.CT_FOURIER_FUSED)
    yield h
    h.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_sampled_outputs_against_the_exact_dft(dev, F):
    """400 samples of F x against sum_p x_p exp(-i omega_j . c_p) / sqrt(n_bins):
    the six digits M_sp = 6 promises."""
    n = GEOM[0]
    x = inputs.ellipse_phantom(n, 1000).ravel()
    y = torch.empty(2 * F.rows, dtype=torch.float32, device=dev)
    F.forward(torch.tensor(x, dtype=torch.float32, device=dev), y)
    a = y.cpu().numpy().astype(np.float64)
    got = a[0::2] + 1j * a[1::2]
    rows = np.sort(np.random.Generator(np.random.PCG64(3)).choice(F.rows, 400, replace=False))
    wx, wy = fo.sample_points(*GEOM[1:])
    cx, cy = fo.pixel_centres(n)
    x32 = x.astype(np.float32).astype(np.float64)
    want = np.array([np.exp(-1j * (wx[j] * cx + wy[j] * cy)) @ x32 for j in rows]) / np.sqrt(GEOM[3])
    assert _rel(got[rows], want) <= 1e-5


def test_normal_operator_against_the_oracle(dev, F):
    n = GEOM[0]
    x = inputs.random_vector(n * n, 41).astype(np.float32).astype(np.float64)
    out = torch.empty(n * n, dtype=torch.float32, device=dev)
    F.normal(torch.tensor(x, dtype=torch.float32, device=dev), out)
    g = fo.Gridding(*GEOM, 6)
    assert _rel(out.cpu().double().numpy(), g.normal(x)) <= 1e-5


def test_first_update_against_the_oracle(dev, F):
    """One update of 20 CG steps (the bench's first update): the GPU within
    1e-4 of the FP64 oracle, whose own spread with the library's FP32
    weights is 3e-6."""
    n = GEOM[0]
    A = radon.siddon_matrix(*GEOM)
    f = inputs.gaussian_noisy(A @ inputs.ellipse_phantom(n, 1000).ravel(), 0.01, 1001)
    u = torch.zeros(n * n, dtype=torch.float32, device=dev)
    st = F.split_bregman(torch.tensor(f, dtype=torch.float32, device=dev), u, 1.0, 1.0, 1, 20)
    assert st["status"] == 0
    g = fo.Gridding(*GEOM, 6)
    S = fo.FourierSystem(*GEOM, gridding=g)
    fhat = fo.sinogram_dft(f, radon.num_kept(GEOM[1], GEOM[2]), GEOM[3])
    want = tv.split_bregman(S, fhat, (n, n), 1.0, 1.0, 1, 20, normal=g.normal)
    assert _rel(u.cpu().double().numpy(), want["u"].ravel()) <= 1e-4
