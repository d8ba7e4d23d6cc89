"""The Fourier-domain data term on the GPU (Sec. 2, Eqs. four_obj, SBFFT;
Sec. 3.1, Eq. fusedop) against the FP64 oracle with the same gridding
parameters.

Tolerances: the grid and sample vectors are double-float, but the tables
(weights, twiddles, E, the fused matrix) are FP32, a fixed perturbation of
the operator of about 1e-7 that the Gaussian deconvolution E(k) amplifies
towards the corners of the frequency square (E spans a factor exp(m_sp / 2)
per side): bounds 3e-6 at m_sp = 2 and 1e-4 at m_sp = 6, relative L2 against
the FP64 gridding."""

import functools

import numpy as np
import pytest

from oracle import fourier as fo
from oracle import radon, tv
from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GEOMS = [(32, 40, 2, 46), (64, 90, 1, 91)]
TOL = {2: 3e-6, 6: 1e-4}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


@functools.lru_cache(maxsize=None)
def oracle_grid(geom, m_sp):
    return fo.Gridding(*geom, m_sp)


@functools.lru_cache(maxsize=None)
def gpu_F(geom, m_sp, mode):
    return ct.FourierMatrix(*geom, m_sp=m_sp, mode=mode)


def rel(a, b):
    a = np.asarray(a)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def as_complex(t):
    a = t.cpu().numpy().astype(np.float64)
    return a[0::2] + 1j * a[1::2]


def interleave(c):
    out = np.empty(2 * len(c), np.float32)
    out[0::2] = c.real
    out[1::2] = c.imag
    return out


MODES = [ct.CT_FOURIER_FUSED, ct.CT_FOURIER_GRIDDING]


@pytest.mark.parametrize("geom", GEOMS)
@pytest.mark.parametrize("m_sp", [2, 6])
@pytest.mark.parametrize("mode", MODES)
def test_products_match_the_oracle(dev, geom, m_sp, mode):
    n = geom[0]
    g = oracle_grid(geom, m_sp)
    F = gpu_F(geom, m_sp, mode)
    assert F.rows == len(g.wx) and F.cols == n * n
    x = inputs.random_vector(n * n, 1000 + n).astype(np.float64)
    xt = torch.tensor(x, dtype=torch.float32, device=dev)
    y = torch.empty(2 * F.rows, dtype=torch.float32, device=dev)
    F.forward(xt, y)
    assert rel(as_complex(y), g.forward(x)) <= TOL[m_sp]
    c = g.forward(x) + 0.1 * (inputs.random_vector(F.rows, 7) + 1j * inputs.random_vector(F.rows, 8))
    ct_ = torch.tensor(interleave(c), device=dev)
    out = torch.empty(n * n, dtype=torch.float32, device=dev)
    F.adjoint(ct_, out)
    assert rel(out.cpu().numpy(), g.adjoint(c)) <= TOL[m_sp]
    F.normal(xt, out)
    assert rel(out.cpu().numpy(), g.normal_fused(x)) <= TOL[m_sp]


@pytest.mark.parametrize("geom", GEOMS)
def test_fused_and_gridding_modes_agree(dev, geom):
    """The same operator by the fused matrix and by interpolate-then-spread."""
    n = geom[0]
    x = torch.tensor(inputs.random_vector(n * n, 11), dtype=torch.float32, device=dev)
    a = torch.empty(n * n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    gpu_F(geom, 6, ct.CT_FOURIER_FUSED).normal(x, a)
    gpu_F(geom, 6, ct.CT_FOURIER_GRIDDING).normal(x, b)
    assert rel(a.cpu().numpy(), b.cpu().double().numpy()) <= 1e-5


def test_small_grid_with_aliased_offsets(dev):
    """N = 16, m_sp = 3: the fused matrix's offsets |d| <= 6 stay distinct,
    m_sp = 8: 33 offsets per dimension on a 32-point grid alias (d and d - 32
    address the same column) and must still sum to G^T G."""
    geom = (16, 24, 1, 23)
    x = inputs.random_vector(256, 12).astype(np.float64)
    xt = torch.tensor(x, dtype=torch.float32, device=dev)
    out = torch.empty(256, dtype=torch.float32, device=dev)
    for m_sp, tol in [(3, 1e-5), (8, 2e-3)]:
        F = ct.FourierMatrix(*geom, m_sp=m_sp)
        F.normal(xt, out)
        assert rel(out.cpu().numpy(), fo.Gridding(*geom, m_sp).normal_fused(x)) <= tol, m_sp
        F.close()


@pytest.mark.parametrize("n_bins", [46, 45])
def test_data_transform(dev, n_bins):
    geom = (32, 40, 2, n_bins)
    F = gpu_F(geom, 2, ct.CT_FOURIER_FUSED)
    n_kept = radon.num_kept(40, 2)
    f = inputs.random_vector(n_kept * n_bins, 13).astype(np.float64)
    fh = torch.empty(2 * F.rows, dtype=torch.float32, device=dev)
    F.data(torch.tensor(f, dtype=torch.float32, device=dev), fh)
    assert rel(as_complex(fh), fo.sinogram_dft(f, n_kept, n_bins)) <= 2e-6


@pytest.mark.parametrize("m_sp", [2, 6])
@pytest.mark.parametrize("mode", MODES)
def test_cg_matches_the_oracle(dev, m_sp, mode):
    """Five CG steps on alpha Re(F^H F) + lambda grad^T grad."""
    geom = GEOMS[1]
    n = geom[0]
    g = oracle_grid(geom, m_sp)
    F = gpu_F(geom, m_sp, mode)
    rhs = inputs.random_vector(n * n, 14).astype(np.float64)
    u = torch.zeros(n * n, dtype=torch.float32, device=dev)
    st = F.cg_solve(torch.tensor(rhs, dtype=torch.float32, device=dev), u, 0.0, 1.0, 0.5, 5)
    assert st["status"] == 0 and st["iters"] == 5
    op = tv.make_operator(None, (n, n), 0.0, 1.0, 0.5, normal=g.normal_fused)
    want, _ = tv.cg(op, rhs, np.zeros(n * n), 5)
    assert rel(u.cpu().numpy(), want) <= 10 * TOL[m_sp]


def _fourier_problem(geom, seed):
    n = geom[0]
    A = radon.siddon_matrix(*geom)
    f = A @ inputs.ellipse_phantom(n, seed).ravel()
    return A, inputs.gaussian_noisy(f, 0.01, seed + 1)


@pytest.mark.parametrize("mode", MODES)
def test_split_bregman_matches_the_oracle(dev, mode):
    """Two updates of five CG steps from the measured sinogram: the library
    forms fhat and alpha Re(F^H fhat) itself."""
    geom, m_sp = GEOMS[1], 2
    n = geom[0]
    _, f = _fourier_problem(geom, 5100)
    F = gpu_F(geom, m_sp, mode)
    u = torch.zeros(n * n, dtype=torch.float32, device=dev)
    st = F.split_bregman(torch.tensor(f, dtype=torch.float32, device=dev), u, 1.0, 1.0, 2, 5)
    g = oracle_grid(geom, m_sp)
    S = fo.FourierSystem(*geom, gridding=g)
    fhat = fo.sinogram_dft(f, radon.num_kept(geom[1], geom[2]), geom[3])
    want = tv.split_bregman(S, fhat, (n, n), 1.0, 1.0, 2, 5, normal=g.normal_fused)
    assert st["status"] == 0 and st["outer_done"] == 2
    assert rel(u.cpu().numpy(), want["u"].ravel()) <= 1e-4
    assert abs(st["first_update_l1"] - want["updates"][0]) <= 1e-4 * want["updates"][0]


def test_surrogate_from_the_fourier_normal_operator(dev):
    """Sec. 3.2 builds T from the point response of the Fourier normal
    operator; the handle's stencil is its exact FP64 sum, symmetrised."""
    geom = GEOMS[0]
    F = gpu_F(geom, 2, ct.CT_FOURIER_FUSED)
    taps = F.surrogate_stencil(3)
    h = fo.point_response(*geom, 3)
    assert len(taps) == 29
    for (di, dj), v in taps.items():
        want = 0.5 * (h[di + 3, dj + 3] + h[-di + 3, -dj + 3])
        assert abs(v - want) <= 1e-12 * abs(h[3, 3])
    # surrogate split Bregman runs on the handle (no Fourier products inside CG)
    n = geom[0]
    _, f = _fourier_problem(geom, 5200)
    u = torch.zeros(n * n, dtype=torch.float32, device=dev)
    st = F.split_bregman(torch.tensor(f, dtype=torch.float32, device=dev), u, 1.0, 1.0, 3, 5, surrogate_r=3)
    assert st["status"] == 0 and st["outer_done"] == 3


def test_chambolle_pock_on_the_fourier_term(dev):
    geom, m_sp = GEOMS[0], 2
    n = geom[0]
    _, f = _fourier_problem(geom, 5300)
    F = gpu_F(geom, m_sp, ct.CT_FOURIER_FUSED)
    u = torch.zeros(n * n, dtype=torch.float32, device=dev)
    st = F.chambolle_pock(torch.tensor(f, dtype=torch.float32, device=dev), u, 1.0, 0.35, 0.35, 3, 5)
    g = oracle_grid(geom, m_sp)
    S = fo.FourierSystem(*geom, gridding=g)
    fhat = fo.sinogram_dft(f, radon.num_kept(geom[1], geom[2]), geom[3])
    want = tv.chambolle_pock(S, fhat, (n, n), 1.0, 0.35, 0.35, 3, 5)
    assert st["status"] == 0 and st["outer_done"] == 3
    assert rel(u.cpu().numpy(), want["u"].ravel()) <= 1e-4


def test_allocation_free_cg_on_a_fourier_handle(dev):
    """The fixed-scratch CG entry runs the same kernels: identical bits."""
    geom = GEOMS[0]
    n = geom[0]
    F = gpu_F(geom, 2, ct.CT_FOURIER_FUSED)
    rhs = torch.tensor(inputs.random_vector(n * n, 15), dtype=torch.float32, device=dev)
    u1 = torch.zeros(n * n, dtype=torch.float32, device=dev)
    u2 = torch.zeros_like(u1)
    F.cg_solve(rhs, u1, 0.0, 1.0, 0.5, 6)
    p = ct.CgParams(0.0, 1.0, 0.5, 6, 0.0, 0, 0, 0)
    ct.ct_cg_solve_noalloc(F.handle, p, rhs, u2)
    torch.cuda.synchronize()
    assert torch.equal(u1, u2)


def test_siddon_only_calls_are_rejected(dev):
    geom = GEOMS[0]
    n = geom[0]
    F = gpu_F(geom, 2, ct.CT_FOURIER_FUSED)
    x = torch.zeros(n * n, dtype=torch.float32, device=dev)
    y = torch.zeros(F.rows, dtype=torch.float32, device=dev)
    with pytest.raises(ct.CtError) as e:
        ct.ct_forward(F.handle, x, y, 1)
    assert e.value.code == ct.CT_ERR_UNSUPPORTED
    with pytest.raises(ct.CtError) as e:
        F.cg_solve(torch.zeros(2 * n * n, device=dev), torch.zeros(2 * n * n, device=dev), 0.0, 1.0, 1.0, 2)
    assert e.value.code == ct.CT_ERR_UNSUPPORTED
    M = ct.Matrix(*geom)
    with pytest.raises(ct.CtError) as e:
        ct.ct_fourier_normal(M.handle, x, x)
    assert e.value.code == ct.CT_ERR_UNSUPPORTED
    M.close()
