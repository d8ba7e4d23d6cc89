"""The largest geometry the ragged workload draws: a 1024 x 1024 image, 900
angles (all kept), 1449 bins, about 1.2e9 entries per matrix.  The oracle
cannot build it whole, so sampled rows come from its per-ray tracer; the
adjoint is checked through the adjoint identity, which holds at any size, and
the solvers through an invariant of the first CG step."""

import numpy as np
import pytest

from oracle import radon
from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GEOM = (1024, 900, 1, 1449)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


@pytest.fixture(scope="module")
def sampled_rows():
    rows = np.sort(np.random.Generator(np.random.PCG64(11)).choice(900 * 1449, 1500, replace=False))
    return rows, radon.siddon_rows(*GEOM, rows)


def _solvers_run(M, dev, seed):
    """The solvers at this size: one CG step from zero gives u = c rhs with
    c = (r.r) / (r.Op r) > 0, and one split-Bregman update completes."""
    rhs = torch.tensor(inputs.random_vector(M.cols, seed), dtype=torch.float32, device=dev)
    u = torch.zeros(M.cols, device=dev)
    st = M.cg_solve(rhs, u, 0.0, 1.0, 1.0, 1)
    assert st["status"] == 0 and st["iters"] == 1
    ud, rd = u.double(), rhs.double()
    cos = float((ud * rd).sum() / (ud.norm() * rd.norm()))
    assert cos >= 1.0 - 1e-6
    y = torch.empty(M.rows, device=dev)
    M.forward(torch.tensor(inputs.ellipse_phantom(M.n, seed + 1).ravel(), dtype=torch.float32, device=dev), y)
    u.zero_()
    sb = M.split_bregman(y, u, 1.0, 1.0, 1, 3)
    assert sb["status"] == 0 and sb["outer_done"] == 1 and sb["first_update_l1"] > 0
    assert torch.isfinite(u).all()


def _rel_max(got, want):
    return float(np.abs(got - want).max() / np.abs(want).max())


def test_largest_geometry_fp32(dev, sampled_rows):
    rows, R = sampled_rows
    M = ct.Matrix(*GEOM)
    try:
        assert M.rows == 900 * 1449 and M.cols == 1024 * 1024
        x = inputs.ellipse_phantom(1024, 5000).ravel()
        y = torch.empty(M.rows, device=dev)
        M.forward(torch.tensor(x, dtype=torch.float32, device=dev), y)
        assert _rel_max(y.cpu().numpy()[rows], R @ x) <= 1e-5
        # adjoint identity <A x, v> = <x, A^T v> with random x, v
        xr = torch.tensor(inputs.random_vector(M.cols, 51), dtype=torch.float32, device=dev)
        v = torch.tensor(inputs.random_vector(M.rows, 52), dtype=torch.float32, device=dev)
        Ax = torch.empty(M.rows, device=dev)
        Atv = torch.empty(M.cols, device=dev)
        M.forward(xr, Ax)
        M.adjoint(v, Atv)
        lhs = float((Ax.double() * v.double()).sum())
        rhs = float((xr.double() * Atv.double()).sum())
        assert abs(lhs - rhs) <= 1e-6 * float((Ax.double().abs() * v.double().abs()).sum())
        _solvers_run(M, dev, 53)
    finally:
        M.close()


def test_largest_geometry_fp16(dev, sampled_rows):
    rows, R = sampled_rows
    s, Q = radon.quantize_rowscale(R)  # complete rows: the same row maxima as the whole matrix
    R16 = radon.dequantize(s, Q).tocsr()
    M = ct.Matrix(*GEOM, ct.CT_VAL_FP16_ROWSCALE)
    try:
        x = inputs.ellipse_phantom(1024, 5001).ravel()
        y = torch.empty(M.rows, device=dev)
        M.forward(torch.tensor(x, dtype=torch.float32, device=dev), y)
        assert _rel_max(y.cpu().numpy()[rows], R16 @ x) <= 1e-5
        _solvers_run(M, dev, 55)
    finally:
        M.close()
