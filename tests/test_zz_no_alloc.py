"""The allocation-free CG entry point (ct_cg_solve_noalloc) against ct_cg_solve.

Some callers cannot allocate device memory when they need a solve (a
real-time loop that must not stall on an allocation, or a process whose
device memory another allocator already holds); ct_cg_solve_noalloc serves
them from a fixed scratch array inside the library.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""

import ctypes

import numpy as np
import pytest

from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CG_TOL = 1e-4  # the relative tolerance of the CG parity tests


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _two_calls(dev, M, coef, tol):
    n2 = M.cols
    params = ct.CgParams(coef[0], coef[1], coef[2], 12, 0.0, 0, 0, 0)
    for call in range(2):
        rhs = torch.tensor(inputs.random_vector(n2, 40 + call), dtype=torch.float32, device=dev)
        u0 = torch.tensor(0.1 * inputs.random_vector(n2, 50 + call), dtype=torch.float32, device=dev)
        u_ref = u0.clone()
        st_ref = ct.CgStats()
        ct.ct_cg_solve(M.handle, params, rhs, u_ref, 1, st_ref)
        u_na = u0.clone()
        st_na = ct.CgStats()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        ct.ct_cg_solve_noalloc(M.handle, params, rhs, u_na, st_na)
        torch.cuda.synchronize()
        # the call commits no device memory (the scratch array was committed
        # when the handle was built)
        assert torch.cuda.mem_get_info(dev)[0] == free_before
        assert st_na.status == 0 and st_na.iters == st_ref.iters == 12
        assert _rel(u_na, u_ref) <= tol
        assert abs(st_na.final_rel_res - st_ref.final_rel_res) <= tol * st_ref.final_rel_res


@pytest.mark.parametrize("geom,coef,flags", [((64, 90, 3, 91), (0.0, 1.0, 0.1), ct.CT_VAL_FP32),
                                             ((512, 720, 4, 725), (1.0, 0.05, 0.0), ct.CT_VAL_FP32),
                                             ((64, 90, 3, 91), (0.0, 1.0, 0.1), ct.CT_VAL_FP16_ROWSCALE)])
def test_noalloc_matches_cg_solve_on_two_calls(dev, geom, coef, flags):
    M = ct.Matrix(*geom, flags=flags)
    _two_calls(dev, M, coef, CG_TOL)
    M.close()


def test_noalloc_on_a_fourier_handle_matches_cg_solve(dev):
    M = ct.FourierMatrix(64, 90, 3, 91, m_sp=6)
    _two_calls(dev, M, (0.0, 1.0, 0.1), CG_TOL)
    M.close()


def test_noalloc_rejects_problems_beyond_the_scratch_limit(dev):
    M = ct.Matrix(1024, 4, 1, inputs.n_bins_for(1024))
    params = ct.CgParams(1.0, 1.0, 0.0, 2, 0.0, 0, 0, 0)
    rhs = torch.ones(M.cols, dtype=torch.float32, device=dev)
    u = torch.zeros(M.cols, dtype=torch.float32, device=dev)
    with pytest.raises(ct.CtError) as ei:
        ct.ct_cg_solve_noalloc(M.handle, params, rhs, u)
    assert ei.value.code == ct.CT_ERR_ARG
    assert "CT_NOALLOC_SCRATCH_BYTES" in str(ei.value)
    M.close()
