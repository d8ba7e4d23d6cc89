"""Launch-shape tuning of the sparse products (ct_tune / ct_set_tuning).

Every candidate launch shape must compute the same bits: each row of A and
A^T is summed in the same order whatever the warps per block, the chunks in
flight or the register budget, so the tuner's choice can only change speed.
"""

import numpy as np
import pytest

from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SINGLE = [dict(fwd_warps=w, fwd_unroll=u) for w in (8, 4) for u in (8, 4, 2, 16)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _bits(t):
    return t.cpu().numpy().view(np.uint32).copy()


@pytest.mark.parametrize("geom,flags,ctas", [((64, 90, 3, 91), ct.CT_VAL_FP32, (7, 4, 3)),
                                             ((64, 360, 1, 91), ct.CT_VAL_FP32, (5, 3)),
                                             ((96, 120, 1, 137), ct.CT_VAL_FP16_ROWSCALE, (7, 4, 3))])
def test_every_single_slice_launch_shape_gives_the_same_bits(dev, geom, flags, ctas):
    M = ct.Matrix(*geom, flags=flags)
    x = torch.tensor(inputs.random_vector(M.cols, 31), dtype=torch.float32, device=dev)
    rhs = torch.tensor(inputs.random_vector(M.cols, 32), dtype=torch.float32, device=dev)
    ref_y = ref_u = None
    ops = [(c, 1) for c in ctas] + ([(7, 2)] if 7 in ctas else [])
    for shape in SINGLE:
        for c, px in ops:
            ct.ct_set_tuning(M.handle, 1, op_ctas=c, op_pixels=px, **shape)
            assert ct.ct_get_tuning(M.handle, 1) == dict(shape, op_ctas=c, op_pixels=px, spmm_unroll=0)
            y = torch.empty(M.rows, device=dev)
            M.forward(x, y)
            u = torch.zeros(M.cols, device=dev)
            M.cg_solve(rhs, u, 0.0, 1.0, 0.3, 7)
            torch.cuda.synchronize()
            if ref_y is None:
                ref_y, ref_u = _bits(y), _bits(u)
            np.testing.assert_array_equal(_bits(y), ref_y)
            np.testing.assert_array_equal(_bits(u), ref_u)
    M.close()


def test_tuner_picks_listed_shapes_and_caches_them_by_geometry(dev):
    geom = (128, 180, 1, inputs.n_bins_for(128))
    M = ct.Matrix(*geom)
    assert ct.ct_get_tuning(M.handle, 1)["fwd_warps"] == 0
    ct.ct_tune(M.handle, 1)
    t = ct.ct_get_tuning(M.handle, 1)
    assert t["fwd_warps"] in (4, 8) and t["fwd_unroll"] in (2, 4, 8, 16) and t["op_ctas"] in (7, 4, 3)
    assert t["op_pixels"] in (1, 2)
    # a second handle of the same geometry takes the cached choice; the
    # first solve fills it in
    M2 = ct.Matrix(*geom)
    rhs = torch.ones(M2.cols, device=dev)
    u = torch.zeros(M2.cols, device=dev)
    M2.cg_solve(rhs, u, 0.0, 1.0, 1.0, 2)
    assert ct.ct_get_tuning(M2.handle, 1) == t
    M.close()
    M2.close()


def test_batched_tuning_gives_the_same_bits_and_rejects_single_fields(dev):
    M = ct.Matrix(64, 90, 3, 91)
    B = 5
    rhs = torch.tensor(inputs.random_vector(M.cols * B, 33).reshape(M.cols, B), dtype=torch.float32, device=dev)
    outs = []
    for unroll in (4, 8):
        ct.ct_set_tuning(M.handle, B, spmm_unroll=unroll)
        u = torch.zeros((M.cols, B), device=dev)
        M.cg_solve(rhs, u, 0.0, 1.0, 0.3, 6)
        outs.append(_bits(u))
    np.testing.assert_array_equal(outs[0], outs[1])
    ct.ct_set_tuning(M.handle, B, spmm_unroll=0)
    ct.ct_tune(M.handle, B)
    assert ct.ct_get_tuning(M.handle, B)["spmm_unroll"] in (4, 8)
    with pytest.raises(ct.CtError):
        ct.ct_set_tuning(M.handle, B, fwd_warps=8)
    with pytest.raises(ct.CtError):
        ct.ct_set_tuning(M.handle, 1, fwd_warps=6)
    with pytest.raises(ct.CtError):
        ct.ct_set_tuning(M.handle, 1, op_ctas=5)  # this matrix stages its band in one chunk
    with pytest.raises(ct.CtError):
        ct.ct_set_tuning(M.handle, 1, op_ctas=6)
    with pytest.raises(ct.CtError):
        ct.ct_set_tuning(M.handle, 1, op_ctas=4, op_pixels=2)
    M.close()
