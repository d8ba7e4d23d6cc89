"""The experiment replay (Sec. 4) on a small case: it runs through the
library, and the two ways of evaluating the same Fourier-domain operator
(gridding on every product, the fused matrix) give the same reconstruction."""

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def test_fixed_iterations_small(dev):
    from paper_1705_07497_gb300 import replay

    rows = replay.fixed_iterations([64], updates=20, inner=5, m_sps=(2,))
    by = {r["method"]: r for r in rows}
    assert set(by) == {"Siddon sparse matrix (image domain)", "NUFFT, M_sp=2", "Convolution fusing, M_sp=2",
                       "Sparse surrogate 3x3, M_sp=2"}
    for r in rows:
        assert r["status"] == 0 and r["total_s"] > 0.0 and r["cg_s"] >= 0.0
    nufft, fused = by["NUFFT, M_sp=2"]["rel_l1"], by["Convolution fusing, M_sp=2"]["rel_l1"]
    assert abs(nufft - fused) <= 1e-6 * fused
    assert by["Siddon sparse matrix (image domain)"]["rel_l1"] < 0.1


def test_stopping_rule_small(dev):
    from paper_1705_07497_gb300 import replay

    rows = replay.stopping_rule(n=64, ds=(2,), tols=(1e-2, 1e-4), max_updates=300)
    assert len(rows) == 4
    fused = [r for r in rows if r["method"] == "Convolution fusing"]
    assert fused[0]["updates"] is not None and fused[0]["updates"] < 300
    for r in rows:
        if r["updates"] is not None:
            assert r["time_s"] > 0.0 and r["rel_l1"] is not None
