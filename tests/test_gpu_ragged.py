"""Ragged batches: split Bregman over problems of different geometries in one
ct_split_bregman_ragged call, each problem against its own FP64 oracle run."""

import functools

import numpy as np
import pytest

from oracle import radon, tv
from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GEOMS = [(32, 40, 1, 46), (48, 60, 2, 68), (64, 90, 3, 91)]


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
def gpu_A(geom, flags=0):
    return ct.Matrix(*geom, flags)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _problems(order, seed0):
    """(geometry, data) per problem: random ellipses projected by the oracle, 1% noise."""
    out = []
    for k, g in enumerate(order):
        geom = GEOMS[g]
        A = oracle_A(*geom)
        clean = A @ inputs.ellipse_phantom(geom[0], seed0 + k).ravel()
        out.append((geom, inputs.gaussian_noisy(clean, 0.01, seed0 + 100 + k)))
    return out


@pytest.mark.parametrize("outer", [2, 6])
def test_ragged_matches_per_problem_oracle(dev, outer):
    """Six problems over three geometries, handles interleaved; outer = 2 runs the
    updates directly, outer = 6 through the captured multi-stream graph."""
    probs = _problems([0, 1, 0, 2, 1, 2], 4000)
    mats = [gpu_A(g) for g, _ in probs]
    fs = [torch.tensor(f, dtype=torch.float32, device=dev) for _, f in probs]
    us = [torch.zeros(g[0] * g[0], dtype=torch.float32, device=dev) for g, _ in probs]
    stats = ct.split_bregman_ragged(mats, fs, us, 1.0, 0.5, outer, 8)
    # the persistent launch was captured into a graph (outer > 2) or launched directly
    assert ct.lib().ct_last_error() == b"", ct.lib().ct_last_error()
    for k, (geom, f) in enumerate(probs):
        n = geom[0]
        want = tv.split_bregman(oracle_A(*geom), f, (n, n), 1.0, 0.5, outer, 8)
        assert rel(us[k].cpu().numpy(), want["u"].ravel()) <= 1e-4, k
        assert stats[k]["status"] == 0 and stats[k]["outer_done"] == outer
        first = np.abs(want["updates"][0])
        assert abs(stats[k]["first_update_l1"] - first) <= 1e-4 * first, k


def test_ragged_equals_separate_calls(dev):
    """A problem solved inside a ragged call and alone through ct_split_bregman."""
    probs = _problems([2, 0, 1], 4100)
    mats = [gpu_A(g) for g, _ in probs]
    fs = [torch.tensor(f, dtype=torch.float32, device=dev) for _, f in probs]
    us = [torch.zeros(g[0] * g[0], dtype=torch.float32, device=dev) for g, _ in probs]
    ct.split_bregman_ragged(mats, fs, us, 1.0, 1.0, 5, 10)
    for k, (geom, _) in enumerate(probs):
        u1 = torch.zeros_like(us[k])
        mats[k].split_bregman(fs[k], u1, 1.0, 1.0, 5, 10)
        assert rel(us[k].cpu().numpy(), u1.cpu().double().numpy()) <= 1e-5, k


def test_ragged_mixed_storage_and_stop_rule(dev):
    """An FP16 handle beside FP32 handles; with the stop rule each problem stops on its own."""
    probs = _problems([0, 1, 1], 4200)
    mats = [gpu_A(probs[0][0], ct.CT_VAL_FP16_ROWSCALE), gpu_A(probs[1][0]), gpu_A(probs[2][0])]
    fs = [torch.tensor(f, dtype=torch.float32, device=dev) for _, f in probs]
    us = [torch.zeros(g[0] * g[0], dtype=torch.float32, device=dev) for g, _ in probs]
    stats = ct.split_bregman_ragged(mats, fs, us, 1.0, 0.5, 200, 8, stop_rel_update=0.05)
    for k, (geom, f) in enumerate(probs):
        n = geom[0]
        A = oracle_A(*geom)
        if k == 0:
            s, Q = radon.quantize_rowscale(A)
            A = radon.dequantize(s, Q).tocsr()
        want = tv.split_bregman(A, f, (n, n), 1.0, 0.5, 200, 8, stop_rel_update=0.05)
        assert want["outer_done"] < 200
        assert abs(stats[k]["outer_done"] - want["outer_done"]) <= 1, k
        if stats[k]["outer_done"] == want["outer_done"]:
            assert rel(us[k].cpu().numpy(), want["u"].ravel()) <= 1e-4, k


def test_ragged_rejects_host_pointers(dev):
    g, f = _problems([0], 4300)[0]
    M = gpu_A(g)
    with pytest.raises(ct.CtError) as e:
        ct.split_bregman_ragged([M], [f.astype(np.float32)], [np.zeros(g[0] * g[0], np.float32)],
                                1.0, 1.0, 3, 3)
    assert e.value.code == ct.CT_ERR_ARG


def test_ragged_large_group_uses_the_batched_products(dev):
    """Ten problems on one handle (above the single-run limit of eight: the
    batched SpMM path) beside two problems on another handle."""
    probs = _problems([0] * 10 + [1, 1], 4400)
    mats = [gpu_A(g) for g, _ in probs]
    fs = [torch.tensor(f, dtype=torch.float32, device=dev) for _, f in probs]
    us = [torch.zeros(g[0] * g[0], dtype=torch.float32, device=dev) for g, _ in probs]
    stats = ct.split_bregman_ragged(mats, fs, us, 1.0, 0.5, 5, 8)
    for k, (geom, f) in enumerate(probs):
        n = geom[0]
        want = tv.split_bregman(oracle_A(*geom), f, (n, n), 1.0, 0.5, 5, 8)
        assert rel(us[k].cpu().numpy(), want["u"].ravel()) <= 1e-4, k
        assert stats[k]["outer_done"] == 5


def test_ragged_persistent_kernel_with_staged_band_chunks_and_fp16(dev):
    """The persistent kernel on geometries whose sinogram band is staged in
    angle chunks (360 kept angles) beside small ones, FP16 and FP32 storage."""
    geoms = [(64, 360, 1, 91), (32, 40, 1, 46), (48, 400, 1, 68)]
    flags = [ct.CT_VAL_FP32, ct.CT_VAL_FP16_ROWSCALE, ct.CT_VAL_FP32]
    mats, fs, us, refs = [], [], [], []
    for k, (geom, fl) in enumerate(zip(geoms, flags)):
        A = oracle_A(*geom)
        f = inputs.gaussian_noisy(A @ inputs.ellipse_phantom(geom[0], 4500 + k).ravel(), 0.01, 4600 + k)
        if fl == ct.CT_VAL_FP16_ROWSCALE:
            s, Q = radon.quantize_rowscale(A)
            A = radon.dequantize(s, Q).tocsr()
        refs.append(tv.split_bregman(A, f, (geom[0], geom[0]), 1.0, 0.5, 4, 6)["u"].ravel())
        mats.append(gpu_A(geom, fl))
        fs.append(torch.tensor(f, dtype=torch.float32, device=dev))
        us.append(torch.zeros(geom[0] * geom[0], dtype=torch.float32, device=dev))
    stats = ct.split_bregman_ragged(mats, fs, us, 1.0, 0.5, 4, 6)
    for k in range(len(geoms)):
        assert stats[k]["status"] == 0 and stats[k]["outer_done"] == 4
        assert rel(us[k].cpu().numpy(), refs[k]) <= 1e-4, k


def test_ragged_bounded_wait_runs_out_and_the_gpu_answers_after(dev):
    """A dependency held back on purpose (a flag nothing sets) with a short
    wait limit: the persistent kernel returns CT_ERR_TIMEOUT instead of
    hanging, and the next call (default limit) solves correctly."""
    probs = _problems([0, 2, 1], 4700)
    mats = [gpu_A(g) for g, _ in probs]
    fs = [torch.tensor(f, dtype=torch.float32, device=dev) for _, f in probs]
    us = [torch.zeros(g[0] * g[0], dtype=torch.float32, device=dev) for g, _ in probs]
    ct.ct_set_wait_limit(2000, hold_first=True)
    try:
        with pytest.raises(ct.CtError) as e:
            ct.split_bregman_ragged(mats, fs, us, 1.0, 0.5, 3, 8)
        assert e.value.code == ct.CT_ERR_TIMEOUT
        assert "bounded wait" in str(e.value)
    finally:
        ct.ct_set_wait_limit(0, hold_first=False)
    torch.cuda.synchronize()
    for u in us:
        u.zero_()
    stats = ct.split_bregman_ragged(mats, fs, us, 1.0, 0.5, 3, 8)
    for k, (geom, f) in enumerate(probs):
        n = geom[0]
        want = tv.split_bregman(oracle_A(*geom), f, (n, n), 1.0, 0.5, 3, 8)
        assert stats[k]["status"] == 0
        assert rel(us[k].cpu().numpy(), want["u"].ravel()) <= 1e-4, k
