"""Whole reconstructions against the FP64 oracle's whole runs.

A fixed count of CG steps per Bregman update makes a long run an extremely
sensitive function of its inputs (the FP64 oracle drifts from itself by about
3e-2 over the 512 x 512 slice's 50 updates under a 1e-15 change of its
matrix), so a whole run is compared in the tolerance-stopped form: the same
updates with every inner CG run to ||r|| <= tol ||rhs||, where the result is
a function of the problem alone.  The 64 x 64 workload is compared with the
oracle run here; the 512 x 512 slice and a slice of the batched FP16 workload
against the values the oracle wrote (tests/golden/fullrun_*.txt, written by
tests/golden/make_fullrun_golden.py from the oracle only).
"""

import os

import numpy as np
import pytest

from oracle import radon, tv
from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
RECON_TOL = 1e-3   # per reconstruction, relative L2 against the FP64 oracle
CG_TOL = 1e-8      # the golden runs' inner tolerance
CG_CAP = 3000


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def read_golden(name):
    path = os.path.join(GOLDEN, "fullrun_%s.txt" % name)
    if not os.path.exists(path):
        pytest.skip("golden values %s not written yet" % path)
    g = {"idx": [], "val": []}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, rest = line.split(" ", 1)
        if key.isdigit():
            g["idx"].append(int(key))
            g["val"].append(float(rest))
        elif key in ("cg_iters",):
            g[key] = [int(v) for v in rest.split()]
        elif key == "update_l1":
            g[key] = [float(v) for v in rest.split()]
        elif key == "name":
            g[key] = rest.strip()
        else:
            g[key] = float(rest)
    g["idx"] = np.array(g["idx"])
    g["val"] = np.array(g["val"])
    return g


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_tolerance_form_whole_64_run_matches_the_oracle(dev):
    wl = inputs.WORKLOADS["plain_64"]
    n = wl["n"]
    A = radon.siddon_matrix(n, wl["n_angles_total"], wl["keep_every"], wl["n_bins"])
    f = A @ inputs.ellipse_phantom(n, wl["seed"]).ravel()
    want = tv.split_bregman(A, f, (n, n), wl["alpha"], wl["lam"], wl["outer"], CG_CAP, cg_tol=1e-10)
    M = ct.Matrix(n, wl["n_angles_total"], wl["keep_every"], wl["n_bins"])
    u = torch.zeros(n * n, device=dev)
    st = M.split_bregman(torch.tensor(f, dtype=torch.float32, device=dev), u, wl["alpha"], wl["lam"],
                         wl["outer"], CG_CAP, cg_rel_tol=1e-10)
    assert st["status"] == 0 and st["outer_done"] == wl["outer"]
    assert rel(u.cpu().numpy(), want["u"].ravel()) <= 1e-6
    np.testing.assert_allclose(st["first_update_l1"], want["updates"][0], rtol=1e-6)
    np.testing.assert_allclose(st["last_update_l1"], want["updates"][-1], rtol=1e-4)
    M.close()


def _slice_problem(wl):
    n = wl["n"]
    A = radon.siddon_matrix(n, wl["n_angles_total"], wl["keep_every"], wl["n_bins"])
    return A


def _compare(got, A, f, g, alpha):
    """Errors of a whole reconstruction against the oracle's stored values."""
    flat = np.asarray(got, np.float64).ravel()
    return {
        "samples": rel(flat[g["idx"]], g["val"]),
        "l1_norm": abs(np.abs(flat).sum() - g["l1_norm"]) / g["l1_norm"],
        "l2_norm": abs(np.linalg.norm(flat) - g["l2_norm"]) / g["l2_norm"],
        "objective": abs(tv.tv_objective(A, f, flat.reshape(int(np.sqrt(flat.size)), -1), alpha)
                         - g["objective"]) / g["objective"],
    }


def test_slice512_whole_run_in_tolerance_form_matches_the_oracle(dev):
    g = read_golden("slice512_f64")
    wl = inputs.WORKLOADS["slice_512"]
    n = wl["n"]
    A = _slice_problem(wl)
    f = inputs.gaussian_noisy(A @ inputs.ellipse_phantom(n, wl["seed"]).ravel(), wl["sigma_rel"], wl["seed"] + 1)
    M = ct.Matrix(n, wl["n_angles_total"], wl["keep_every"], wl["n_bins"])
    u = torch.zeros(n * n, device=dev)
    st = M.split_bregman(torch.tensor(f, dtype=torch.float32, device=dev), u, wl["alpha"], wl["lam"],
                         wl["outer"], CG_CAP, cg_rel_tol=CG_TOL)
    assert st["status"] == 0 and st["outer_done"] == wl["outer"]
    err = _compare(u.cpu().numpy(), A, f, g, wl["alpha"])
    print("512x512 slice, tolerance form, 50 updates vs FP64 oracle:", err)
    assert err["samples"] <= RECON_TOL
    assert err["l1_norm"] <= RECON_TOL and err["l2_norm"] <= RECON_TOL and err["objective"] <= RECON_TOL
    np.testing.assert_allclose(st["first_update_l1"], g["update_l1"][0], rtol=1e-4)
    np.testing.assert_allclose(st["last_update_l1"], g["update_l1"][-1], rtol=1e-2)
    M.close()


def test_batched_fp16_whole_run_in_tolerance_form_matches_the_oracle(dev):
    """Slice 0 of the batched FP16 workload, solved in a batch of two slices
    (the batched SpMM kernels) in the tolerance form: against the oracle on
    the dequantised FP16 matrix (the kernels' error) and on the FP64 matrix
    (what the FP16 storage costs, stated)."""
    g16 = read_golden("batch512_s0_fp16")
    g64 = read_golden("batch512_s0_f64")
    wl = inputs.WORKLOADS["batch_512x256"]
    n = wl["n"]
    A = _slice_problem(wl)
    F = np.stack([inputs.poisson_noisy(A @ inputs.ellipse_phantom(n, wl["seed"] + k).ravel(), wl["counts"],
                                       wl["seed"] + 10000 + k) for k in (0, 1)], axis=1)
    M = ct.Matrix(n, wl["n_angles_total"], wl["keep_every"], wl["n_bins"], ct.CT_VAL_FP16_ROWSCALE)
    U = torch.zeros((n * n, 2), device=dev)
    st = M.split_bregman(torch.tensor(F, dtype=torch.float32, device=dev), U, wl["alpha"], wl["lam"],
                         wl["outer"], CG_CAP, cg_rel_tol=CG_TOL)
    assert st["status"] == 0 and st["outer_done"] == wl["outer"]
    got = U[:, 0].cpu().numpy()
    s, Q = radon.quantize_rowscale(A)
    A16 = radon.dequantize(s, Q).tocsr()
    e16 = _compare(got, A16, F[:, 0], g16, wl["alpha"])
    e64 = _compare(got, A, F[:, 0], g64, wl["alpha"])
    print("batched FP16 slice 0, tolerance form vs the dequantised oracle:", e16, "vs the FP64 oracle:", e64)
    assert e16["samples"] <= RECON_TOL and e16["objective"] <= RECON_TOL
    M.close()
