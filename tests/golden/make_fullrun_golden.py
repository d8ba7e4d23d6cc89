"""Writes the FP64 oracle's values for whole reconstructions in the
tolerance-stopped form (tests/golden/fullrun_*.txt).

A fixed number of CG steps per Bregman update makes a long split-Bregman run
an extremely sensitive function of its inputs: two FP64 runs of the 512 x 512
slice whose matrices differ by 1e-15 relative end about 3e-2 apart after 50
updates, so no implementation can match another there to 1e-3.  With every
inner solve run to a tight relative residual (the same 50 updates, CG stopped
once ||r|| <= 1e-8 ||rhs||, at most 3000 steps) the run depends on the problem
alone: the same perturbation then moves the first two updates by 5.3e-6 and
4.3e-6 (about 850 and 750 CG steps; at 1e-10, 1300 steps and 7e-8).  This script
runs that form with the oracle only (``oracle/`` and the seeded input
generators; nothing from the CUDA library) and stores, per run, the CG steps
and the L1 size of every update, the final TV objective and norms of the image,
and the values of 4096 seeded sample pixels.

Runs (the sinogram is projected by the oracle's own FP64 matrix):
  slice512_f64      the 512 x 512 slice workload (180 of 720 angles, 725 bins,
                    1% Gaussian noise, alpha = lambda = 1), FP64 matrix;
  slice512_f32vals  the same with the matrix values and the sinogram rounded
                    to FP32 (what the library stores and receives): the
                    oracle's own spread from that rounding;
  batch512_s<k>_f64 / _fp16
                    slice k of the 256-slice batched workload (Poisson noise at
                    1e4 counts per bin), with the FP64 matrix and with the
                    dequantised FP16 row-scale matrix;
  slice512_fixed_f64 / _fixed_pert
                    the slice workload in its fixed-count form (50 updates of
                    20 CG steps), with the FP64 matrix and with its values
                    multiplied by 1 + 1e-15 z (z standard normal, seed 5): how
                    far the oracle drifts from itself in that form.

Usage: python tests/golden/make_fullrun_golden.py [run names]   (the runs go
to separate processes; the CSR products of each run share ORACLE_THREADS
threads, about an hour per run on two threads).
"""

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUTER = 50
CG_TOL = 1e-8
CG_CAP = 3000
FIXED_INNER = 20
N_SAMPLES = 4096
SAMPLE_SEED = 777
BATCH_SLICES = (0,)


def sample_indices(n2):
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    return np.sort(rng.choice(n2, size=N_SAMPLES, replace=False))


def problem(name):
    """(A, f, shape, alpha, lam, description) of a named run."""
    from oracle import radon
    from paper_1705_07497_gb300 import inputs

    if name.startswith("slice512"):
        wl = inputs.WORKLOADS["slice_512"]
        n = wl["n"]
        A = radon.siddon_matrix(n, wl["n_angles_total"], wl["keep_every"], wl["n_bins"])
        truth = inputs.ellipse_phantom(n, wl["seed"])
        f = inputs.gaussian_noisy(A @ truth.ravel(), wl["sigma_rel"], wl["seed"] + 1)
        desc = "slice_512 workload: phantom seed %d, Gaussian noise seed %d" % (wl["seed"], wl["seed"] + 1)
        if name == "slice512_fixed_pert":
            rng = np.random.Generator(np.random.PCG64(5))
            A.data = A.data * (1.0 + 1e-15 * rng.standard_normal(A.data.shape))
            desc += "; matrix values times 1 + 1e-15 z"
        if name == "slice512_f32vals":
            A.data = A.data.astype(np.float32).astype(np.float64)
            f = f.astype(np.float32).astype(np.float64)
            desc += "; matrix values and sinogram rounded to FP32"
        return A, f, (n, n), wl["alpha"], wl["lam"], desc
    # batch512_s<k>_<f64|fp16>
    wl = inputs.WORKLOADS["batch_512x256"]
    n = wl["n"]
    k = int(name.split("_")[1][1:])
    A = radon.siddon_matrix(n, wl["n_angles_total"], wl["keep_every"], wl["n_bins"])
    truth = inputs.ellipse_phantom(n, wl["seed"] + k)
    f = inputs.poisson_noisy(A @ truth.ravel(), wl["counts"], wl["seed"] + 10000 + k)
    desc = ("batch_512x256 workload, slice %d: phantom seed %d, Poisson noise (%g counts) seed %d"
            % (k, wl["seed"] + k, wl["counts"], wl["seed"] + 10000 + k))
    if name.endswith("_fp16"):
        s, Q = radon.quantize_rowscale(A)
        A = radon.dequantize(s, Q).tocsr()
        desc += "; dequantised FP16 row-scale matrix"
    return A, f, (n, n), wl["alpha"], wl["lam"], desc


def run(name):
    from oracle import spmv, tv

    A, f, shape, alpha, lam, desc = problem(name)
    Ap = spmv.ThreadedCSR(A)
    iters = []
    cg = tv.cg

    def counting_cg(*a, **k):
        u, st = cg(*a, **k)
        iters.append(st["iters"])
        return u, st

    tv.cg = counting_cg
    t0 = time.time()
    fixed = "_fixed" in name
    inner, tol = (FIXED_INNER, 0.0) if fixed else (CG_CAP, CG_TOL)
    res = tv.split_bregman(Ap, f, shape, alpha, lam, OUTER, inner, cg_tol=tol)
    secs = time.time() - t0
    tv.cg = cg
    u = res["u"]
    idx = sample_indices(u.size)
    flat = u.ravel()
    lines = [
        "# FP64 oracle, split Bregman (Eq. SB_solve, anisotropic TV, Sec. 4): %d updates, each inner CG"
        % OUTER,
        ("# warm-started, %d steps (the fixed-count form)." % FIXED_INNER) if fixed else
        ("# warm-started and stopped at ||r|| <= %g ||rhs|| (at most %d steps)." % (CG_TOL, CG_CAP)),
        "# Written by tests/golden/make_fullrun_golden.py (oracle only) in %.0f s." % secs,
        "# %s" % desc,
        "# alpha %r lambda %r" % (alpha, lam),
        "name %s" % name,
        "outer_done %d" % res["outer_done"],
        "cg_iters " + " ".join(str(i) for i in iters),
        "update_l1 " + " ".join("%.17g" % v for v in res["updates"]),
        "objective %.17g" % tv.tv_objective(A, f, u, alpha),
        "l1_norm %.17g" % float(np.abs(flat).sum()),
        "l2_norm %.17g" % float(np.linalg.norm(flat)),
        "# sample pixels: row-major index, value",
    ]
    lines += ["%d %.17g" % (i, flat[i]) for i in idx]
    with open(os.path.join(HERE, "fullrun_%s.txt" % name), "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return name, secs


ALL = (["slice512_f64", "slice512_f32vals"] + ["batch512_s%d_%s" % (k, m) for k in BATCH_SLICES
                                              for m in ("f64", "fp16")]
       + ["slice512_fixed_f64", "slice512_fixed_pert"])

if __name__ == "__main__":
    names = sys.argv[1:] or ALL
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for name, secs in pool.imap_unordered(run, names):
            print(name, "%.0f s" % secs, flush=True)
