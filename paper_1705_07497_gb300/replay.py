"""Replays the experiments of Sec. 4 on synthetic data, one GPU.

    python -m paper_1705_07497_gb300.replay [--sizes 128 256 512] [--max-updates 2000]

Sec. 4 compares, for anisotropic-TV split Bregman with alpha = lambda = 1
and 5 CG steps per update, three ways of evaluating the Fourier-domain
data term: the NUFFT (gridding on every product), convolution fusing (the
precomputed B*B of Eq. fusedop) and the sparse surrogate T (Eq.
surr_SBupd), at window half-widths M_sp = 2, 6, 12 and image sizes N = 128,
256, 512 with N pi / 4 evenly spaced angles.  This module runs the same
grid of cases through the library and prints the same columns:

  fixed iterations   200 updates: total time, CG time (the same call with no
                     CG steps subtracted), relative L1 error against the
                     phantom (the paper's Tables of fixed-iteration time and
                     error); the library's own image-domain Siddon operator
                     is listed beside them
  stopping rule      N = 512, 512 pi / (4 d) angles for d = 1, 2, 4,
                     convolution fusing at M_sp = 6 against the surrogate:
                     updates and time until the L1 size of an update falls
                     below 1e-2, 1e-4, 1e-6, 1e-8 of the first one, and the
                     error there (the paper's Sub tables); "*" marks a
                     threshold not reached within max_updates

The surrogate windows: truncating this data term's point response (it
decays like 1/|d|, the polar samples being dense near the origin) to the
disc of radius 1 or to radius 3 (disc or square) gives an indefinite T,
and CG then stops with a breakdown.  The replay uses the SPD windows
nearest the paper's: the 3 x 3 square for r = 1 and the disc of radius 2
(13 taps) for r = 3.

The phantom is the library's seeded random-ellipse image (the paper's
Shepp-Logan phantom is not used) and the data are its exact Siddon
projections.  Times are CUDA-event times of whole ct_split_bregman calls on
device-resident data.
"""

import argparse
import json
import math
import time

import numpy as np

from . import ct, inputs


def _geometry(n, d=1):
    n_total = int(round(n * math.pi / 4))
    return n, n_total, d, inputs.n_bins_for(n)


def _timed(fn):
    import torch

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out = fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3, out


def _rel_l1(u, truth):
    return float(np.abs(u - truth).sum() / np.abs(truth).sum())


def _data(geom, seed, dev):
    import torch

    n = geom[0]
    truth = inputs.ellipse_phantom(n, seed).ravel()
    A = ct.Matrix(*geom)
    f = torch.empty(A.rows, dtype=torch.float32, device=dev)
    A.forward(torch.tensor(truth, dtype=torch.float32, device=dev), f)
    return A, truth, f


def fixed_iterations(sizes, updates=200, inner=5, m_sps=(2, 6, 12), seed=7000):
    import torch

    dev = torch.device("cuda", 0)
    rows = []
    for n in sizes:
        geom = _geometry(n)
        A, truth, f = _data(geom, seed + n, dev)
        methods = [("Siddon sparse matrix (image domain)", A, 0)]
        handles = []
        for m_sp in m_sps:
            grid = ct.FourierMatrix(*geom, m_sp=m_sp, mode=ct.CT_FOURIER_GRIDDING)
            fused = ct.FourierMatrix(*geom, m_sp=m_sp, mode=ct.CT_FOURIER_FUSED)
            handles += [grid, fused]
            # the surrogate replaces the normal operator only; its right-hand
            # side is still gridded with this M_sp (Eq. surr_SBupd)
            methods += [("NUFFT, M_sp=%d" % m_sp, grid, 0), ("Convolution fusing, M_sp=%d" % m_sp, fused, 0),
                        ("Sparse surrogate 3x3, M_sp=%d" % m_sp, grid, 1)]
        for label, M, r in methods:
            u = torch.zeros(n * n, dtype=torch.float32, device=dev)

            def run(k, outer=updates):
                u.zero_()
                return M.split_bregman(f, u, 1.0, 1.0, outer, k, surrogate_r=r, square=True)

            run(inner, 3)  # warm-up: stencil build, caches
            total, st = _timed(lambda: run(inner))
            err = _rel_l1(u.cpu().double().numpy(), truth)
            no_cg, _ = _timed(lambda: run(0))
            rows.append({"N": n, "method": label, "total_s": total, "cg_s": max(total - no_cg, 0.0),
                         "rel_l1": err, "status": st["status"]})
        for F in handles:
            F.close()
        A.close()
    return rows


def stopping_rule(n=512, ds=(1, 2, 4), tols=(1e-2, 1e-4, 1e-6, 1e-8), max_updates=2000, inner=5, m_sp=6, r=2,
                  seed=7100):
    import torch

    dev = torch.device("cuda", 0)
    rows = []
    for d in ds:
        geom = _geometry(n, d)
        A, truth, f = _data(geom, seed + d, dev)
        F = ct.FourierMatrix(*geom, m_sp=m_sp, mode=ct.CT_FOURIER_FUSED)
        for label, rr in (("Convolution fusing", 0), ("Sparse surrogate, disc r=%d" % r, r)):
            u = torch.zeros(n * n, dtype=torch.float32, device=dev)
            F.split_bregman(f, u, 1.0, 1.0, 3, inner, surrogate_r=rr)  # warm-up
            reached = True
            for tol in tols:
                if not reached:
                    rows.append({"d": d, "method": label, "tol": tol, "updates": None, "time_s": None,
                                 "rel_l1": None})
                    continue
                u.zero_()
                secs, st = _timed(lambda: F.split_bregman(f, u, 1.0, 1.0, max_updates, inner,
                                                          stop_rel_update=tol, surrogate_r=rr))
                reached = st["outer_done"] < max_updates
                rows.append({"d": d, "method": label, "tol": tol,
                             "updates": st["outer_done"] if reached else None, "time_s": secs,
                             "rel_l1": _rel_l1(u.cpu().double().numpy(), truth) if reached else None})
        F.close()
        A.close()
    return rows


def _fmt(v, spec):
    return "*" if v is None else format(v, spec)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sizes", type=int, nargs="+", default=[128, 256, 512])
    ap.add_argument("--max-updates", type=int, default=2000)
    ap.add_argument("--skip-stopping", action="store_true")
    args = ap.parse_args()
    import torch

    torch.cuda.set_device(0)
    t0 = time.time()
    fixed = fixed_iterations(args.sizes)
    print("## 200 split-Bregman updates, 5 CG steps each (time in s, relative L1 error)\n")
    print("| method | " + " | ".join("N=%d total | CG | rel. L1" % n for n in args.sizes) + " |")
    print("|---|" + "---|---|---|" * len(args.sizes))
    for label in dict.fromkeys(r["method"] for r in fixed):
        cells = []
        for n in args.sizes:
            r = next(x for x in fixed if x["N"] == n and x["method"] == label)
            cells.append("%.3f | %.3f | %.4f" % (r["total_s"], r["cg_s"], r["rel_l1"]))
        print("| %s | %s |" % (label, " | ".join(cells)))
    out = {"fixed_iterations": fixed}
    if not args.skip_stopping:
        stop = stopping_rule(max_updates=args.max_updates)
        print("\n## N = 512, stop once an update falls below tol x the first (max %d updates)\n" % args.max_updates)
        print("| d | method | tol | updates | time (s) | rel. L1 |")
        print("|---|---|---|---|---|---|")
        for r in stop:
            print("| %d | %s | %g | %s | %s | %s |" % (r["d"], r["method"], r["tol"], _fmt(r["updates"], "d"),
                                                     _fmt(r["time_s"], ".3f"), _fmt(r["rel_l1"], ".4f")))
        out["stopping_rule"] = stop
    out["wall_s"] = time.time() - t0
    print("\n" + json.dumps(out))


if __name__ == "__main__":
    main()
