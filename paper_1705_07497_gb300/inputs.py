"""Seeded synthetic inputs: geometries, random-ellipse phantoms, noise draws.

This module holds no arithmetic of the reconstruction method; it only makes
the inputs that both the library and its tests consume.  The paper's
experiments (Sec. 4) use the Shepp-Logan phantom, which is not reproduced
here: every workload uses seeded random ellipses instead.

Phantom recipe (one reading of "random ellipses"): 10 additive ellipses in
normalised coordinates [-1, 1]^2 with centres uniform in the disc of radius
0.5, semi-axes U[0.05, 0.4], rotation U[0, pi), intensity U[0, 1]; every
ellipse is clipped to the disc of radius 0.9 so that the object stays inside
the inscribed circle and several pixels away from the edges (Sec. 3.2 asks
for r pixels).  A pixel takes the value of the indicator at its centre.
"""

import math

import numpy as np


def n_bins_for(n):
    """Detector bins of width 1 covering the image diagonal: ceil(sqrt(2) N)."""
    return int(math.ceil(math.sqrt(2.0) * n))


# Workloads.  Sizes follow the paper's regime (N up to 512, N pi / (4 d)
# angles, hundreds of Bregman updates); each entry names what it is.
WORKLOADS = {
    # 64x64, 90 angles keeping every 3rd, 91 bins, 20 x 10, alpha 1, lambda 0.1
    "plain_64": dict(n=64, n_angles_total=90, keep_every=3, n_bins=91, batch=1,
                     outer=20, inner=10, alpha=1.0, lam=0.1, noise="none", seed=0),
    # 512x512, 720 angles keeping every 4th, 725 bins, 1% Gaussian noise, 50 x 20
    "slice_512": dict(n=512, n_angles_total=720, keep_every=4, n_bins=725, batch=1,
                      outer=50, inner=20, alpha=1.0, lam=1.0, noise="gauss", sigma_rel=0.01,
                      seed=1000),
    # the 512x512 slice reconstructed by Chambolle-Pock: 50 primal-dual updates,
    # each resolvent (Eq. PD_resolve) by 20 CG steps, tau = sigma = 0.99 / sqrt(8)
    "cp_512": dict(n=512, n_angles_total=720, keep_every=4, n_bins=725, batch=1, solver="cp",
                   outer=50, inner=20, alpha=1.0, tau=0.35, sigma=0.35, theta=1.0, noise="gauss",
                   sigma_rel=0.01, seed=1000),
    # the p = 2 normal equations (Eq. KKT) on the same slice: (alpha A^T A +
    # grad^T grad) u = alpha A^T f by a fixed number of CG steps from zero
    "kkt_512": dict(n=512, n_angles_total=720, keep_every=4, n_bins=725, batch=1, solver="kkt",
                    cg_iters=200, alpha=1.0, noise="gauss", sigma_rel=0.01, seed=1000),
    # 256 slices of 512x512 on the same geometry, Poisson noise at 1e4 counts/bin,
    # FP16 storage with a per-row FP32 scale (no FP32 residual refresh: it
    # measured worse than none with double-float recurrences)
    "batch_512x256": dict(n=512, n_angles_total=720, keep_every=4, n_bins=725, batch=256,
                          outer=50, inner=20, alpha=1.0, lam=1.0, noise="poisson",
                          counts=1e4, seed=2000, refresh_every=0, fp16=True),
    # 64 problems of different geometries in one call: N and the angle count
    # drawn uniformly per problem (ragged_problems), all angles kept,
    # ceil(sqrt(2) N) bins, FP16 storage, 1% Gaussian noise
    "ragged_64": dict(count=64, sizes=(128, 256, 512, 1024), angle_counts=(60, 120, 360, 900),
                      outer=50, inner=20, alpha=1.0, lam=1.0, noise="gauss", sigma_rel=0.01,
                      seed=4000, fp16=True),
    # the 512x512 slice through the Fourier-domain data term: Gaussian gridding
    # with window half-width 6 (six digits) and the fused matrix
    "fourier_512": dict(n=512, n_angles_total=720, keep_every=4, n_bins=725, outer=50, inner=20,
                        alpha=1.0, lam=1.0, noise="gauss", sigma_rel=0.01, seed=1000, m_sp=6,
                        fourier_mode=0),
    # 16 slices of 256x256, 360 angles keeping every 2nd, 363 bins, 10 unrolled updates
    "grad_256x16": dict(n=256, n_angles_total=360, keep_every=2, n_bins=363, batch=16,
                        outer=10, inner=10, alpha=1.0, lam=1.0, noise="gauss", sigma_rel=0.01,
                        seed=3000),
}


def ragged_problems(wl):
    """(n, n_angles_total, keep_every, n_bins, seed) of every problem of a ragged workload:
    N and the angle count drawn uniformly (PCG64, seed + i) from the workload's lists."""
    out = []
    for i in range(wl["count"]):
        rng = np.random.Generator(np.random.PCG64(wl["seed"] + i))
        n = int(wl["sizes"][rng.integers(len(wl["sizes"]))])
        a = int(wl["angle_counts"][rng.integers(len(wl["angle_counts"]))])
        out.append((n, a, 1, n_bins_for(n), wl["seed"] + i))
    return out


def ellipse_params(seed, n_ellipses=10):
    """Random ellipse parameters (cx, cy, a, b, phi, value) for one phantom."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_ellipses):
        rad = 0.5 * math.sqrt(rng.uniform(0.0, 1.0))
        ang = rng.uniform(0.0, 2.0 * math.pi)
        cx, cy = rad * math.cos(ang), rad * math.sin(ang)
        a, b = rng.uniform(0.05, 0.4), rng.uniform(0.05, 0.4)
        phi = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.0, 1.0)
        out.append((cx, cy, a, b, phi, val))
    return out


def ellipse_phantom(n, seed, n_ellipses=10, supersample=1):
    """N x N float64 phantom of additive random ellipses (seeded, PCG64).

    With supersample > 1 each pixel is the mean over supersample^2 sub-points.
    """
    ss = supersample
    t = (np.arange(n * ss, dtype=np.float64) + 0.5) / ss  # sub-pixel centres in [0, n)
    coord = (t - 0.5 * n) / (0.5 * n)  # normalised, x along j, y along i
    y, x = np.meshgrid(coord, coord, indexing="ij")
    img = np.zeros_like(x)
    inside = x * x + y * y <= 0.9 * 0.9
    for cx, cy, a, b, phi, val in ellipse_params(seed, n_ellipses):
        c, s = math.cos(phi), math.sin(phi)
        xr = (x - cx) * c + (y - cy) * s
        yr = -(x - cx) * s + (y - cy) * c
        img += val * (((xr / a) ** 2 + (yr / b) ** 2 <= 1.0) & inside)
    if ss > 1:
        img = img.reshape(n, ss, n, ss).mean(axis=(1, 3))
    return img


def disk_image(n, radius_px, supersample=8):
    """Supersampled indicator of a centred disk of the given radius in pixels."""
    ss = supersample
    t = (np.arange(n * ss, dtype=np.float64) + 0.5) / ss - 0.5 * n
    y, x = np.meshgrid(t, t, indexing="ij")
    img = (x * x + y * y <= radius_px * radius_px).astype(np.float64)
    return img.reshape(n, ss, n, ss).mean(axis=(1, 3))


def standard_normal(shape, seed):
    """Seeded N(0, 1) draws (PCG64) for additive Gaussian noise."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)


def gaussian_noisy(clean, sigma_rel, seed):
    """clean + sigma * z with sigma = sigma_rel * max(clean)."""
    sigma = sigma_rel * float(np.max(clean))
    return clean + sigma * standard_normal(clean.shape, seed)


def poisson_noisy(clean, counts, seed):
    """Scaled-projection Poisson model: Poisson(c * clean) / c, c = counts / max(clean)."""
    c = counts / float(np.max(clean))
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.poisson(c * np.maximum(clean, 0.0)) / c


def random_vector(size, seed, dtype=np.float64):
    """Seeded U[-1, 1) vector for operator tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size).astype(dtype)
