"""The seeded input recipe: random-ellipse phantoms, noise models, ragged
draws and bin counts are what the design states, and reproducible."""

import math

import numpy as np

from paper_1705_07497_gb300 import inputs


def test_bins_cover_the_diagonal():
    for n in (16, 64, 128, 256, 512, 1024):
        nb = inputs.n_bins_for(n)
        assert nb - 1 < math.sqrt(2.0) * n <= nb
    assert [inputs.n_bins_for(n) for n in (64, 256, 512, 1024)] == [91, 363, 725, 1449]


def test_phantom_is_seeded_nonnegative_and_inside_the_clipping_disc():
    n = 128
    a = inputs.ellipse_phantom(n, 7)
    assert np.array_equal(a, inputs.ellipse_phantom(n, 7))
    assert not np.array_equal(a, inputs.ellipse_phantom(n, 8))
    assert a.min() >= 0.0 and a.max() > 0.0 and a.max() <= 10.0
    c = (np.arange(n) + 0.5 - 0.5 * n) / (0.5 * n)
    y, x = np.meshgrid(c, c, indexing="ij")
    assert np.all(a[x * x + y * y > 0.81] == 0.0)
    # the object keeps clear of the image edges (the surrogate's translates
    # near the boundary are dropped): at least 0.05 N pixels of margin
    margin = int(0.05 * n)
    assert np.all(a[:margin] == 0) and np.all(a[-margin:] == 0)
    assert np.all(a[:, :margin] == 0) and np.all(a[:, -margin:] == 0)


def test_ellipse_parameters_follow_the_stated_distributions():
    params = np.array([p for s in range(200) for p in inputs.ellipse_params(s)])
    cx, cy, a, b, phi, val = params.T
    assert np.all(cx * cx + cy * cy <= 0.25)
    assert a.min() >= 0.05 and a.max() <= 0.4 and b.min() >= 0.05 and b.max() <= 0.4
    assert phi.min() >= 0.0 and phi.max() < math.pi
    assert val.min() >= 0.0 and val.max() < 1.0
    # centres uniform in the disc: the squared radius is uniform on [0, 0.25]
    r2 = (cx * cx + cy * cy) / 0.25
    assert abs(r2.mean() - 0.5) < 0.03 and abs(np.median(r2) - 0.5) < 0.05


def test_gaussian_noise_level_is_one_percent_of_the_maximum():
    clean = np.linspace(0.0, 50.0, 200000)
    noisy = inputs.gaussian_noisy(clean, 0.01, 3)
    sd = float(np.std(noisy - clean))
    assert abs(sd - 0.5) < 0.01
    assert np.array_equal(noisy, inputs.gaussian_noisy(clean, 0.01, 3))


def test_poisson_noise_scales_counts_to_the_maximum_bin():
    clean = np.full(200000, 20.0)
    clean[0] = 40.0  # the maximum bin gets 1e4 expected counts
    noisy = inputs.poisson_noisy(clean, 1e4, 5)
    c = 1e4 / 40.0
    rest = noisy[1:]
    assert abs(rest.mean() - 20.0) < 0.01
    # Poisson(c y) / c has variance y / c
    assert abs(rest.var() / (20.0 / c) - 1.0) < 0.02
    assert np.allclose(rest * c, np.round(rest * c))


def test_ragged_problems_are_seeded_uniform_draws():
    wl = inputs.WORKLOADS["ragged_64"]
    probs = inputs.ragged_problems(wl)
    assert probs == inputs.ragged_problems(wl)
    assert len(probs) == 64
    for i, (n, a, d, nb, seed) in enumerate(probs):
        assert n in wl["sizes"] and a in wl["angle_counts"]
        assert d == 1 and nb == inputs.n_bins_for(n) and seed == wl["seed"] + i
    assert {p[0] for p in probs} == set(wl["sizes"])
    assert {p[1] for p in probs} == set(wl["angle_counts"])
