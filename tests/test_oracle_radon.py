"""Pins of the FP64 Siddon oracle (A = M R, Sec. 1 Eq. objmin) to geometry.

Each test checks the oracle against something other than itself: a
hand-derived fixture, closed-form chord lengths, exact sums at axis angles,
an independent per-pixel clipping brute force, and the analytic projection
of a disk.
"""

import math
import os

import numpy as np
import pytest

from oracle import radon
from paper_1705_07497_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_two_by_two_hand_derived():
    A = radon.siddon_matrix(2, 4, 1, 3).toarray()
    want = np.zeros_like(A)
    sqrt2 = math.sqrt(2.0)
    with open(os.path.join(GOLDEN, "siddon_n2.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            q, p, expr = line.split()
            want[int(q), int(p)] = eval(expr, {"sqrt2": sqrt2})
    np.testing.assert_allclose(A, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize(
    "geom",
    [
        (16, 12, 1, 23),   # integer bin offsets: rays on pixel edges at 0 and pi/2
        (16, 30, 3, 24),   # half-integer offsets
        (15, 17, 2, 22),   # odd N, no exact axis angle except 0
        (16, 90, 3, 23),
        (8, 8, 1, 12),
    ],
)
def test_siddon_matches_per_pixel_clipping(geom):
    A = radon.siddon_matrix(*geom).toarray()
    B = radon.brute_force_matrix(*geom)
    assert np.abs(A - B).max() <= 1e-12


def _square_chord(c, s, sb, half):
    """Chord of the line x c + y s = sb through the closed square [-h, h]^2.

    Intersections with the four side lines, kept when on the side segment;
    the chord is the distance between the extreme intersection points.  A
    line lying on a side counts half of that side (the edge reading).
    """
    if s == 0.0 or c == 0.0:
        v = sb / (c if s == 0.0 else s)
        if abs(v) > half:
            return 0.0
        return half if abs(v) == half else 2.0 * half
    pts = []
    for x in (-half, half):
        y = (sb - x * c) / s
        if -half - 1e-13 <= y <= half + 1e-13:
            pts.append((x, y))
    for y in (-half, half):
        x = (sb - y * s) / c
        if -half - 1e-13 <= x <= half + 1e-13:
            pts.append((x, y))
    if len(pts) < 2:
        return 0.0
    d = 0.0
    for a in pts:
        for b in pts:
            d = max(d, math.hypot(a[0] - b[0], a[1] - b[1]))
    return d


@pytest.mark.parametrize("geom", [(64, 90, 3, 91), (128, 100, 1, 182), (33, 37, 2, 47)])
def test_row_sums_are_chord_lengths(geom):
    n, nt, keep, nb = geom
    A = radon.siddon_matrix(*geom)
    rows = np.asarray(A.sum(axis=1)).ravel()
    c, s = radon.directions(nt, keep)
    offs = radon.bin_offsets(nb)
    want = np.array([_square_chord(c[k], s[k], sb, 0.5 * n) for k in range(len(c)) for sb in offs])
    np.testing.assert_allclose(rows, want, rtol=0, atol=1e-11 * n)


@pytest.mark.parametrize("nb", [91, 92])
def test_axis_angles_column_sums_are_one(nb):
    n, nt = 64, 90
    A = radon.siddon_matrix(n, nt, 1, nb).toarray()
    for k in (0, nt // 2):  # theta = 0 and pi/2
        block = A[k * nb:(k + 1) * nb]
        np.testing.assert_array_equal(block.sum(axis=0), np.ones(n * n))
        assert set(np.unique(block)).issubset({0.0, 0.5, 1.0})


def test_direction_snapping():
    c, s = radon.directions(720, 4)
    assert (c[0], s[0]) == (1.0, 0.0)
    assert (c[90], s[90]) == (0.0, 1.0)  # k = 360 -> pi/2
    k = np.arange(180) * 4
    th = k * 3.14159265358979323846 / 720
    mask = (k != 0) & (2 * k != 720)
    np.testing.assert_array_equal(c[mask], np.cos(th[mask]))
    np.testing.assert_array_equal(s[mask], np.sin(th[mask]))


def test_entry_bounds_and_sorted_rows():
    A = radon.siddon_matrix(64, 90, 3, 91)
    assert A.data.min() >= 1e-12
    assert A.data.max() <= math.sqrt(2.0) + 1e-12
    assert A.has_sorted_indices
    assert A.nnz == 164536  # count of the 64x64, 30-angle, 91-bin workload


def test_disk_projection_is_closed_form():
    n, rho = 256, 80.0
    A = radon.siddon_matrix(n, 16, 1, inputs.n_bins_for(n))
    img = inputs.disk_image(n, rho, supersample=8)
    y = (A @ img.ravel()).reshape(16, -1)
    offs = radon.bin_offsets(inputs.n_bins_for(n))
    want = 2.0 * np.sqrt(np.maximum(rho * rho - offs * offs, 0.0))
    for k in range(16):
        err = np.linalg.norm(y[k] - want) / np.linalg.norm(want)
        assert err <= 0.02, (k, err)


def test_adjoint_identity_fp64():
    A = radon.siddon_matrix(64, 90, 3, 91)
    x = inputs.random_vector(A.shape[1], 1)
    y = inputs.random_vector(A.shape[0], 2)
    lhs = float((A @ x) @ y)
    rhs = float(x @ (A.T @ y))
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(A @ x) @ np.abs(y))


def test_quantize_rowscale_bounds():
    A = radon.siddon_matrix(32, 40, 2, 46)
    s, Q = radon.quantize_rowscale(A)
    q = Q.data.astype(np.float64)
    assert q.min() >= 0.0 and q.max() == 1.0
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    # every nonempty row has its maximum exactly at 1
    row_max = np.zeros(A.shape[0])
    np.maximum.at(row_max, rows, q)
    assert np.all(row_max[np.diff(A.indptr) > 0] == 1.0)
    # binary16 rounding: relative 2^-11 for normals, absolute 2^-25 below 2^-14
    exact = A.data / s[rows].astype(np.float64)
    bound = np.maximum(np.abs(exact) * 2.0 ** -11, 2.0 ** -25)
    assert np.all(np.abs(q - exact) <= bound)
    # known binary16 bit patterns (round to nearest even)
    assert np.float16(1.0 / 3.0).view(np.uint16) == 0x3555
    assert np.float16(0.1).view(np.uint16) == 0x2E66
    assert np.float16(1.0 + 2.0 ** -11).view(np.uint16) == 0x3C00  # tie -> even


def test_dequantized_matrix_is_within_binary16_rounding_of_a():
    """diag(s) Q reproduces A entry by entry within the rounding binary16 allows
    (2^-11 relative, 2^-25 s absolute below the normal range), and every
    nonempty row's largest entry is exactly its FP32 scale (Q = 1 there)."""
    A = radon.siddon_matrix(32, 40, 2, 46)
    s, Q = radon.quantize_rowscale(A)
    D = radon.dequantize(s, Q).toarray()
    Ad = A.toarray()
    srow = s.astype(np.float64)[:, None]
    assert np.all(np.abs(D - Ad) <= 2.0 ** -11 * np.abs(Ad) + 2.0 ** -25 * srow + 1e-15)
    assert np.all((D != 0) <= (Ad != 0))
    nonempty = np.diff(A.indptr) > 0
    np.testing.assert_array_equal(D.max(axis=1)[nonempty], s[nonempty].astype(np.float64))


@pytest.mark.parametrize("geom", [(16, 12, 1, 23), (33, 37, 2, 47), (64, 90, 3, 91)])
def test_siddon_rows_equal_the_full_matrix(geom):
    """The per-ray entry point (used at sizes too large to build whole) returns
    exactly the rows of the full matrix."""
    A = radon.siddon_matrix(*geom)
    rows = np.random.Generator(np.random.PCG64(5)).choice(A.shape[0], 40, replace=False)
    R = radon.siddon_rows(*geom, rows)
    assert (R != A[rows]).nnz == 0
    with pytest.raises(ValueError):
        radon.siddon_rows(*geom, [A.shape[0]])
