"""FP64 oracle of the restricted Radon transform A = M R as a sparse matrix.

Test infrastructure only (see the package docstring).

Sec. 1 (Eq. objmin) defines the data term through M R: R is the Radon
transform and M keeps the angles along which measurements are taken.  The
paper never discretises R in the image domain; the reading used here (and by
the CUDA library, written independently) is the exact intersection length of
each ray with each pixel:

  image N x N, pixel (i, j) covers x in [j - N/2, j - N/2 + 1] and
  y in [i - N/2, i - N/2 + 1]; column p = i * N + j;
  theta_k = k pi / n_total, kept when k % keep_every == 0 (the row selector M);
  bin b at offset s_b = b - (n_bins - 1) / 2; ray (k, b) is the line
  x cos(theta_k) + y sin(theta_k) = s_b; row q = (k / keep_every) n_bins + b;
  a ray exactly on a grid line gives half its length to each adjacent pixel;
  theta exactly 0 or pi/2 use the exact direction cosines; lengths < 1e-12
  are dropped.
"""

import math

import numpy as np
import scipy.sparse as sp

from . import _native

MIN_LEN = 1e-12


def num_kept(n_total, keep_every):
    """Number of angles the row selector M keeps (k = 0, d, 2d, ... < n_total)."""
    return (n_total + keep_every - 1) // keep_every


def directions(n_total, keep_every):
    """(cos, sin) of every kept angle, as the C tracer uses them."""
    L = _native.lib()
    m = num_kept(n_total, keep_every)
    c = np.zeros(m)
    s = np.zeros(m)
    L.oracle_directions(
        n_total,
        keep_every,
        c.ctypes.data_as(_native.ctypes.POINTER(_native.ctypes.c_double)),
        s.ctypes.data_as(_native.ctypes.POINTER(_native.ctypes.c_double)),
    )
    return c, s


def bin_offsets(n_bins):
    return np.arange(n_bins, dtype=np.float64) - 0.5 * (n_bins - 1)


def siddon_matrix(n, n_total, keep_every, n_bins):
    """Exact FP64 system matrix A (rows = kept angle x bin, cols = pixels).

    Returns a ``scipy.sparse.csr_matrix`` with sorted column indices, built by
    Siddon's ray tracing in ``siddon.c`` (count pass, then fill pass).
    """
    L = _native.lib()
    rows = num_kept(n_total, keep_every) * n_bins
    row_nnz = np.zeros(rows, dtype=np.int64)
    ct = _native.ctypes
    total = L.oracle_siddon_count(n, n_total, keep_every, n_bins, row_nnz.ctypes.data_as(ct.POINTER(ct.c_int64)))
    if total < 0:
        raise ValueError("invalid geometry")
    row_ptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(row_nnz, out=row_ptr[1:])
    cols = np.zeros(total, dtype=np.int32)
    vals = np.zeros(total, dtype=np.float64)
    rc = L.oracle_siddon_fill(
        n,
        n_total,
        keep_every,
        n_bins,
        row_ptr.ctypes.data_as(ct.POINTER(ct.c_int64)),
        cols.ctypes.data_as(ct.POINTER(ct.c_int32)),
        vals.ctypes.data_as(ct.POINTER(ct.c_double)),
    )
    if rc != 0:
        raise RuntimeError("siddon fill failed: %d" % rc)
    return sp.csr_matrix((vals, cols, row_ptr), shape=(rows, n * n))


def siddon_rows(n, n_total, keep_every, n_bins, rows):
    """Rows `rows` of A (same tracer as siddon_matrix) as a CSR matrix of
    len(rows) x N^2, for geometries too large to build whole."""
    L = _native.lib()
    ct = _native.ctypes
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    i64p = ct.POINTER(ct.c_int64)
    nnz = np.zeros(len(rows), dtype=np.int64)
    total = L.oracle_siddon_rows(n, n_total, keep_every, n_bins, len(rows), rows.ctypes.data_as(i64p), None,
                                 nnz.ctypes.data_as(i64p), None, None)
    if total < 0:
        raise ValueError("invalid geometry or row")
    row_ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(nnz, out=row_ptr[1:])
    cols = np.zeros(total, dtype=np.int32)
    vals = np.zeros(total, dtype=np.float64)
    rc = L.oracle_siddon_rows(n, n_total, keep_every, n_bins, len(rows), rows.ctypes.data_as(i64p),
                              row_ptr.ctypes.data_as(i64p), nnz.ctypes.data_as(i64p),
                              cols.ctypes.data_as(ct.POINTER(ct.c_int32)), vals.ctypes.data_as(ct.POINTER(ct.c_double)))
    if rc < 0:
        raise RuntimeError("oracle_siddon_rows failed (%d)" % rc)
    return sp.csr_matrix((vals, cols, row_ptr), shape=(len(rows), n * n))


def _clip_length(x0, y0, dx, dy, bx0, bx1, by0, by1):
    """Length of the line (x0 + t dx, y0 + t dy) inside the box (Liang-Barsky).

    A line lying exactly on the box's boundary counts half of the boundary
    segment (the half-and-half reading for rays on pixel edges).
    """
    factor = 1.0
    lo, hi = -math.inf, math.inf
    for p0, dp, b0, b1 in ((x0, dx, bx0, bx1), (y0, dy, by0, by1)):
        if dp == 0.0:
            if p0 < b0 or p0 > b1:
                return 0.0
            if p0 == b0 or p0 == b1:
                factor = 0.5
            continue
        t0, t1 = (b0 - p0) / dp, (b1 - p0) / dp
        if t0 > t1:
            t0, t1 = t1, t0
        lo, hi = max(lo, t0), min(hi, t1)
    length = max(0.0, hi - lo) * factor
    return length if length >= MIN_LEN else 0.0


def brute_force_matrix(n, n_total, keep_every, n_bins):
    """Dense A by clipping every ray against every pixel box independently.

    Pure Python; meant for N <= 16.  Independent of the Siddon tracer: no
    plane lists, no merge, no midpoint lookup.
    """
    c, s = directions(n_total, keep_every)
    offs = bin_offsets(n_bins)
    A = np.zeros((len(c) * n_bins, n * n))
    half = 0.5 * n
    for kk in range(len(c)):
        for b, sb in enumerate(offs):
            x0, y0, dx, dy = sb * c[kk], sb * s[kk], -s[kk], c[kk]
            q = kk * n_bins + b
            for i in range(n):
                for j in range(n):
                    A[q, i * n + j] = _clip_length(
                        x0, y0, dx, dy, j - half, j - half + 1.0, i - half, i - half + 1.0
                    )
    return A


def quantize_rowscale(A):
    """FP16 storage form A ~ diag(s) Q of a CSR matrix.

    s_q = fp32(max_p A_qp), Q_qp = fp16(A_qp / s_q) rounded to nearest even
    (numpy's IEEE-754 binary16 conversion).  The adjoint reuses Q and s so the
    quantised normal operator stays exactly symmetric.
    Returns (s float32 [rows], Q as CSR with float16 data).
    """
    A = sp.csr_matrix(A)
    rows = A.shape[0]
    s = np.zeros(rows, dtype=np.float32)
    lens = np.diff(A.indptr)
    nz = lens > 0
    s[nz] = np.maximum.reduceat(A.data, A.indptr[:-1][nz]).astype(np.float32)
    scale = np.repeat(s.astype(np.float64), lens)
    q = (A.data / scale).astype(np.float16)
    Q = sp.csr_matrix((q, A.indices.copy(), A.indptr.copy()), shape=A.shape)
    return s, Q


def dequantize(s, Q):
    """FP64 matrix diag(s) Q (what the FP16 storage form represents)."""
    Qd = sp.csr_matrix((Q.data.astype(np.float64), Q.indices, Q.indptr), shape=Q.shape)
    return sp.diags(s.astype(np.float64)) @ Qd
