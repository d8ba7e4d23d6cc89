"""FP64 oracle of the Fourier-domain data term (Sec. 2, Eqs. four_obj, SBFFT)
and of its fast evaluation by Gaussian gridding and convolution fusing
(Sec. 3.1, Eq. fusedop).

Test infrastructure only (see the package docstring).

Readings taken where the paper is silent or garbled:
  * Samples.  By the Fourier slice theorem (Sec. 2) the 1-D Fourier transform
    of the projection at angle theta is the 2-D transform of the image on the
    line rho (cos theta, sin theta).  The discrete samples are the kept angles
    of the Siddon geometry and rho_m = 2 pi (m - floor(n_bins/2)) / n_bins,
    m = 0..n_bins-1 (the DFT frequencies of a projection with unit bin
    spacing); sample index j = k' n_bins + m, the shape of the sinogram.
  * The nonuniform transform.  (F mu)_j = n_bins^{-1/2} sum_p mu_p
    exp(-i omega_j . x_p) with x_p the pixel centre of the Siddon geometry,
    x = j - N/2 + 1/2, y = i - N/2 + 1/2.  The data are the DFTs of the
    measured projections, fhat_j = n_bins^{-1/2} sum_b f_b exp(-i rho_m s_b),
    s_b = b - (n_bins - 1)/2.  The factor n_bins^{-1/2} makes the DFT of a
    projection unitary, so that ||F mu - fhat|| is the sinogram residual of
    point-sampled pixels and alpha, lambda keep their meaning.
  * Real images.  The unknown is real, so the normal operator of Eq. SBFFT
    is Re(F^H F) and its right-hand side alpha Re(F^H fhat) (for an even
    number of bins the sample set is not symmetric under omega -> -omega and
    F^H F mu has an imaginary part).
  * Gaussian gridding (Greengard and Lee, as reviewed in Sec. 3.1): fine grid
    of M_r = 2N points per dimension at eta_m = 2 pi m / M_r; tau = M_sp / N^2
    unless given; 2-D kernel the product of 1-D Gaussians
    exp(-(x - eta)^2 / (4 tau)) of the nearest periodic image; deconvolution
    E(k) = sqrt(pi / tau) exp(k^2 tau) per dimension (the paper's diagonal
    "A", Eq. fusedop).  The window: Sec. 3.1 describes it once as the 2 M_sp
    grid points closest to a sample and once as the set |m_j - m| <= M_sp
    with m_j = floor(x_j M_r / 2 pi); the explicit set (2 M_sp + 1 points per
    dimension) is taken.
  * Convolution fusing (Eq. fusedop): with G the sample-by-grid matrix of
    kernel weights, F = c Phi G FFT Z E (Z zero padding, Phi the unit phases
    of the half-pixel centre offset, c = 1 / (M_r^2 n_bins^{1/2})) and the
    fused matrix is C = G^T G, a sparse real symmetric matrix whose entries
    lie on the offsets |d| <= 2 M_sp of the periodic fine grid.
"""

import math

import numpy as np
import scipy.sparse as sp

from . import radon


# --------------------------------------------------------------------------
# Geometry of the Fourier samples and the exact nonuniform DFT
# --------------------------------------------------------------------------
def radial_frequencies(n_bins):
    """rho_m = 2 pi (m - floor(n_bins/2)) / n_bins, m = 0..n_bins-1."""
    return 2.0 * math.pi * (np.arange(n_bins, dtype=np.float64) - (n_bins // 2)) / n_bins


def sample_points(n_total, keep_every, n_bins):
    """(omega_x, omega_y) of every sample, row j = k' n_bins + m."""
    c, s = radon.directions(n_total, keep_every)
    rho = radial_frequencies(n_bins)
    return np.outer(c, rho).ravel(), np.outer(s, rho).ravel()


def pixel_centres(n):
    """(x, y) of pixel (i, j) for the flattened index p = i n + j."""
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return (jj - n / 2.0 + 0.5).ravel(), (ii - n / 2.0 + 0.5).ravel()


def nudft_matrix(n, n_total, keep_every, n_bins):
    """Dense F (J x N^2): the nonuniform DFT by its definition (brute force)."""
    wx, wy = sample_points(n_total, keep_every, n_bins)
    x, y = pixel_centres(n)
    return np.exp(-1j * (np.outer(wx, x) + np.outer(wy, y))) / math.sqrt(n_bins)


def sinogram_dft(f, n_kept, n_bins):
    """fhat[k', m] = n_bins^{-1/2} sum_b f[k', b] exp(-i rho_m s_b), by its definition."""
    f = np.asarray(f, dtype=np.float64).reshape(n_kept, n_bins)
    phase = np.exp(-1j * np.outer(radial_frequencies(n_bins), radon.bin_offsets(n_bins)))
    return (f @ phase.T).ravel() / math.sqrt(n_bins)


def point_response(n, n_total, keep_every, n_bins, r):
    """h(d) = Re(F^H F e_c)[c + d] = n_bins^{-1} sum_j cos(omega_j . d) for
    |d_i|, |d_j| <= r: the exact point response of the Fourier normal operator
    (translation invariant), as a (2r+1) x (2r+1) array indexed [di + r, dj + r]."""
    wx, wy = sample_points(n_total, keep_every, n_bins)
    h = np.zeros((2 * r + 1, 2 * r + 1))
    for di in range(-r, r + 1):
        for dj in range(-r, r + 1):
            h[di + r, dj + r] = np.cos(wx * dj + wy * di).sum() / n_bins
    return h


# --------------------------------------------------------------------------
# Gaussian gridding (Sec. 3.1)
# --------------------------------------------------------------------------
def default_tau(n, m_sp):
    """tau = M_sp / N^2 (Sec. 3.1: 6 digits at M_sp = 6, 12 digits at M_sp = 12)."""
    return m_sp / float(n * n)


def deconvolution(n, tau):
    """E(k) = sqrt(pi / tau) exp(k^2 tau) for k = -N/2 .. N/2 - 1."""
    k = np.arange(n, dtype=np.float64) - n // 2
    return math.sqrt(math.pi / tau) * np.exp(k * k * tau)


def window_weights(w, m_r, m_sp, tau):
    """Base points m_j = floor(w M_r / 2 pi) and the 1-D weights
    exp(-(w - 2 pi (m_j + t) / M_r)^2 / (4 tau)) for t = -M_sp .. M_sp."""
    base = np.floor(w * m_r / (2.0 * math.pi)).astype(np.int64)
    t = np.arange(-m_sp, m_sp + 1)
    eta = 2.0 * math.pi * (base[:, None] + t[None, :]) / m_r
    return base, np.exp(-((w[:, None] - eta) ** 2) / (4.0 * tau))


class Gridding:
    """Gaussian gridding of the samples onto the 2N x 2N periodic fine grid."""

    def __init__(self, n, n_total, keep_every, n_bins, m_sp, tau=None):
        self.n, self.n_bins, self.m_sp = n, n_bins, m_sp
        self.tau = default_tau(n, m_sp) if tau is None else float(tau)
        self.m_r = 2 * n
        self.wx, self.wy = sample_points(n_total, keep_every, n_bins)
        self.E = deconvolution(n, self.tau)
        self.phase = np.exp(-0.5j * (self.wx + self.wy))  # half-pixel centre offset
        self.G = self._interp_matrix()
        self._C = None

    def _interp_matrix(self):
        """G[j, my * M_r + mx] = gx_j(mx) gy_j(my) over the window (indices wrapped)."""
        m_r, m_sp = self.m_r, self.m_sp
        bx, gx = window_weights(self.wx, m_r, m_sp, self.tau)
        by, gy = window_weights(self.wy, m_r, m_sp, self.tau)
        t = np.arange(-m_sp, m_sp + 1)
        J, W = len(self.wx), len(t)
        ix = (bx[:, None] + t[None, :]) % m_r
        iy = (by[:, None] + t[None, :]) % m_r
        rows = np.repeat(np.arange(J), W * W)
        cols = (iy[:, :, None] * m_r + ix[:, None, :]).ravel()
        vals = (gy[:, :, None] * gx[:, None, :]).ravel()
        return sp.csr_matrix((vals, (rows, cols)), shape=(J, m_r * m_r))

    def scale(self):
        return 1.0 / (self.m_r * self.m_r * math.sqrt(self.n_bins))

    def pad(self, mu):
        """Z E mu: the deconvolved image at fine-grid index (k mod M_r) per axis."""
        n, m_r = self.n, self.m_r
        P = np.zeros((m_r, m_r), dtype=np.complex128)
        k = (np.arange(n) - n // 2) % m_r
        P[np.ix_(k, k)] = np.asarray(mu, dtype=np.float64).reshape(n, n) * np.outer(self.E, self.E)
        return P

    def crop(self, P):
        """E Z^T P (complex): the inverse of ``pad``'s placement."""
        n, m_r = self.n, self.m_r
        k = (np.arange(n) - n // 2) % m_r
        return P[np.ix_(k, k)] * np.outer(self.E, self.E)

    def forward(self, mu):
        """F mu (type-2 NUFFT): c Phi G FFT Z E mu."""
        h = np.fft.fft2(self.pad(mu)).ravel()
        return self.scale() * self.phase * (self.G @ h)

    def adjoint(self, c):
        """Re(F^H c) (type-1 NUFFT): c E Z^T FFT^H G^T conj(Phi) c, real part."""
        s = self.G.T @ (np.conj(self.phase) * np.asarray(c))
        m_r = self.m_r
        P = np.fft.ifft2(s.reshape(m_r, m_r)) * (m_r * m_r)
        return np.real(self.scale() * self.crop(P)).ravel()

    def fused_matrix(self):
        """C = G^T G (Eq. fusedop's B* B), M_r^2 x M_r^2 (formed once)."""
        if self._C is None:
            self._C = (self.G.T @ self.G).tocsr()
        return self._C

    def normal_fused(self, mu, C=None):
        """Re(F^H F mu) evaluated as E Z^T FFT^H C FFT Z E mu (2 FFTs, one
        sparse product, 2 diagonals), times c^2."""
        C = self.fused_matrix() if C is None else C
        m_r = self.m_r
        h = np.fft.fft2(self.pad(mu)).ravel()
        P = np.fft.ifft2((C @ h).reshape(m_r, m_r)) * (m_r * m_r)
        return np.real(self.scale() ** 2 * self.crop(P)).ravel()

    def normal(self, mu):
        """Re(F^H F mu) as the NUFFT pair (type 2, then type 1), unfused."""
        return self.adjoint(self.forward(mu))


class FourierSystem:
    """The data operator of Eq. four_obj for the solvers of ``tv``: ``A @ mu``
    is F mu (complex samples), ``A.T @ c`` is Re(F^H c).  ``gridding`` = None
    uses the exact nonuniform DFT, else the Gaussian gridding (NUFFT)."""

    def __init__(self, n, n_total, keep_every, n_bins, gridding=None):
        self.n = n
        self.g = gridding
        self.F = nudft_matrix(n, n_total, keep_every, n_bins) if gridding is None else None
        self.T = _Adjoint(self)

    def __matmul__(self, mu):
        return self.F @ mu if self.g is None else self.g.forward(mu)

    def normal(self, mu):
        if self.g is None:
            return np.real(self.F.conj().T @ (self.F @ mu))
        return self.g.normal(mu)


class _Adjoint:
    def __init__(self, sysm):
        self.s = sysm

    def __matmul__(self, c):
        if self.s.g is None:
            return np.real(self.s.F.conj().T @ c)
        return self.s.g.adjoint(c)
