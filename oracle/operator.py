"""The discrete IE operator (I - G dsigma) of eq. 8, three ways (direct sum, FFT, dense). FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Discretisation (Section 2.2, method of moments on a uniform grid):
    (G J)_i = sum_{j != i} dv G^E(r_i - r_j) J_j  +  S J_i,
where S is the equal-volume-sphere self term (``physics.self_cell``).
Reading: the paper only says the singular cell is integrated over a sphere of equal volume; the
non-singular cells are taken at their centroids (one-point rule).

Fields are complex arrays shaped (3, nz, ny, nx) (component first, x fastest); the contrast is
dsigma = sigma - sigma0 I (Section 2.1), a real symmetric 3x3 tensor per voxel, shaped
(nz, ny, nx, 3, 3).
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft

from . import physics

FFT_WORKERS = os.cpu_count() or 1


def contrast(sigma6: np.ndarray, sigma0: float) -> np.ndarray:
    """dsigma = sigma - sigma0 I per voxel (Section 2.1), from the 6-component storage."""
    s = np.empty(sigma6.shape[:-1] + (3, 3))
    s[..., 0, 0] = sigma6[..., 0] - sigma0
    s[..., 1, 1] = sigma6[..., 1] - sigma0
    s[..., 2, 2] = sigma6[..., 2] - sigma0
    s[..., 0, 1] = s[..., 1, 0] = sigma6[..., 3]
    s[..., 0, 2] = s[..., 2, 0] = sigma6[..., 4]
    s[..., 1, 2] = s[..., 2, 1] = sigma6[..., 5]
    return s


def apply_contrast(dsig: np.ndarray, E: np.ndarray) -> np.ndarray:
    """Contrast current J = dsigma E per voxel; E (3, nz, ny, nx) -> J (3, nz, ny, nx)."""
    return np.einsum("zyxpq,qzyx->pzyx", dsig, E)


def kernel_at_offsets(dz, dy, dx, h: float, freq: float, sigma0: float) -> np.ndarray:
    """K_pq(d) = dv G^E_pq(d h) for integer offsets d != 0 and the self term at d = 0.

    ``dz, dy, dx`` are broadcastable integer arrays; returns (..., 3, 3) complex.
    """
    dz, dy, dx = np.broadcast_arrays(np.asarray(dz), np.asarray(dy), np.asarray(dx))
    R = np.stack([dx * h, dy * h, dz * h], axis=-1).astype(np.float64)
    zero = (dx == 0) & (dy == 0) & (dz == 0)
    Rsafe = np.where(zero[..., None], 1.0, R)
    dv = h**3
    K = dv * physics.electric_dyadic(Rsafe, freq, sigma0)
    K[zero] = physics.self_cell(dv, freq, sigma0) * np.eye(3)
    return K


def matvec_direct(E: np.ndarray, dsig: np.ndarray, h: float, freq: float, sigma0: float) -> np.ndarray:
    """y = (I - G dsigma) E by direct O(n^2) summation over all cell pairs (eq. 8 as written)."""
    _, nz, ny, nx = E.shape
    J = apply_contrast(dsig, E).reshape(3, -1)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    iz, iy, ix = iz.ravel(), iy.ravel(), ix.ravel()
    n = iz.size
    out = np.empty((3, n), dtype=np.complex128)
    chunk = max(1, 2_000_000 // n)
    for t0 in range(0, n, chunk):
        t = slice(t0, min(n, t0 + chunk))
        K = kernel_at_offsets(iz[t, None] - iz[None, :], iy[t, None] - iy[None, :],
                              ix[t, None] - ix[None, :], h, freq, sigma0)  # (nt, n, 3, 3)
        out[:, t] = np.einsum("tjpq,qj->pt", K, J)
    return E - out.reshape(E.shape)


def padded_kernel(shape, h: float, freq: float, sigma0: float, pad=None) -> np.ndarray:
    """Circulant embedding of K on a padded grid (pz, py, px), default twice the grid (eq. 10).

    Along an axis of length n padded to p >= 2n - 1, index m holds offset m for m <= n - 1, offset
    m - p for m >= p - (n - 1), and zero otherwise. Returns (3, 3, pz, py, px) complex.
    """
    nz, ny, nx = shape
    pz, py, px = pad if pad is not None else (2 * nz, 2 * ny, 2 * nx)
    assert pz >= 2 * nz - 1 and py >= 2 * ny - 1 and px >= 2 * nx - 1

    def offsets(n, p):
        m = np.arange(p)
        d = np.where(m <= n - 1, m, m - p)
        valid = (m <= n - 1) | (m >= p - (n - 1))
        return d, valid

    dz, vz = offsets(nz, pz)
    dy, vy = offsets(ny, py)
    dx, vx = offsets(nx, px)
    K = kernel_at_offsets(dz[:, None, None], dy[None, :, None], dx[None, None, :], h, freq, sigma0)
    valid = vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
    K[~valid] = 0.0
    return np.moveaxis(K, (-2, -1), (0, 1)).copy()


def green_spectrum(shape, h: float, freq: float, sigma0: float, pad=None) -> np.ndarray:
    """F[K_pq] on the padded grid (the precomputed Green spectra of Section 2.2), (3, 3, pz, py, px)."""
    K = padded_kernel(shape, h, freq, sigma0, pad)
    return scipy.fft.fftn(K, axes=(2, 3, 4), workers=FFT_WORKERS)


def convolve_fft(J: np.ndarray, Khat: np.ndarray) -> np.ndarray:
    """G J by eq. 10: zero-pad J, FFT, multiply by F[K_pq] and sum over q, inverse FFT, crop."""
    _, nz, ny, nx = J.shape
    pz, py, px = Khat.shape[2:]
    Jp = np.zeros((3, pz, py, px), dtype=np.complex128)
    Jp[:, :nz, :ny, :nx] = J
    Jh = scipy.fft.fftn(Jp, axes=(1, 2, 3), workers=FFT_WORKERS)
    Yh = np.einsum("pqzyx,qzyx->pzyx", Khat, Jh)
    Y = scipy.fft.ifftn(Yh, axes=(1, 2, 3), workers=FFT_WORKERS)
    return Y[:, :nz, :ny, :nx]


class FFTOperator:
    """The operator (I - G dsigma) on one rectangular grid with precomputed Green spectra."""

    def __init__(self, dsig: np.ndarray, h: float, freq: float, sigma0: float, pad=None):
        self.dsig = dsig
        self.shape = dsig.shape[:3]
        self.Khat = green_spectrum(self.shape, h, freq, sigma0, pad)

    def G(self, J: np.ndarray) -> np.ndarray:
        return convolve_fft(J, self.Khat)

    def __call__(self, E: np.ndarray) -> np.ndarray:
        return E - self.G(apply_contrast(self.dsig, E))


def dense_matrix(dsig: np.ndarray, h: float, freq: float, sigma0: float) -> np.ndarray:
    """A = I - K dsigma as a dense (3n x 3n) matrix, rows/cols ordered (component, z, y, x)."""
    nz, ny, nx = dsig.shape[:3]
    n = nz * ny * nx
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    iz, iy, ix = iz.ravel(), iy.ravel(), ix.ravel()
    K = kernel_at_offsets(iz[:, None] - iz[None, :], iy[:, None] - iy[None, :],
                          ix[:, None] - ix[None, :], h, freq, sigma0)  # (n, n, 3, 3)
    D = dsig.reshape(n, 3, 3)
    KD = np.einsum("ijpr,jrq->ipjq", K, D).reshape(3 * n, 3 * n)  # rows (i, p), cols (j, q)
    # reorder from (voxel, comp) to (comp, voxel)
    perm = np.arange(3 * n).reshape(n, 3).T.ravel()
    KD = KD[np.ix_(perm, perm)]
    return np.eye(3 * n) - KD
