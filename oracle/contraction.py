"""Contraction form of the discrete IE (the remedy for high contrast that the paper names at the end of
Section 2.3, after Zhdanov et al. and Endo et al.). FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Parity unpinned against the paper itself (the
paper does not print the form); pinned here by equivalence with the conventional solution and by the
contraction property of the discrete operator (tests/test_oracle_contraction.py).

For a real positive background sigma0 the continuous operator C = I + 2 sigma0 G is a contraction (the
energy inequality of the background medium; the point-sampled discrete G exceeds that bound slightly:
the largest singular value of the discrete C is about 1.13 on a 6^3 grid of 0.5 m cells at 100 kHz,
while the spectral radius of C r stays below 1), and for a positive definite conductivity the reflection tensor
r = (sigma - sigma0 I)(sigma + sigma0 I)^-1 has spectral norm < 1. With the per-voxel tensor
    M = 2 sigma0 (sigma + sigma0 I)^-1 = I - r
and the scaled unknown u = M^-1 E, the conventional system (I - G dsigma) E = E0 (eq. 8) becomes
    (M - G dsigma M) u = E0,        E = M u,
and M - G dsigma M = I - r - 2 sigma0 G r = I - C r: the identity minus a contraction, whose spectrum
lies in the unit disc around 1 whatever the contrast. It is the conventional operator right-multiplied
by M, so the residual b - A_c u equals b - A E for E = M u: stopping rules carry over unchanged.
"""
from __future__ import annotations

import numpy as np

from .operator import FFTOperator, apply_contrast, contrast, dense_matrix  # noqa: F401 (apply_contrast re-exported)


def sigma_tensor(sigma6: np.ndarray) -> np.ndarray:
    """Absolute conductivity (..., 3, 3) from the 6-component storage (xx, yy, zz, xy, xz, yz)."""
    s = np.empty(sigma6.shape[:-1] + (3, 3))
    for k, (p, q) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        s[..., p, q] = s[..., q, p] = sigma6[..., k]
    return s


def scaling_tensor(sigma6: np.ndarray, sigma0: float) -> np.ndarray:
    """M = 2 sigma0 (sigma + sigma0 I)^-1 per voxel, (..., 3, 3)."""
    return 2.0 * sigma0 * np.linalg.inv(sigma_tensor(sigma6) + sigma0 * np.eye(3))


def reflection_tensor(sigma6: np.ndarray, sigma0: float) -> np.ndarray:
    """r = (sigma - sigma0 I)(sigma + sigma0 I)^-1 = I - M per voxel."""
    return np.eye(3) - scaling_tensor(sigma6, sigma0)


class ContractionOperator:
    """u -> (M - G dsigma M) u on one grid (FFT convolution of eq. 10 for G)."""

    def __init__(self, sigma6: np.ndarray, h: float, freq: float, sigma0: float, pad=None):
        self.M = scaling_tensor(sigma6, sigma0)
        self.conv = FFTOperator(contrast(sigma6, sigma0), h, freq, sigma0, pad)

    def field(self, u: np.ndarray) -> np.ndarray:
        """E = M u."""
        return apply_contrast(self.M, u)

    def __call__(self, u: np.ndarray) -> np.ndarray:
        return self.conv(self.field(u))


def dense_contraction_matrix(sigma6: np.ndarray, h: float, freq: float, sigma0: float) -> np.ndarray:
    """A_c = (I - K dsigma) M as a dense (3n x 3n) matrix, rows/cols ordered (component, z, y, x)."""
    A = dense_matrix(contrast(sigma6, sigma0), h, freq, sigma0)
    n = int(np.prod(sigma6.shape[:-1]))
    M = scaling_tensor(sigma6, sigma0).reshape(n, 3, 3)
    Md = np.zeros((3 * n, 3 * n))
    idx = np.arange(n)
    for p in range(3):
        for q in range(3):
            Md[p * n + idx, q * n + idx] = M[:, p, q]
    return A @ Md
