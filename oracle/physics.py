"""Closed-form physics of the IE method (Section 2.1, eqs. 1-7; Section 2.2 self term). FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Time convention e^{-i omega t}: the complex conductivity is sigma - i omega eps (Section 2.1), and
displacement currents are dropped (diffusive regime), so every conductivity here is real and
mu = mu0 everywhere.
"""
from __future__ import annotations

import numpy as np

MU0 = 4.0e-7 * np.pi


def omega(freq: float) -> float:
    return 2.0 * np.pi * freq


def k0(freq: float, sigma0: float) -> complex:
    """Background wavenumber k0 = sqrt(i omega mu0 sigma0) (eq. 7), principal branch.

    The principal root has Im k0 > 0, so e^{i k0 R} decays with distance, as it must for the
    e^{-i omega t} convention.
    """
    return complex(np.sqrt(1j * omega(freq) * MU0 * sigma0))


def scalar_green(R, k):
    """g = e^{i k R} / (4 pi R) (eq. 7)."""
    R = np.asarray(R, dtype=np.float64)
    return np.exp(1j * k * R) / (4.0 * np.pi * R)


def electric_dyadic(Rvec, freq: float, sigma0: float):
    """Electric Green's dyadic G^E = (i omega mu0 I + grad grad / sigma0) g (eq. 5), R != 0.

    ``Rvec`` has shape (..., 3) (observation minus source); returns (..., 3, 3) complex.
    Differentiating g twice gives, with R_hat = Rvec/|Rvec|,
        d_p d_q g = g [ (ikR - 1)/R^2 delta_pq + (3 - 3ikR - k^2 R^2)/R^2 Rhat_p Rhat_q ].
    """
    Rvec = np.asarray(Rvec, dtype=np.float64)
    k = k0(freq, sigma0)
    R = np.linalg.norm(Rvec, axis=-1)
    g = scalar_green(R, k)
    Rh = Rvec / R[..., None]
    iwm = 1j * omega(freq) * MU0
    a = iwm * g + (g / sigma0) * (1j * k * R - 1.0) / R**2
    b = (g / sigma0) * (3.0 - 3.0j * k * R - (k * R) ** 2) / R**2
    return a[..., None, None] * np.eye(3) + b[..., None, None] * (Rh[..., :, None] * Rh[..., None, :])


def self_cell(dv: float, freq: float, sigma0: float) -> complex:
    """Integral of G^E over a sphere of the cell's volume centred on the singularity (Section 2.2).

    With a = (3 dv / (4 pi))^{1/3}: the integral of g over the ball is ((1 - ika) e^{ika} - 1)/k^2 and
    the integral of grad grad g (including its delta part) is (1/3)(ika - 1) e^{ika} I (divergence
    theorem), so with i omega mu0 / k^2 = 1/sigma0
        int G^E dV = (1/sigma0) [ (2/3)(1 - i k a) e^{i k a} - 1 ] I.
    Returns the scalar multiplying I.
    """
    a = (3.0 * dv / (4.0 * np.pi)) ** (1.0 / 3.0)
    k = k0(freq, sigma0)
    return complex(((2.0 / 3.0) * (1.0 - 1j * k * a) * np.exp(1j * k * a) - 1.0) / sigma0)


def grad_scalar_green(Rvec, k):
    """grad g (with respect to the observation point) = g (ik - 1/R) Rhat, shape (..., 3)."""
    Rvec = np.asarray(Rvec, dtype=np.float64)
    R = np.linalg.norm(Rvec, axis=-1)
    g = scalar_green(R, k)
    return (g * (1j * k - 1.0 / R) / R)[..., None] * Rvec


def incident_E(points, src_pos, moment, freq: float, sigma0: float):
    """Background electric field of a magnetic dipole of moment m (A m^2) at ``src_pos``.

    From eqs. 1-2 in the homogeneous background, (lap + k0^2) E = -curl J^H, so E = curl(g * J^H).
    Reading (the paper prints no source formula): a magnetic dipole of moment m is the magnetic
    current J^H = i omega mu0 m delta(r - r_s); this makes H^(0) the textbook dipole field below.
    Then E^(0)(r) = i omega mu0 grad g(r - r_s) x m.
    """
    Rvec = np.asarray(points, dtype=np.float64) - np.asarray(src_pos, dtype=np.float64)
    k = k0(freq, sigma0)
    gg = grad_scalar_green(Rvec, k)
    m = np.asarray(moment, dtype=np.complex128)
    return 1j * omega(freq) * MU0 * np.cross(gg, m)


def incident_H(points, src_pos, moment, freq: float, sigma0: float):
    """Background magnetic field of the same dipole: H^(0) = (k0^2 g I + grad grad g) m.

    Follows from eq. 1, H = (curl E - J^H)/(i omega mu0), off the source point.
    """
    Rvec = np.asarray(points, dtype=np.float64) - np.asarray(src_pos, dtype=np.float64)
    k = k0(freq, sigma0)
    R = np.linalg.norm(Rvec, axis=-1)
    g = scalar_green(R, k)
    Rh = Rvec / R[..., None]
    a = g * (k * k + (1j * k * R - 1.0) / R**2)
    b = g * (3.0 - 3.0j * k * R - (k * R) ** 2) / R**2
    m = np.asarray(moment, dtype=np.complex128)
    return a[..., None] * m + b[..., None] * Rh * (Rh @ m)[..., None]


def scattered_H(points, cell_centres, J, dv: float, freq: float, sigma0: float):
    """Scattered magnetic field of eq. 4 with G^H from eq. 6 (midpoint rule, one point per cell).

    curl of the grad-grad part of G^E vanishes, so G^H J = (i omega mu0)^{-1} curl(i omega mu0 g J)
    = grad g x J, and
        H^s(r) = sum_j dv grad g(r - r_j) x J_j,   J = delta_sigma E (the contrast current).
    ``cell_centres`` (n, 3), ``J`` (n, 3) complex, ``points`` (n_rx, 3). Returns (n_rx, 3).
    """
    k = k0(freq, sigma0)
    out = np.zeros((len(points), 3), dtype=np.complex128)
    for r, p in enumerate(np.asarray(points, dtype=np.float64)):
        gg = grad_scalar_green(p[None, :] - cell_centres, k)
        out[r] = dv * np.sum(np.cross(gg, J), axis=0)
    return out
