"""Pins for the oracle's closed-form physics (eqs. 5-7, the self term, the dipole fields, eq. 4).

Each check compares against something other than the formula itself: finite differences of the
scalar Green's function, textbook limits, numerical quadrature, or Maxwell's equations.
"""
import numpy as np
import pytest

from oracle import physics
from oracle.operator import contrast

F, S0 = 2.0e4, 0.3  # a frequency / background where k0 R ~ 1 over a few metres


def fd_hessian_g(R, k, step):
    H = np.zeros((3, 3), dtype=complex)
    e = np.eye(3) * step
    g = lambda r: physics.scalar_green(np.linalg.norm(r), k)
    for p in range(3):
        for q in range(3):
            H[p, q] = (g(R + e[p] + e[q]) - g(R + e[p] - e[q]) - g(R - e[p] + e[q])
                       + g(R - e[p] - e[q])) / (4 * step * step)
    return H


def test_k0_branch_decays():
    k = physics.k0(F, S0)
    assert k.imag > 0 and k.real > 0
    assert abs(k * k - 1j * physics.omega(F) * physics.MU0 * S0) < 1e-12 * abs(k * k)


@pytest.mark.parametrize("R", [np.array([0.7, -0.3, 1.1]), np.array([3.0, 2.0, -4.0]),
                               np.array([0.0, 0.0, 2.5]), np.array([0.25, 0.0, 0.0])])
def test_electric_dyadic_matches_finite_difference_hessian(R):
    k = physics.k0(F, S0)
    G = physics.electric_dyadic(R, F, S0)
    step = 1e-4 * np.linalg.norm(R)
    Gfd = 1j * physics.omega(F) * physics.MU0 * physics.scalar_green(np.linalg.norm(R), k) * np.eye(3) \
        + fd_hessian_g(R, k, step) / S0
    assert np.max(np.abs(G - Gfd)) < 1e-6 * np.max(np.abs(G))


def test_electric_dyadic_symmetric_and_even():
    rng = np.random.default_rng(1)
    R = rng.normal(size=(20, 3))
    G = physics.electric_dyadic(R, F, S0)
    assert np.allclose(G, np.swapaxes(G, -1, -2), rtol=0, atol=1e-14 * np.abs(G).max())
    assert np.allclose(G, physics.electric_dyadic(-R, F, S0), rtol=1e-14)


def test_electric_dyadic_static_limit():
    # k0 -> 0: grad grad (1/(4 pi R)) / sigma0 = (3 Rhat Rhat - I) / (4 pi sigma0 R^3)
    R = np.array([0.4, -1.2, 0.9])
    r = np.linalg.norm(R)
    Rh = R / r
    G = physics.electric_dyadic(R, 1e-9, S0)
    G_static = (3 * np.outer(Rh, Rh) - np.eye(3)) / (4 * np.pi * S0 * r**3)
    assert np.allclose(G, G_static, rtol=1e-6, atol=1e-12)


def test_self_cell_static_depolarisation():
    # a small sphere: the integral tends to -I/(3 sigma0) (textbook depolarisation factor 1/3)
    assert abs(physics.self_cell(1e-12, F, S0) - (-1.0 / (3 * S0))) < 1e-6 / S0


def test_self_cell_matches_quadrature():
    # principal-value quadrature of the full tensor over eps < r < a, plus the delta part of the
    # grad grad term inside the small ball (-I/(3 sigma0), static depolarisation)
    dv = 0.5**3
    a = (3 * dv / (4 * np.pi)) ** (1 / 3)
    f, s0 = 4e5, 0.1
    xr, wr = np.polynomial.legendre.leggauss(60)
    xt, wt = np.polynomial.legendre.leggauss(16)
    nph = 16
    eps = 1e-7 * a
    t = 0.5 * (xr + 1) * (np.log(a) - np.log(eps)) + np.log(eps)  # log-radial
    r = np.exp(t)
    w_r = 0.5 * (np.log(a) - np.log(eps)) * wr * r  # dr = r dt
    ct = xt
    st = np.sqrt(1 - ct**2)
    ph = 2 * np.pi * np.arange(nph) / nph
    tot = np.zeros((3, 3), dtype=complex)
    for ri, wri in zip(r, w_r):
        for c, s, wti in zip(ct, st, wt):
            dirs = np.stack([s * np.cos(ph), s * np.sin(ph), np.full(nph, c)], axis=-1)
            G = physics.electric_dyadic(ri * dirs, f, s0)
            tot += wri * ri**2 * wti * (2 * np.pi / nph) * G.sum(axis=0)
    tot += -np.eye(3) / (3 * s0)
    exact = physics.self_cell(dv, f, s0) * np.eye(3)
    assert np.max(np.abs(tot - exact)) < 1e-8 * np.max(np.abs(exact))


def test_single_voxel_clausius_mossotti():
    # A lone cell at low frequency behaves like a small sphere in a uniform field:
    # E_in = 3 sigma0 (sigma + 2 sigma0 I)^{-1} E0 (textbook, holds for a tensor sigma too).
    s0 = 0.5
    sig = np.array([[2.0, 0.3, -0.1], [0.3, 0.7, 0.2], [-0.1, 0.2, 1.3]])
    s6 = np.array([[[[sig[0, 0], sig[1, 1], sig[2, 2], sig[0, 1], sig[0, 2], sig[1, 2]]]]])
    dsig = contrast(s6, s0)[0, 0, 0]
    S = physics.self_cell(1e-3, 1.0, s0)  # 1 Hz, 10 cm cell: k a ~ 1e-4
    E0 = np.array([1.0, -2.0, 0.5])
    E = np.linalg.solve(np.eye(3) - S * dsig, E0)
    E_cm = 3 * s0 * np.linalg.solve(sig + 2 * s0 * np.eye(3), E0)
    assert np.allclose(E, E_cm, rtol=1e-6)


def test_incident_H_coaxial_closed_form():
    # z-dipole, on-axis receiver at distance L: H_z = e^{ikL}(1 - ikL)/(2 pi L^3) (textbook)
    k = physics.k0(F, S0)
    for L in (0.5, 1.0, 7.0, 15.0):
        H = physics.incident_H(np.array([[0, 0, L]]), (0, 0, 0), (0, 0, 1), F, S0)[0]
        ref = np.exp(1j * k * L) * (1 - 1j * k * L) / (2 * np.pi * L**3)
        assert abs(H[2] - ref) < 1e-13 * abs(ref)
        assert abs(H[0]) < 1e-15 and abs(H[1]) < 1e-15


def test_incident_H_static_dipole_limit():
    R = np.array([0.3, 0.8, -0.5])
    m = np.array([0.2, -1.0, 0.7])
    r = np.linalg.norm(R)
    Rh = R / r
    H = physics.incident_H(R[None], (0, 0, 0), m, 1e-9, S0)[0]
    ref = (3 * Rh * (Rh @ m) - m) / (4 * np.pi * r**3)
    assert np.allclose(H, ref, rtol=1e-6)


def fd_curl(fun, p, step):
    J = np.zeros((3, 3), dtype=complex)  # J[i, j] = d f_i / d x_j
    for j in range(3):
        e = np.zeros(3)
        e[j] = step
        J[:, j] = (fun(p + e) - fun(p - e)) / (2 * step)
    return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]]), np.trace(J)


def test_incident_fields_satisfy_maxwell():
    src, m = np.array([0.1, -0.2, 0.3]), np.array([0.3, 0.5, -1.0])
    p = np.array([1.3, 0.4, -0.8])
    E = lambda r: physics.incident_E(r[None], src, m, F, S0)[0]
    Hf = lambda r: physics.incident_H(r[None], src, m, F, S0)[0]
    curlE, divE = fd_curl(E, p, 1e-5)
    iwm = 1j * physics.omega(F) * physics.MU0
    H = Hf(p)
    assert np.allclose(curlE, iwm * H, rtol=1e-6, atol=1e-8 * np.abs(iwm * H).max())
    assert abs(divE) < 1e-6 * np.abs(E(p)).max()
    curlH, divH = fd_curl(Hf, p, 1e-5)
    assert np.allclose(curlH, S0 * E(p), rtol=1e-5, atol=1e-6 * np.abs(S0 * E(p)).max())
    assert abs(divH) < 1e-6 * np.abs(H).max()


def test_scattered_H_is_curl_of_scattered_E():
    rng = np.random.default_rng(3)
    cells = rng.uniform(-1, 1, size=(7, 3))
    J = rng.normal(size=(7, 3)) + 1j * rng.normal(size=(7, 3))
    dv = 0.1
    p = np.array([2.5, -1.7, 1.9])

    def Es(r):
        G = physics.electric_dyadic(r[None] - cells, F, S0)
        return dv * np.einsum("jpq,jq->p", G, J)

    curlE, _ = fd_curl(Es, p, 1e-5)
    Hs = physics.scattered_H(p[None], cells, J, dv, F, S0)[0]
    iwm = 1j * physics.omega(F) * physics.MU0
    assert np.allclose(curlE, iwm * Hs, rtol=1e-6, atol=1e-7 * np.abs(iwm * Hs).max())
