"""Pins for the contraction form of the IE (oracle/contraction.py).

* The reflection tensor r = (sigma - sigma0)(sigma + sigma0)^-1 has the eigenvalues (s - sigma0)/(s + sigma0)
  of the conductivity's eigenvalues s, on the same eigenvectors (closed form via eigh).
* The contraction system (M - G dsigma M) u = E0 with E = M u gives the same field as the conventional
  system (dense LU both), whatever the contrast.
* The spectral radius of I - A_c stays below 1 at contrasts where the conventional I - A has radius >> 1
  (the contraction property that motivates the form).
* The FFT operator equals the dense matrix; GMRES needs fewer iterations on a high-contrast model.
"""
import numpy as np

from oracle import contraction as oc
from oracle import operator as oop
from oracle import solve as osolve
from oracle.gmres import gmres
from paper_2306_17537_gb300 import inputs


def test_reflection_tensor_eigenvalues():
    s6 = inputs.random_contrast_sigma6((3, 4, 5), 7, 0.1, spread=2.0)
    r = oc.reflection_tensor(s6, 0.1).reshape(-1, 3, 3)
    S = oc.sigma_tensor(s6).reshape(-1, 3, 3)
    w, V = np.linalg.eigh(S)
    expect = np.einsum("npk,nk,nqk->npq", V, (w - 0.1) / (w + 0.1), V)
    assert np.allclose(r, expect, atol=1e-13)
    assert np.all(np.abs((w - 0.1) / (w + 0.1)) < 1)


def test_contraction_solution_equals_conventional_solution():
    n, h, f, s0 = 5, 0.5, 1e5, 0.1
    s6 = inputs.random_contrast_sigma6((n, n, n), 3, s0, spread=3.0)
    g = inputs.centred_grid(n, n, n, h)
    E0 = osolve.incident_field_on_grid(g, inputs.Dipole((0.1, 0.0, 0.0), (0.0, 0.0, 1.0)), f, s0).ravel()
    A = oop.dense_matrix(oop.contrast(s6, s0), h, f, s0)
    Ac = oc.dense_contraction_matrix(s6, h, f, s0)
    E = np.linalg.solve(A, E0)
    u = np.linalg.solve(Ac, E0)
    Ec = oc.apply_contrast(oc.scaling_tensor(s6, s0), u.reshape(3, n, n, n)).ravel()
    assert np.linalg.norm(Ec - E) <= 1e-10 * np.linalg.norm(E)


def test_spectral_radius_below_one_at_high_contrast():
    n, h, f, s0 = 5, 0.5, 1e5, 0.1
    s6 = inputs.random_contrast_sigma6((n, n, n), 1, s0, spread=3.0)
    N = 3 * n ** 3
    rho_conv = np.max(np.abs(np.linalg.eigvals(np.eye(N) - oop.dense_matrix(oop.contrast(s6, s0), h, f, s0))))
    rho_c = np.max(np.abs(np.linalg.eigvals(np.eye(N) - oc.dense_contraction_matrix(s6, h, f, s0))))
    assert rho_conv > 5.0
    assert rho_c < 1.0


def test_fft_operator_matches_dense_matrix():
    s6 = inputs.random_contrast_sigma6((3, 4, 5), 2, 0.1, spread=1.0)
    rng = np.random.default_rng(0)
    u = rng.normal(size=(3, 3, 4, 5)) + 1j * rng.normal(size=(3, 3, 4, 5))
    op = oc.ContractionOperator(s6, 0.5, 4e5, 0.1)
    dense = oc.dense_contraction_matrix(s6, 0.5, 4e5, 0.1)
    assert np.allclose(op(u).ravel(), dense @ u.ravel(), rtol=0, atol=1e-12 * np.abs(dense @ u.ravel()).max())


def test_gmres_needs_fewer_iterations_at_high_contrast():
    n, h, f, s0 = 8, 0.5, 1e5, 0.1
    s6 = inputs.random_contrast_sigma6((n, n, n), 4, s0, spread=3.0)
    g = inputs.centred_grid(n, n, n, h)
    E0 = osolve.incident_field_on_grid(g, inputs.Dipole((0.0, 0.0, 0.0), (0.0, 0.0, 1.0)), f, s0)
    A = oop.FFTOperator(oop.contrast(s6, s0), h, f, s0)
    Ac = oc.ContractionOperator(s6, h, f, s0)
    _, gi = gmres(A, E0, x0=E0, tol=1e-8, restart=30, max_iter=5000)
    u, gc = gmres(Ac, E0, tol=1e-8, restart=30, max_iter=5000)
    E = Ac.field(u)
    assert np.linalg.norm(E0 - A(E)) <= 1.01e-8 * np.linalg.norm(E0)
    assert gc.iterations < gi.iterations
