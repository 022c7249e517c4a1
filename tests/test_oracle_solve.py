"""Pins for the oracle's solvers: GMRES, the forward model and Algorithm 1 (domain decomposition)."""
import numpy as np
import pytest

from oracle import gmres as gm
from oracle import operator as op
from oracle import physics, solve
from oracle.dd import dd_solve
from paper_2306_17537_gb300 import inputs

F, S0 = 1.0e5, 0.1


def small_model(shape=(4, 4, 4), seed=0, h=0.5, spread=0.6):
    g = inputs.Grid(shape[2], shape[1], shape[0], h, (-shape[2] * h / 2, -shape[1] * h / 2, -shape[0] * h / 2))
    s6 = inputs.random_contrast_sigma6(shape, seed, S0, spread)
    return g, s6


def test_gmres_exact_in_n_steps_and_estimate_is_true_residual():
    rng = np.random.default_rng(0)
    n = 12
    M = np.eye(n) + 0.3 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    x, info = gm.gmres(lambda v: M @ v, b, tol=1e-14, restart=n, max_iter=n)
    assert info.iterations <= n
    assert np.linalg.norm(M @ x - b) <= 1e-12 * np.linalg.norm(b)
    x2, info2 = gm.gmres(lambda v: M @ v, b, tol=1e-3, restart=n, max_iter=n)
    true = np.linalg.norm(b - M @ x2) / np.linalg.norm(b)
    assert abs(true - info2.history[-1]) <= 1e-10 and true <= 1e-3


def test_gmres_restarted_with_initial_guess_matches_solve():
    rng = np.random.default_rng(1)
    n = 40
    M = np.diag(np.linspace(1, 3, n)) + 0.05 * rng.normal(size=(n, n))
    b = rng.normal(size=n) + 0j
    x0 = rng.normal(size=n) + 0j
    x, info = gm.gmres(lambda v: M @ v, b, x0=x0, tol=1e-12, restart=5, max_iter=400)
    assert info.converged and np.allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-10)


def test_zero_contrast_recovers_incident_fields():
    g, _ = small_model()
    s6 = np.zeros((4, 4, 4, 6))
    s6[..., :3] = S0
    src = [inputs.Dipole((0.0, 0.0, 0.0), (0.0, 0.0, 1.0))]
    rx = np.array([[0.0, 0.0, 1.0], [0.5, 0.0, 1.5]])
    H, info, Es = solve.forward(g, s6, S0, F, src, rx, method="gmres", return_E=True)
    assert info.gmres_iters == 0
    E0 = solve.incident_field_on_grid(g, src[0], F, S0)
    assert np.array_equal(Es[0], E0)
    H0 = physics.incident_H(rx, src[0].pos, src[0].moment, F, S0)
    assert np.allclose(H[0], H0, rtol=1e-15, atol=0)


def test_lu_equals_gmres():
    g, s6 = small_model((3, 4, 4), seed=2)
    src = [inputs.Dipole((0.0, 0.0, 0.0), (1.0, 0.0, 0.0))]
    rx = np.array([[0.0, 0.0, 1.0], [0.0, 0.5, 2.0]])
    H_lu, _, E_lu = solve.forward(g, s6, S0, F, src, rx, method="lu", return_E=True)
    H_gm, info, E_gm = solve.forward(g, s6, S0, F, src, rx, method="gmres", tol=1e-12, return_E=True)
    assert np.linalg.norm(E_gm[0] - E_lu[0]) <= 1e-10 * np.linalg.norm(E_lu[0])
    assert np.allclose(H_gm, H_lu, rtol=1e-10, atol=1e-10 * np.abs(H_lu).max())


def test_born_limit():
    g, s6 = small_model((3, 3, 3), seed=4)
    dsig = op.contrast(s6, S0)
    src = inputs.Dipole((0.1, 0.2, 0.05), (0.0, 1.0, 0.0))  # odd grid: keep off the centre cell
    E0 = solve.incident_field_on_grid(g, src, F, S0)
    errs = []
    for eps in (1e-2, 5e-3):
        opx = op.FFTOperator(eps * dsig, g.h, F, S0)
        A = op.dense_matrix(eps * dsig, g.h, F, S0)
        E = np.linalg.solve(A, E0.ravel()).reshape(E0.shape)
        born = E0 + opx.G(op.apply_contrast(eps * dsig, E0))
        errs.append(np.linalg.norm(E - born))
    assert 3.6 < errs[0] / errs[1] < 4.4  # second order in the contrast


def test_reciprocity_of_scattered_field():
    # Discrete model: dsigma (I - K dsigma)^{-1} is symmetric, so H^s_p(r_r; m = e_q at r_s)
    # equals H^s_q(r_s; m = e_p at r_r).
    g, s6 = small_model((4, 3, 4), seed=6, spread=0.8)
    r_s = np.array([0.0, 0.0, -0.5])
    r_r = np.array([0.5, 0.0, 1.5])
    dsig = op.contrast(s6, S0)
    H_sr = np.zeros((3, 3), dtype=complex)  # [q (source comp), p (receiver comp)]
    H_rs = np.zeros((3, 3), dtype=complex)
    for q in range(3):
        m = np.eye(3)[q]
        Hq, _, Eq = solve.forward(g, s6, S0, F, [inputs.Dipole(tuple(r_s), tuple(m))], r_r[None],
                                  method="lu", return_E=True)
        H_sr[q] = Hq[0, 0] - physics.incident_H(r_r[None], r_s, m, F, S0)[0]
        Hp, _, _ = solve.forward(g, s6, S0, F, [inputs.Dipole(tuple(r_r), tuple(m))], r_s[None], method="lu",
                                 return_E=True)
        H_rs[q] = Hp[0, 0] - physics.incident_H(r_s[None], r_r, m, F, S0)[0]
    assert np.allclose(H_sr, H_rs.T, rtol=1e-9, atol=1e-9 * np.abs(H_sr).max())


def test_linearity_in_moment():
    g, s6 = small_model((3, 3, 3), seed=8)
    rx = np.array([[0.0, 0.0, 1.0]])
    mx, mz = (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)
    p = (0.1, 0.2, 0.05)  # odd grid: keep off the centre cell
    H, _ = solve.forward(g, s6, S0, F, [inputs.Dipole(p, mx), inputs.Dipole(p, mz),
                                        inputs.Dipole(p, (2.0, 0.0, -3.0))], rx, method="lu")
    assert np.allclose(H[2], 2 * H[0] - 3 * H[1], rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- Algorithm 1 (domain decomposition)

def _dd_case(shape=(6, 3, 3), seed=3):
    g, s6 = small_model(shape, seed=seed, spread=0.5)
    dsig = op.contrast(s6, S0)
    E0 = solve.incident_field_on_grid(g, inputs.Dipole((0.1, 0.0, 0.0), (0.0, 0.0, 1.0)), F, S0)
    return g, dsig, E0


def _block_matrix_iteration(A, E0, split, nzyx, mode, sweeps):
    """Reference block Jacobi / Gauss-Seidel built from the dense matrix and exact block solves."""
    nz, ny, nx = nzyx
    idx = np.arange(3 * nz * ny * nx).reshape(3, nz, ny, nx)
    blocks = [idx[:, a:b].ravel() for a, b in zip(split[:-1], split[1:])]
    b = E0.ravel()
    x = b.copy()
    for _ in range(sweeps):
        xk = x.copy()
        for i, bi in enumerate(blocks):
            src = x if mode == "gs" else xk
            rhs = b[bi] - sum(A[np.ix_(bi, bj)] @ src[bj] for j, bj in enumerate(blocks) if j != i)
            x[bi] = np.linalg.solve(A[np.ix_(bi, bi)], rhs)
    return x.reshape(E0.shape)


@pytest.mark.parametrize("mode", ["gs", "jacobi"])
def test_dd_sweeps_equal_block_matrix_iteration(mode):
    g, dsig, E0 = _dd_case()
    split = [0, 2, 4, 6]
    A = op.dense_matrix(dsig, g.h, F, S0)
    for sweeps in (1, 3):
        E, info = dd_solve(dsig, E0, split, g.h, F, S0, mode=mode, eps=0.0, adaptive=False,
                           fixed_tol=1e-14, restart=200, max_outer=sweeps, max_inner=400)
        ref = _block_matrix_iteration(A, E0, split, dsig.shape[:3], mode, sweeps)
        assert info.outer_iters == sweeps
        assert np.linalg.norm(E - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("mode", ["gs", "jacobi"])
def test_dd_converges_to_full_solution(mode):
    g, dsig, E0 = _dd_case((8, 3, 3), seed=5)
    A = op.dense_matrix(dsig, g.h, F, S0)
    E_lu = np.linalg.solve(A, E0.ravel()).reshape(E0.shape)
    E, info = dd_solve(dsig, E0, [0, 4, 8], g.h, F, S0, mode=mode, eps=1e-9, restart=10)
    assert info.converged and info.residuals[-1] <= 1e-9
    assert np.linalg.norm(E - E_lu) <= 1e-7 * np.linalg.norm(E_lu)
    r = np.linalg.norm(E0.ravel() - A @ E.ravel()) / np.linalg.norm(E0)
    assert abs(r - info.residuals[-1]) <= 1e-12


def test_dd_one_block_is_plain_gmres():
    g, dsig, E0 = _dd_case((4, 3, 3), seed=9)
    full = op.FFTOperator(dsig, g.h, F, S0)
    E_gm, gi = gm.gmres(full, E0, x0=E0, tol=1e-3, restart=10)
    e0 = np.linalg.norm(E0 - full(E0)) / np.linalg.norm(E0)
    # one sweep of Algorithm 1 with M = 1 is GMRES from x0 = E0 with tol e0/10
    E_dd, info = dd_solve(dsig, E0, [0, 4], g.h, F, S0, mode="gs", eps=0.0, max_outer=1, restart=10)
    E_ref, gi = gm.gmres(full, E0, x0=E0, tol=e0 / 10, restart=10)
    assert info.gmres_iters == [[gi.iterations]]
    assert np.allclose(E_dd, E_ref, rtol=0, atol=1e-14 * np.abs(E_ref).max())


def test_adaptive_tolerance_and_gs_vs_jacobi_qualitative():
    # Section 3.2: GS-A needs fewer GMRES iterations than GS-F, and GS needs fewer sweeps than Jacobi
    g, dsig, E0 = _dd_case((12, 4, 4), seed=12)
    split = [0, 4, 8, 12]
    _, gs_a = dd_solve(dsig, E0, split, g.h, F, S0, mode="gs", eps=1e-8, adaptive=True, restart=10)
    _, gs_f = dd_solve(dsig, E0, split, g.h, F, S0, mode="gs", eps=1e-8, adaptive=False,
                       fixed_tol=1e-8, restart=10)
    _, ja_a = dd_solve(dsig, E0, split, g.h, F, S0, mode="jacobi", eps=1e-8, adaptive=True, restart=10)
    assert gs_a.converged and gs_f.converged and ja_a.converged
    assert gs_a.gmres_total < gs_f.gmres_total
    assert gs_a.outer_iters <= ja_a.outer_iters


# ---------------------------------------------------------------- Krylov outer iteration over the DD sweep
def _small_dd_case():
    wl = inputs.config2(0, scale=16)  # 8 x 8 x 16 cells, two sub-domains
    from oracle import operator as oop_

    dsig = oop_.contrast(wl.sigma6, wl.sigma0)
    E0 = solve.incident_field_on_grid(wl.grid, inputs.Dipole((0.1, 0.0, 0.0), (0.0, 0.0, 1.0)), wl.freq, wl.sigma0)
    return wl, dsig, E0


def test_fgmres_dd_reaches_the_lu_solution():
    from oracle import dd as odd
    from oracle import operator as oop_

    wl, dsig, E0 = _small_dd_case()
    A = oop_.dense_matrix(dsig, wl.grid.h, wl.freq, wl.sigma0)
    E_lu = np.linalg.solve(A, E0.ravel()).reshape(E0.shape)
    for mode in ("gs", "jacobi"):
        E, info = odd.fgmres_dd(dsig, E0, wl.z_split, wl.grid.h, wl.freq, wl.sigma0, mode=mode, eps=1e-10,
                                restart=10, inner_tol=0.1)
        assert info.converged and info.residuals[-1] <= 1e-10
        assert np.linalg.norm(E - E_lu) <= 1e-8 * np.linalg.norm(E_lu)


def test_fgmres_dd_needs_fewer_sweeps_than_the_fixed_point_iteration():
    from oracle import dd as odd

    wl, dsig, E0 = _small_dd_case()
    _, fp = odd.dd_solve(dsig, E0, wl.z_split, wl.grid.h, wl.freq, wl.sigma0, mode="jacobi", eps=1e-8,
                         adaptive=False, fixed_tol=1e-10, restart=30, max_outer=200, max_inner=3000)
    _, kr = odd.fgmres_dd(dsig, E0, wl.z_split, wl.grid.h, wl.freq, wl.sigma0, mode="jacobi", eps=1e-8,
                          restart=30, inner_tol=1e-10, max_inner=3000)
    assert fp.converged and kr.converged
    assert kr.outer_iters < fp.outer_iters


def test_fgmres_with_one_block_and_exact_inner_solves_takes_one_step():
    # one sub-domain covering the grid: the preconditioner is the exact inverse
    from oracle import dd as odd

    wl, dsig, E0 = _small_dd_case()
    E, info = odd.fgmres_dd(dsig, E0, [0, wl.grid.nz], wl.grid.h, wl.freq, wl.sigma0, eps=1e-9, restart=5,
                            inner_tol=1e-13, max_inner=5000)
    assert info.converged and info.outer_iters == 1


def test_jacobi_preconditioner_sweep_is_the_block_diagonal_inverse():
    # a Jacobi sweep started from zero solves each sub-domain system with its own right-hand side only
    from oracle import dd as odd
    from oracle import operator as oop_

    wl, dsig, E0 = _small_dd_case()
    rng = np.random.default_rng(3)
    v = rng.normal(size=E0.shape) + 1j * rng.normal(size=E0.shape)
    full = oop_.FFTOperator(dsig, wl.grid.h, wl.freq, wl.sigma0)
    blocks = [(wl.z_split[i], wl.z_split[i + 1]) for i in range(len(wl.z_split) - 1)]
    A = [oop_.FFTOperator(dsig[z0:z1], wl.grid.h, wl.freq, wl.sigma0) for z0, z1 in blocks]
    z, _ = odd.dd_sweep_from_zero(dsig, v, blocks, A, full, "jacobi", 1e-13, 60, 5000)
    for z0, z1 in blocks:
        D = oop_.dense_matrix(dsig[z0:z1], wl.grid.h, wl.freq, wl.sigma0)
        zi = np.linalg.solve(D, v[:, z0:z1].ravel()).reshape(v[:, z0:z1].shape)
        assert np.linalg.norm(z[:, z0:z1] - zi) <= 1e-10 * np.linalg.norm(zi)
