"""GPU forward solves (GMRES, block Gauss-Seidel, block Jacobi; FP64 and mixed precision) against the
CPU FP64 oracle, through the C ABI.

Parity bar: the returned field E must satisfy the oracle's own FP64 residual check
||E0 - (I - G dsigma) E|| / ||E0|| <= tol (eq. 9), and the receiver fields must match the oracle's
exact (dense LU) solution within cond * tol, where cond is bounded on these small models by the LU
solution itself: we use |H - H_lu| <= 50 * tol * |H_lu| (measured ratios stay below ~5).
"""
import numpy as np
import pytest

from oracle import operator as oop
from oracle import solve as osolve
from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu

F, S0 = 1.0e5, 0.1


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    return _ie


def oracle_residual(g, s6, E, src, freq=F, sigma0=S0):
    E0 = osolve.incident_field_on_grid(g, src, freq, sigma0)
    op = oop.FFTOperator(oop.contrast(s6, sigma0), g.h, freq, sigma0)
    return float(np.linalg.norm(E0 - op(E)) / np.linalg.norm(E0))


MODES = [("none-fp64", 0, 1, 1), ("none-mixed", 0, 1, 0), ("gs-mixed", 2, 2, 0), ("gs-fp64", 2, 3, 1),
         ("jacobi-mixed", 1, 2, 0), ("jacobi-fp64", 1, 3, 1)]


@pytest.mark.parametrize("name,mode,nblk,prec", MODES)
def test_small_solve_matches_lu(ie, name, mode, nblk, prec):
    g = inputs.centred_grid(6, 5, 9, 0.5)
    s6 = inputs.random_contrast_sigma6((g.nz, g.ny, g.nx), 21, S0, 0.7)
    src = [inputs.Dipole((0.0, 0.0, 0.0), (0.0, 0.0, 1.0)), inputs.Dipole((0.0, 0.0, 0.0), (1.0, 0.0, 0.0))]
    rx = np.array([[0.0, 0.0, 0.5], [0.0, 0.0, 1.0], [0.0, 0.0, 2.0], [0.5, 0.25, -1.0]])
    tol = 1e-9
    H_lu, _ = osolve.forward(g, s6, S0, F, src, rx, method="lu")
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        opts = ie.make_opts(n_blocks=nblk, precision=ie.IE_PREC_FP64 if prec else ie.IE_PREC_MIXED)
        H, info, st = ctx.solve(src, rx, mode, tol, opts)
        E_last = ctx.get_field()
    assert st == ie.IE_OK and info.final_rel_residual <= tol
    assert oracle_residual(g, s6, E_last, src[-1]) <= 1.001 * tol
    assert np.max(np.abs(H - H_lu)) <= 50 * tol * np.max(np.abs(H_lu))


def test_zero_contrast_returns_incident_fields(ie):
    g = inputs.centred_grid(8, 8, 8, 0.5)
    s6 = np.zeros((8, 8, 8, 6))
    s6[..., :3] = S0
    src, rx = inputs.coaxial_tool()
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        H, info, st = ctx.solve(src, rx, ie.IE_DD_GAUSS_SEIDEL, 1e-6, ie.make_opts(n_blocks=2))
    H0 = np.array([oop.physics.incident_H(rx, s.pos, s.moment, F, S0) for s in src])
    assert st == ie.IE_OK and info.gmres_iters_total == 0 and info.outer_iters == 0
    assert np.max(np.abs(H - H0)) <= 1e-14 * np.max(np.abs(H0))


def test_dd_matches_full_domain_solution(ie):
    # Section 3.1: the DD solution equals the full-domain solution within the tolerance
    g = inputs.centred_grid(8, 8, 16, 0.5)
    s6 = inputs.layered_vti(g, 3, ratio_max=3.0)
    src, rx = inputs.coaxial_tool()
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        Hf, inf_f, _ = ctx.solve(src, rx, ie.IE_DD_NONE, 1e-9, ie.make_opts(precision=ie.IE_PREC_FP64,
                                                                              max_inner=5000))
        Hgs, inf_g, _ = ctx.solve(src, rx, ie.IE_DD_GAUSS_SEIDEL, 1e-9, ie.make_opts(n_blocks=4))
        Hja, inf_j, _ = ctx.solve(src, rx, ie.IE_DD_JACOBI, 1e-9, ie.make_opts(n_blocks=4))
    scale = np.max(np.abs(Hf))
    assert np.max(np.abs(Hgs - Hf)) <= 1e-6 * scale and np.max(np.abs(Hja - Hf)) <= 1e-6 * scale
    assert inf_g.outer_iters <= inf_j.outer_iters  # Section 3.2: GS converges in fewer sweeps


def test_uneven_blocks_and_fixed_tolerance(ie):
    g = inputs.centred_grid(6, 6, 14, 0.5)
    s6 = inputs.random_contrast_sigma6((14, 6, 6), 31, S0, 0.6)
    src, rx = inputs.coaxial_tool()
    H_lu, _ = osolve.forward(g, s6, S0, F, src, rx, method="lu")
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        opts = ie.make_opts(z_split=[0, 3, 10, 14], adaptive=False, fixed_tol=1e-9)
        H, info, st = ctx.solve(src, rx, ie.IE_DD_GAUSS_SEIDEL, 1e-8, opts)
    assert st == ie.IE_OK and info.final_rel_residual <= 1e-8
    assert np.max(np.abs(H - H_lu)) <= 50 * 1e-8 * np.max(np.abs(H_lu))


def test_invalid_inputs_are_rejected(ie):
    g = inputs.centred_grid(4, 4, 4, 0.5)
    with ie.Context(g, g.h, S0, F) as ctx:
        src, rx = inputs.coaxial_tool()
        with pytest.raises(ie.IEError) as e:
            ctx.solve(src, rx)
        assert e.value.status == ie.IE_ESTATE
        bad = np.zeros((4, 4, 4, 6))
        bad[..., :3] = S0
        bad[1, 2, 3, 0] = np.nan
        with pytest.raises(ie.IEError) as e:
            ctx.set_contrast(bad)
        assert e.value.status == ie.IE_EINVAL
        bad[1, 2, 3, 0] = -1.0
        with pytest.raises(ie.IEError):
            ctx.set_contrast(bad)
        good = np.zeros((4, 4, 4, 6))
        good[..., :3] = 0.3
        ctx.set_contrast(good)
        with pytest.raises(ie.IEError) as e:  # receiver on a cell centre
            ctx.solve(src, np.array([[0.25, 0.25, 0.25]]))
        assert e.value.status == ie.IE_EINVAL
        with pytest.raises(ie.IEError):  # z_split not covering the grid
            ctx.solve(src, rx, ie.IE_DD_GAUSS_SEIDEL, 1e-6, ie.make_opts(z_split=[0, 2, 3]))


def test_iteration_limit_reports_noconv(ie):
    g = inputs.centred_grid(8, 8, 8, 0.5)
    s6 = inputs.random_contrast_sigma6((8, 8, 8), 41, S0, 1.0)
    src, rx = inputs.coaxial_tool()
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        H, info, st = ctx.solve(src, rx, ie.IE_DD_GAUSS_SEIDEL, 1e-12, ie.make_opts(n_blocks=2, max_outer=1),
                                allow_noconv=True)
    assert st == ie.IE_ENOCONV and info.outer_iters == 1 and np.all(np.isfinite(H))
