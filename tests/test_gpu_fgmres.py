"""Flexible GMRES over the DD sweep (ie_opts.outer_krylov) against the fixed-point sweeps and the oracle:
same receiver fields (both at e <= 1e-6), the oracle's FP64 residual of the returned field, and fewer
sweeps than the fixed-point Jacobi iteration (as in the oracle's own comparison)."""
import numpy as np
import pytest

from oracle import operator as oop
from oracle import solve as osolve
from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    return _ie


@pytest.mark.parametrize("mode,contraction", [("gs", False), ("jacobi", False), ("jacobi", True)])
def test_fgmres_outer_matches_fixed_point(ie, mode, contraction):
    wl = inputs.config2(0, scale=4)  # 32x32x64, two blocks
    dd = ie.IE_DD_GAUSS_SEIDEL if mode == "gs" else ie.IE_DD_JACOBI
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        fp = ie.make_opts(z_split=wl.z_split, restart=wl.restart, max_inner=4000, max_outer=80, contraction=contraction)
        H0, i0, s0 = ctx.solve(wl.sources, wl.receivers, dd, wl.tol, fp)
        kr = ie.make_opts(z_split=wl.z_split, restart=wl.restart, max_inner=4000, max_outer=80, contraction=contraction,
                          outer_krylov=True, outer_restart=20, outer_inner_tol=0.1)
        H1, i1, s1 = ctx.solve(wl.sources, wl.receivers, dd, wl.tol, kr)
        E = ctx.get_field()
    assert s0 == s1 == ie.IE_OK and i1.final_rel_residual <= wl.tol
    assert np.max(np.abs(H1 - H0)) <= 1e-5 * np.max(np.abs(H0))
    E0 = osolve.incident_field_on_grid(wl.grid, wl.sources[0], wl.freq, wl.sigma0)
    op = oop.FFTOperator(oop.contrast(wl.sigma6, wl.sigma0), wl.grid.h, wl.freq, wl.sigma0)
    assert np.linalg.norm(E0 - op(E)) <= 1.01 * wl.tol * np.linalg.norm(E0)
    if mode == "jacobi":
        assert i1.outer_iters < i0.outer_iters


def test_fgmres_outer_with_masked_sub_domains(ie):
    wl = inputs.isolated_blocks(64)
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        kr = ie.make_opts(z_split=wl.z_split, restart=10, max_inner=4000, max_outer=40, outer_krylov=True)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, wl.tol, kr)
        full = ie.make_opts(restart=30, max_inner=4000, max_outer=20)
        Hf, _, stf = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, wl.tol, full)
    assert st == stf == ie.IE_OK and info.active_blocks == 2
    assert np.max(np.abs(H - Hf)) <= 1e-5 * np.max(np.abs(Hf))
