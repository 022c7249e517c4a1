"""Sub-domains without contrast are left out of the DD sweeps (the isolated sub-domains example of
Section 3.1): e is measured over the anomalous sub-domains, only those are solved, and the field of the
others is filled in as E0 + G dsigma E. Checked on the 64^3 version of that model against the
whole-domain solve and against the oracle's residual and scattered field."""
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


@pytest.mark.parametrize("mode,contraction", [("gs", False), ("jacobi", False), ("gs", True)])
def test_masked_dd_matches_whole_domain_solve(ie, mode, contraction):
    wl = inputs.isolated_blocks(64)
    dd = ie.IE_DD_GAUSS_SEIDEL if mode == "gs" else ie.IE_DD_JACOBI
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        # Section 3.1 runs the sub-domain GMRES at the fixed tolerance 1e-6 with restart 10
        opts = ie.make_opts(z_split=wl.z_split, restart=wl.restart, max_inner=4000, max_outer=40, adaptive=False,
                            fixed_tol=1e-6, contraction=contraction)
        H, info, st = ctx.solve(wl.sources, wl.receivers, dd, wl.tol, opts)
        E = ctx.get_field()
        full = ie.make_opts(restart=30, max_inner=4000, max_outer=20, contraction=contraction)
        Hf, infof, stf = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, wl.tol, full)
    assert st == stf == ie.IE_OK
    assert info.active_blocks == 2 and info.final_rel_residual <= wl.tol
    assert np.max(np.abs(H - Hf)) <= 1e-5 * np.max(np.abs(Hf))
    # oracle: the residual over the anomalous slabs, and the filled-in field of the others
    E0 = osolve.incident_field_on_grid(wl.grid, wl.sources[0], wl.freq, wl.sigma0)
    dsig = oop.contrast(wl.sigma6, wl.sigma0)
    op = oop.FFTOperator(dsig, wl.grid.h, wl.freq, wl.sigma0)
    R = E0 - op(E)
    zs = wl.z_split
    anom = np.zeros(wl.grid.nz, bool)
    anom[zs[1]:zs[2]] = anom[zs[3]:zs[4]] = True
    e = np.linalg.norm(R[:, anom]) / np.linalg.norm(E0[:, anom])
    assert e <= 1.01 * wl.tol
    Es = E0 + op.G(oop.apply_contrast(dsig, E))
    assert np.linalg.norm(E[:, ~anom] - Es[:, ~anom]) <= 1e-9 * np.linalg.norm(Es[:, ~anom])


def test_no_contrast_anywhere_returns_the_incident_field(ie):
    wl = inputs.isolated_blocks(32)
    s6 = np.zeros_like(wl.sigma6)
    s6[..., :3] = wl.sigma0
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(s6)
        opts = ie.make_opts(z_split=wl.z_split, restart=10)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, 1e-6, opts)
        E = ctx.get_field()
        E0 = ctx.incident_field(wl.sources[0])
    assert st == ie.IE_OK and info.active_blocks == 0 and info.gmres_iters_total == 0
    assert np.array_equal(E, E0)


def test_isolated_sub_domains_example_reproduces_the_papers_counts(ie):
    # Section 3.1 prints the outcome of this fully specified example: the IE-DD Gauss-Seidel iteration
    # (GMRES(10), block tolerance fixed at 1e-6, background sub-domains excluded) converges in four
    # sweeps with 278 GMRES iterations in total, and the full-domain IE takes 86 iterations. The sweep
    # count is reproduced exactly; the iteration totals depend on discretisation details the paper does
    # not give (self term, source placement), so they are checked to the same order.
    wl = inputs.isolated_blocks(128)
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        opts = ie.make_opts(z_split=wl.z_split, restart=10, max_inner=4000, max_outer=40, adaptive=False,
                            fixed_tol=1e-6)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, 1e-6, opts)
        full = ie.make_opts(restart=10, max_inner=4000, max_outer=20)
        Hf, infof, stf = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, 1e-6, full)
    assert st == stf == ie.IE_OK
    assert info.outer_iters == 4
    assert 0.5 * 278 <= info.gmres_iters_total <= 1.5 * 278
    assert infof.gmres_iters_total <= 2 * 86
    # "less than 0.01 per cent average normalized magnitude difference" between the two
    assert np.mean(np.abs(np.abs(H) - np.abs(Hf)) / np.max(np.abs(Hf))) <= 1e-4
