"""The logging simulation of Section 3.3 at the paper's tool and stopping rule: z-directed dipole at
24 kHz, receivers 7/15/30 m, block Gauss-Seidel with adaptive tolerance to e = 1e-3, GMRES(10), windows
of 128x128x256 cells (two sub-domains) and 256^3 cells (eight). The paper reports fewer than seven
Gauss-Seidel iterations at every position of its own model (known only from a figure). On the
stand-in formation the oracle's own Algorithm 1 needs 9 sweeps at window 1, position 20 with every
window dimension divided by 4, so the count is checked to stay of that order (at most 12), and at the
reduced size the GPU's sweep count and receiver fields are compared with the oracle's run of the same
algorithm. At full size the returned field's FP64 residual (eq. 9) and receiver fields are recomputed by
the oracle, and the fields are compared with a reference to 1e-4 from the flexible-GMRES outer
iteration."""
import numpy as np
import pytest

from oracle import dd as odd
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


@pytest.mark.parametrize("window,position", [(1, 20), (1, 45), (2, 32)])
def test_logging_position_converges_in_a_few_sweeps(ie, window, position):
    wl = inputs.paper_logging_item(position, 64, window)
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        opts = ie.make_opts(z_split=wl.z_split, restart=wl.restart, max_inner=4000, max_outer=40)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, wl.tol, opts)
        assert st == ie.IE_OK and info.final_rel_residual <= 1e-3 and info.outer_iters <= 12
        if window == 2:
            return
        E = ctx.get_field()
        g = wl.grid
        dsig = oop.contrast(wl.sigma6, wl.sigma0)
        E0 = osolve.incident_field_on_grid(g, wl.sources[0], wl.freq, wl.sigma0)
        e = float(np.linalg.norm(E0 - oop.FFTOperator(dsig, g.h, wl.freq, wl.sigma0)(E)) / np.linalg.norm(E0))
        assert e <= 1e-3 and abs(e - info.final_rel_residual) <= 1e-3 * e
        Hr = osolve.receiver_fields(g, dsig, E, wl.sources[0], wl.receivers, wl.freq, wl.sigma0)
        assert np.max(np.abs(H[0] - Hr)) <= 1e-10 * np.max(np.abs(Hr))
        # reference to 1e-4 with the Krylov outer iteration: on these 24 kHz windows the fixed-point
        # sweeps stop converging near e ~ 1e-4 (the Gauss-Seidel iteration matrix is not contracting
        # there), the flexible GMRES over the same sweep keeps converging
        ref = ie.make_opts(z_split=wl.z_split, restart=40, max_inner=4000, max_outer=40, contraction=True,
                           outer_krylov=True, outer_restart=20)
        Ht, infot, stt = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, 1e-4, ref)
    assert stt == ie.IE_OK and infot.final_rel_residual <= 1e-4
    Hzz, Hzz_t = H[0, :, 2], Ht[0, :, 2]
    assert np.all(np.abs(Hzz - Hzz_t) <= 2e-2 * np.abs(Hzz_t))


@pytest.mark.parametrize("position", [20, 45])
def test_logging_reduced_window_matches_oracle_algorithm(ie, position):
    # window 1 with every dimension divided by 4 (32 x 32 x 64 cells, two sub-domains): the GPU's GS-A
    # sweeps against the oracle's Algorithm 1 on the same input (conventional operator, GMRES(10))
    wl = inputs.paper_logging_item(position, 64, 1, scale=4)
    g = wl.grid
    dsig = oop.contrast(wl.sigma6, wl.sigma0)
    E0 = osolve.incident_field_on_grid(g, wl.sources[0], wl.freq, wl.sigma0)
    Eo, oinfo = odd.dd_solve(dsig, E0, wl.z_split, g.h, wl.freq, wl.sigma0, mode="gs", eps=wl.tol, adaptive=True,
                             restart=wl.restart, max_outer=40, max_inner=4000)
    assert oinfo.converged
    Ho = osolve.receiver_fields(g, dsig, Eo, wl.sources[0], wl.receivers, wl.freq, wl.sigma0)
    with ie.Context(g, g.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        opts = ie.make_opts(z_split=wl.z_split, restart=wl.restart, max_inner=4000, max_outer=40)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, wl.tol, opts)
    assert st == ie.IE_OK and abs(info.outer_iters - oinfo.outer_iters) <= 1
    # both stop at e <= 1e-3 after the same sweeps: the fields agree far better than the tolerance
    assert np.max(np.abs(H[0] - Ho)) <= 1e-3 * np.max(np.abs(Ho))
