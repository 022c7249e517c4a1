"""The logging simulation of Section 3.3 at the paper's tool and stopping rule: z-directed dipole at
24 kHz, receivers 7/15/30 m, block Gauss-Seidel with adaptive tolerance to e = 1e-3, GMRES(10), windows
of 128x128x256 cells (two sub-domains) and 256^3 cells (eight). The paper reports fewer than seven
Gauss-Seidel iterations at every position of its own model (known only from a figure); on the
stand-in formation the count is checked to stay of that order (at most 12). The receiver fields at
e = 1e-3 are compared with a reference to 1e-4 from the flexible-GMRES outer iteration."""
import numpy as np
import pytest

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
        # reference to 1e-4 with the Krylov outer iteration: on these 24 kHz windows the fixed-point
        # sweeps stop converging near e ~ 1e-4 (the Gauss-Seidel iteration matrix is not contracting
        # there), the flexible GMRES over the same sweep keeps converging
        ref = ie.make_opts(z_split=wl.z_split, restart=40, max_inner=4000, max_outer=40, contraction=True,
                           outer_krylov=True, outer_restart=20)
        Ht, infot, stt = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, 1e-4, ref)
    assert stt == ie.IE_OK and infot.final_rel_residual <= 1e-4
    Hzz, Hzz_t = H[0, :, 2], Ht[0, :, 2]
    assert np.all(np.abs(Hzz - Hzz_t) <= 2e-2 * np.abs(Hzz_t))
