"""Block Jacobi with the sub-domain solves in flight together (ie_opts.concurrent_blocks, eq. 23).

* The concurrent sweep performs the same arithmetic per block as the one-after-another sweep, so on the
  same context (tile shapes already tuned) the fields, sweep counts and GMRES counts must be identical.
* Against the oracle: the FP64 residual of eq. 9 of the returned field, and the receiver fields of the
  oracle's own block-Jacobi solution (Algorithm 1), on a small model the oracle solves in seconds.
* The 256x256x512 model's generator at a quarter of each size (8 sub-domains), solved as the benchmark
  solves it (flexible GMRES over concurrent block-Jacobi sweeps): identical to the sequential sweeps,
  FP64 residual and receivers checked by the oracle.
"""
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


def _solve(ie, ctx, wl, conc, contraction, split=None):
    opts = ie.make_opts(z_split=split or wl.z_split, restart=wl.restart, max_inner=4000, max_outer=60,
                        contraction=contraction, concurrent_blocks=conc)
    return ctx.solve(wl.sources, wl.receivers, ie.IE_DD_JACOBI, wl.tol, opts)


@pytest.mark.parametrize("contraction", [False, True])
def test_concurrent_equals_sequential_and_oracle(ie, contraction):
    wl = inputs.config2(0, scale=8)  # 16 x 16 x 32, four sub-domains below
    wl.sigma6 = inputs.random_contrast_sigma6((32, 16, 16), 5, wl.sigma0, 0.8)
    split = [0, 6, 16, 23, 32]  # uneven heights
    g = wl.grid
    with ie.Context(g, g.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        Hs, infs, sts = _solve(ie, ctx, wl, False, contraction, split)
        Es = ctx.get_field()
        Hc, infc, stc = _solve(ie, ctx, wl, True, contraction, split)
        Ec = ctx.get_field()
    assert sts == stc == ie.IE_OK
    assert infc.outer_iters == infs.outer_iters and infc.gmres_iters_total == infs.gmres_iters_total
    assert np.array_equal(Ec, Es) and np.array_equal(Hc, Hs)
    E0 = osolve.incident_field_on_grid(g, wl.sources[0], wl.freq, wl.sigma0)
    op = oop.FFTOperator(oop.contrast(wl.sigma6, wl.sigma0), g.h, wl.freq, wl.sigma0)
    assert np.linalg.norm(E0 - op(Ec)) / np.linalg.norm(E0) <= wl.tol
    Ho, oinfo = osolve.forward(g, wl.sigma6, wl.sigma0, wl.freq, wl.sources, wl.receivers, method="jacobi",
                               tol=1e-9, restart=30, z_split=split, max_inner=3000)
    assert np.max(np.abs(Hc - Ho)) <= 1e-5 * np.max(np.abs(Ho))


def test_large_model_generator_concurrent_jacobi(ie):
    # the 256x256x512 model's generator at a quarter of each size (64 x 64 x 128, eight sub-domains of 16
    # planes), solved as the benchmark solves it: flexible GMRES preconditioned by one block-Jacobi sweep
    wl = inputs.config5(0, 5, scale=4)
    g = wl.grid
    res = []
    with ie.Context(g, g.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        for conc in (False, True):
            opts = ie.make_opts(z_split=wl.z_split, restart=wl.restart, max_inner=4000, max_outer=60,
                                contraction=True, concurrent_blocks=conc, outer_krylov=True, outer_restart=20)
            H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_JACOBI, wl.tol, opts)
            res.append((H, info, st, ctx.get_field()))
    (Hs, infs, sts, Es), (Hc, infc, stc, Ec) = res
    assert sts == stc == ie.IE_OK and infc.final_rel_residual <= wl.tol
    assert np.array_equal(Hc, Hs) and infc.gmres_iters_total == infs.gmres_iters_total
    E0 = osolve.incident_field_on_grid(g, wl.sources[0], wl.freq, wl.sigma0)
    op = oop.FFTOperator(oop.contrast(wl.sigma6, wl.sigma0), g.h, wl.freq, wl.sigma0)
    e = float(np.linalg.norm(E0 - op(Ec)) / np.linalg.norm(E0))
    assert e <= wl.tol and abs(e - infc.final_rel_residual) <= 1e-3 * e
    dsig = oop.contrast(wl.sigma6, wl.sigma0)
    ref = osolve.receiver_fields(g, dsig, Ec, wl.sources[0], wl.receivers, wl.freq, wl.sigma0)
    assert np.max(np.abs(Hc[0] - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_concurrent_graph_sweep_equals_sequential(ie):
    # the device-driven variant (ie_opts.graph): every block's GMRES graph launched before the first wait
    wl = inputs.config2(0, scale=8)
    wl.sigma6 = inputs.random_contrast_sigma6((32, 16, 16), 9, wl.sigma0, 0.8)
    split = [0, 9, 21, 32]
    g = wl.grid
    with ie.Context(g, g.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        res = []
        for conc in (False, True):
            opts = ie.make_opts(z_split=split, restart=wl.restart, max_inner=4000, max_outer=60, contraction=True,
                                concurrent_blocks=conc, graph=True)
            H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_JACOBI, wl.tol, opts)
            res.append((H, info, st, ctx.get_field()))
    (Hs, infs, sts, Es), (Hc, infc, stc, Ec) = res
    assert sts == stc == ie.IE_OK and infc.final_rel_residual <= wl.tol
    assert infc.gmres_iters_total == infs.gmres_iters_total and np.array_equal(Ec, Es)
    E0 = osolve.incident_field_on_grid(g, wl.sources[0], wl.freq, wl.sigma0)
    op = oop.FFTOperator(oop.contrast(wl.sigma6, wl.sigma0), g.h, wl.freq, wl.sigma0)
    assert np.linalg.norm(E0 - op(Ec)) / np.linalg.norm(E0) <= wl.tol
