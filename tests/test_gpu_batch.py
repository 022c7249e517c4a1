"""Batched forward solves (ie_solve_batch): several tool positions and two frequencies of the logging
workload, solved concurrently, against the same problems solved one at a time with ie_solve, and the
FFT-tile autotuner's variants against each other."""
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


def test_batch_equals_one_at_a_time(ie):
    # 3 positions x 2 frequencies on windows shrunk by 4 (16x16x40 and 32x32x80), block Jacobi
    probs = [inputs.config3_item(11, p, f, n_positions=3, scale=4) for f in (2.0e6, 1.0e5) for p in range(3)]
    ctxs = {f: [ie.Context(w.grid, w.grid.h, w.sigma0, w.freq) for w in probs if w.freq == f][:2] for f in (2.0e6, 1.0e5)}
    opts = {id(w): ie.make_opts(z_split=w.z_split, restart=w.restart, max_inner=4000, max_outer=60) for w in probs}
    batch = []
    for k, w in enumerate(probs):
        ctx = ctxs[w.freq][k % 2]  # two contexts per frequency, items sharing a context run in order
        batch.append(dict(ctx=ctx, sigma6=w.sigma6, sources=w.sources, receivers=w.receivers,
                          dd_mode=ie.IE_DD_JACOBI, tol=w.tol, opts=opts[id(w)]))
    res = ie.solve_batch(batch)
    for w, (H, info, st) in zip(probs, res):
        assert st == ie.IE_OK and info.final_rel_residual <= w.tol
        with ie.Context(w.grid, w.grid.h, w.sigma0, w.freq) as one:
            one.set_contrast(w.sigma6)
            H1, info1, _ = one.solve(w.sources, w.receivers, ie.IE_DD_JACOBI, w.tol, opts[id(w)])
        assert np.array_equal(H, H1) and info.gmres_iters_total == info1.gmres_iters_total
    for cs in ctxs.values():
        for c in cs:
            c.close()


def test_batch_result_checked_by_oracle(ie):
    w = inputs.config3_item(3, 1, 2.0e6, n_positions=3, scale=4)
    with ie.Context(w.grid, w.grid.h, w.sigma0, w.freq) as ctx:
        [(H, info, st)] = ie.solve_batch([dict(ctx=ctx, sigma6=w.sigma6, sources=w.sources, receivers=w.receivers,
                                               dd_mode=ie.IE_DD_JACOBI, tol=w.tol,
                                               opts=ie.make_opts(z_split=w.z_split, restart=40, max_inner=4000,
                                                                 max_outer=60))])
        E = ctx.get_field()
    assert st == ie.IE_OK
    E0 = osolve.incident_field_on_grid(w.grid, w.sources[0], w.freq, w.sigma0)
    op = oop.FFTOperator(oop.contrast(w.sigma6, w.sigma0), w.grid.h, w.freq, w.sigma0)
    assert np.linalg.norm(E0 - op(E)) / np.linalg.norm(E0) <= w.tol
    ref = osolve.receiver_fields(w.grid, oop.contrast(w.sigma6, w.sigma0), E, w.sources[0], w.receivers, w.freq,
                                 w.sigma0)
    assert np.max(np.abs(H[0] - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_batch_item_initial_guess():
    # an item carrying its converged field as the initial guess needs no iterations; one without is cold
    import torch

    from paper_2306_17537_gb300 import ie

    wl = inputs.config4_item(0, 32)
    n3 = wl.grid.n
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as c1, ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as c2:
        o = ie.make_opts(restart=40, max_inner=4000, max_outer=4)
        c1.set_contrast(wl.sigma6)
        _, i0, _ = c1.solve(wl.sources, [], ie.IE_DD_NONE, 1e-6, o)
        E = torch.empty((3, n3), dtype=torch.complex128, device=torch.device("cuda", 0))
        c1.get_field_dev(E)
        torch.cuda.synchronize()
        res = ie.solve_batch([dict(ctx=c1, sigma6=wl.sigma6, sources=wl.sources, receivers=[], tol=1e-6, opts=o, E_init_dev=E),
                              dict(ctx=c2, sigma6=wl.sigma6, sources=wl.sources, receivers=[], tol=1e-6, opts=o)])
    (_, warm, sw), (_, cold, sc) = res
    assert sw == sc == ie.IE_OK
    assert warm.warm_start_used == 1 and warm.gmres_iters_total == 0
    assert cold.warm_start_used == 0 and cold.gmres_iters_total == i0.gmres_iters_total
