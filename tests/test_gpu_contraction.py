"""The contraction form of the IE on the GPU (ie_matvec_contraction, ie_opts.contraction) against the
oracle (oracle/contraction.py) and against the conventional solve.

Tolerances: complex128 operator 1e-11 and complex64 operator 1e-5 relative L2 (as for the conventional
operator: the same FFT convolution plus a per-voxel 3x3 scaling). Solves: the FP64 residual of eq. 9
must reach the requested tolerance, and the receiver fields must agree with the conventional solve and
with the oracle's LU solution as the conventional tests require.
"""
import json
import os

import numpy as np
import pytest

from oracle import contraction as oc
from oracle import operator as oop
from oracle import solve as osolve
from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu
F, S0 = 1.0e5, 0.1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c1_lu_receivers.json")


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    return _ie


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("shape,spread", [((1, 1, 1), 1.0), ((3, 5, 7), 0.5), ((8, 6, 10), 3.0), ((16, 16, 16), 2.0),
                                          ((33, 4, 6), 1.0)])
def test_contraction_operator_matches_oracle(ie, shape, spread):
    nz, ny, nx = shape
    h = 0.5
    g = inputs.Grid(nx, ny, nz, h, (-nx * h / 2 + 0.1, -ny * h / 2 - 0.05, -nz * h / 2 + 0.02))
    s6 = inputs.random_contrast_sigma6(shape, 11, S0, spread)
    x = inputs.random_field((3,) + shape, 12)
    ref = oc.ContractionOperator(s6, h, F, S0)(x)
    with ie.Context(g, h, S0, F) as ctx:
        ctx.set_contrast(s6)
        assert rel(ctx.matvec_contraction(x, precision=ie.IE_PREC_FP64), ref) <= 1e-11
        assert rel(ctx.matvec_contraction(x, precision=ie.IE_PREC_MIXED), ref) <= 1e-5


@pytest.mark.parametrize("z0,nz", [(0, 5), (5, 7), (11, 1)])
def test_contraction_operator_on_slab(ie, z0, nz):
    shape = (12, 6, 7)
    h = 0.5
    g = inputs.Grid(7, 6, 12, h, (-1.65, -1.55, -2.9))
    s6 = inputs.random_contrast_sigma6(shape, 13, S0, 2.0)
    x = inputs.random_field((3, nz) + shape[1:], 14)
    ref = oc.ContractionOperator(s6[z0:z0 + nz], h, F, S0)(x)
    with ie.Context(g, h, S0, F) as ctx:
        ctx.set_contrast(s6)
        assert rel(ctx.matvec_contraction(x, z0=z0, nz=nz, precision=ie.IE_PREC_FP64), ref) <= 1e-11
        assert rel(ctx.matvec_contraction(x, z0=z0, nz=nz, precision=ie.IE_PREC_MIXED), ref) <= 1e-5
        # a new contrast rebuilds the contraction tensors
        s6b = inputs.random_contrast_sigma6(shape, 15, S0, 0.5)
        ctx.set_contrast(s6b)
        refb = oc.ContractionOperator(s6b[z0:z0 + nz], h, F, S0)(x)
        assert rel(ctx.matvec_contraction(x, z0=z0, nz=nz, precision=ie.IE_PREC_FP64), refb) <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c1_contraction_matches_lu_golden_in_fewer_iterations(ie, precision):
    gold = json.load(open(GOLDEN))
    wl = inputs.config1(gold["seed"])
    H_lu = np.array(gold["H_re"]) + 1j * np.array(gold["H_im"])
    prec = ie.IE_PREC_FP64 if precision == "fp64" else ie.IE_PREC_MIXED
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        opts = ie.make_opts(restart=30, max_inner=20000, max_outer=20, precision=prec, contraction=True)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, 1e-8, opts)
        E = ctx.get_field()
    assert st == ie.IE_OK and info.final_rel_residual <= 1e-8
    E0 = osolve.incident_field_on_grid(wl.grid, wl.sources[0], wl.freq, wl.sigma0)
    op = oop.FFTOperator(oop.contrast(wl.sigma6, wl.sigma0), wl.grid.h, wl.freq, wl.sigma0)
    assert np.linalg.norm(E0 - op(E)) <= 1.01e-8 * np.linalg.norm(E0)
    allowed = max(10 * gold["oracle_gmres30_vs_lu_max_rel"], 1e-9)
    assert np.max(np.abs(H - H_lu)) <= allowed * np.max(np.abs(H_lu))
    assert info.gmres_iters_total < 0.7 * gold["oracle_gmres30_iterations"]


def test_c1_seed_that_stalls_conventionally_converges_with_contraction(ie):
    wl = inputs.config1(1)
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        opts = ie.make_opts(restart=30, max_inner=8000, max_outer=4, precision=ie.IE_PREC_FP64, contraction=True)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, 1e-8, opts)
        E = ctx.get_field()
    assert st == ie.IE_OK and info.final_rel_residual <= 1e-8
    E0 = osolve.incident_field_on_grid(wl.grid, wl.sources[0], wl.freq, wl.sigma0)
    op = oop.FFTOperator(oop.contrast(wl.sigma6, wl.sigma0), wl.grid.h, wl.freq, wl.sigma0)
    assert np.linalg.norm(E0 - op(E)) <= 1.01e-8 * np.linalg.norm(E0)


@pytest.mark.parametrize("mode", ["gs", "jacobi"])
def test_dd_with_contraction_matches_conventional_dd(ie, mode):
    wl = inputs.config2(0, scale=4)  # 32x32x64, two blocks
    dd = ie.IE_DD_GAUSS_SEIDEL if mode == "gs" else ie.IE_DD_JACOBI
    out = {}
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        for contraction in (False, True):
            opts = ie.make_opts(z_split=wl.z_split, restart=wl.restart, max_inner=4000, max_outer=60,
                                contraction=contraction)
            H, info, st = ctx.solve(wl.sources, wl.receivers, dd, wl.tol, opts)
            assert st == ie.IE_OK and info.final_rel_residual <= wl.tol
            out[contraction] = (H, info.gmres_iters_total)
    H0, H1 = out[False][0], out[True][0]
    # both reach e <= 1e-6; their receiver fields agree to the accuracy that residual allows
    assert np.max(np.abs(H1 - H0)) <= 1e-5 * np.max(np.abs(H0))
    assert out[True][1] <= out[False][1]
