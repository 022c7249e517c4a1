"""GPU parity of each hot-path step against the CPU FP64 oracle, called through the C ABI.

Tolerances (relative L2 or max-abs over max):
  * FP64 kernels (Green spectra, incident field, complex128 operator, interactions, receivers) and
    the double-float operator of the outer residual: 1e-11 — the same closed forms and FFT
    convolution at (at least) 46-bit precision, differing only in rounding order.
  * complex64 operator: 1e-5 per matvec (FP32 FFT of length <= 1024 per axis has relative error
    ~ eps32 * log2(P) ~ 1e-6; the Green spectra are rounded from FP64).
Shapes cover single cells, odd and prime sizes, non-power-of-two padding and several FFT tiles.
"""
import numpy as np
import pytest

from oracle import operator as oop
from oracle import physics
from oracle import solve as osolve
from oracle.gmres import gmres as ogmres
from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu

F, S0 = 1.0e5, 0.1
SHAPES = [(1, 1, 1), (3, 5, 7), (8, 6, 10), (16, 16, 16), (5, 20, 9), (33, 4, 6), (2, 1, 40)]  # (nz, ny, nx)
COMP_PQ = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    return _ie


def _grid(shape, h=0.5):
    nz, ny, nx = shape
    return inputs.Grid(nx, ny, nz, h, (-nx * h / 2 + 0.1, -ny * h / 2 - 0.05, -nz * h / 2 + 0.02))


def _ctx(ie, shape, seed=0, spread=0.5):
    g = _grid(shape)
    s6 = inputs.random_contrast_sigma6(shape, seed, S0, spread)
    ctx = ie.Context(g, g.h, S0, F)
    ctx.set_contrast(s6)
    return ctx, g, s6


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("shape", SHAPES)
def test_green_spectrum_matches_oracle(ie, shape):
    ctx, g, _ = _ctx(ie, shape)
    for nz_set in sorted({shape[0], max(1, shape[0] // 2)}):
        Lx, Ly, Lz = ctx.fft_dims(nz_set)
        Kh = oop.green_spectrum((nz_set, shape[1], shape[2]), g.h, F, S0, pad=(Lz, Ly, Lx)) / (Lx * Ly * Lz)
        for comp, (p, q) in enumerate(COMP_PQ):
            got, dims = ctx.green_spectrum(comp, nz_set)
            ref = Kh[p, q][: Lz // 2 + 1, : Ly // 2 + 1, : Lx // 2 + 1]
            assert dims == (Lx, Ly, Lz)
            assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(Kh[p, p] if p == q else Kh[0, 0]))
    ctx.close()


@pytest.mark.parametrize("shape", SHAPES[1:])
def test_incident_field_matches_oracle(ie, shape):
    ctx, g, _ = _ctx(ie, shape)
    for src in [inputs.Dipole((0.0, 0.0, 0.0), (0.0, 0.0, 1.0)), inputs.Dipole((0.3, -0.2, 0.7), (0.5, -1.0, 0.25))]:
        got = ctx.incident_field(src)
        ref = osolve.incident_field_on_grid(g, src, F, S0)
        assert rel(got, ref) <= 1e-13
    ctx.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_operator_fp64_matches_oracle(ie, shape):
    ctx, g, s6 = _ctx(ie, shape, seed=2)
    x = inputs.random_field((3,) + shape, 5)
    ref = oop.FFTOperator(oop.contrast(s6, S0), g.h, F, S0)(x)
    assert rel(ctx.matvec(x, precision=ie.IE_PREC_FP64), ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_operator_double_float_matches_oracle(ie, shape):
    # the FP64-accurate whole-grid residual runs on these FP32-pair kernels (about 46-bit arithmetic)
    ctx, g, s6 = _ctx(ie, shape, seed=2)
    x = inputs.random_field((3,) + shape, 5)
    ref = oop.FFTOperator(oop.contrast(s6, S0), g.h, F, S0)(x)
    assert rel(ctx.matvec(x, precision=ie.IE_PREC_DFLOAT), ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_operator_complex64_matches_oracle(ie, shape):
    ctx, g, s6 = _ctx(ie, shape, seed=3)
    x = inputs.random_field((3,) + shape, 6)
    ref = oop.FFTOperator(oop.contrast(s6, S0), g.h, F, S0)(x)
    assert rel(ctx.matvec(x, precision=ie.IE_PREC_MIXED), ref) <= 1e-5
    ctx.close()


def test_operator_direct_summation_small(ie):
    shape = (4, 3, 5)
    ctx, g, s6 = _ctx(ie, shape, seed=4)
    x = inputs.random_field((3,) + shape, 7)
    ref = oop.matvec_direct(x, oop.contrast(s6, S0), g.h, F, S0)
    assert rel(ctx.matvec(x, precision=ie.IE_PREC_FP64), ref) <= 1e-11


@pytest.mark.parametrize("z0,nz", [(0, 5), (5, 7), (3, 9), (11, 1)])
def test_block_operator_on_slab(ie, z0, nz):
    shape = (12, 6, 7)
    ctx, g, s6 = _ctx(ie, shape, seed=8)
    x = inputs.random_field((3, nz) + shape[1:], 9)
    ref = oop.FFTOperator(oop.contrast(s6, S0)[z0:z0 + nz], g.h, F, S0)(x)
    assert rel(ctx.matvec(x, z0=z0, nz=nz, precision=ie.IE_PREC_FP64), ref) <= 1e-11
    assert rel(ctx.matvec(x, z0=z0, nz=nz, precision=ie.IE_PREC_MIXED), ref) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("src_slab,dst_slab", [((0, 4), (4, 8)), ((6, 6), (0, 3)), ((2, 5), (2, 5)), ((0, 12), (9, 3))])
def test_interaction_matches_oracle(ie, src_slab, dst_slab):
    shape = (12, 5, 6)
    ctx, g, s6 = _ctx(ie, shape, seed=10)
    (zs0, nzs), (zt0, nzt) = src_slab, dst_slab
    x = inputs.random_field((3, nzs) + shape[1:], 11)
    dsig = oop.contrast(s6, S0)
    full = oop.FFTOperator(dsig, g.h, F, S0)
    J = np.zeros((3,) + shape, dtype=complex)
    J[:, zs0:zs0 + nzs] = oop.apply_contrast(dsig[zs0:zs0 + nzs], x)
    ref = full.G(J)[:, zt0:zt0 + nzt]
    assert rel(ctx.interaction(x, zs0, nzs, zt0, nzt), ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("shape", [(4, 4, 4), (9, 7, 5), (16, 16, 16)])
def test_receiver_fields_match_oracle(ie, shape):
    ctx, g, s6 = _ctx(ie, shape, seed=12)
    E = inputs.random_field((3,) + shape, 13)
    src = inputs.Dipole((0.0, 0.0, 0.0), (0.3, 0.1, 1.0))
    rx = np.array([[0.0, 0.0, 0.5], [0.0, 0.0, 1.0], [0.25, -0.5, 2.0], [5.0, 1.0, -3.0], [0.1, 0.2, 0.3],
                   [1.0, 1.0, 1.0], [-2.0, 0.0, 0.0], [0.0, 3.0, 0.0], [0.0, 0.0, -7.5]])
    ref = osolve.receiver_fields(g, oop.contrast(s6, S0), E, src, rx, F, S0)
    got = ctx.receiver_fields(E, src, rx)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    ctx.close()


def test_gmres_fp64_matches_oracle_gmres(ie):
    shape = (6, 5, 7)
    ctx, g, s6 = _ctx(ie, shape, seed=14, spread=0.8)
    op = oop.FFTOperator(oop.contrast(s6, S0), g.h, F, S0)
    b = osolve.incident_field_on_grid(g, inputs.Dipole((0.0, 0.0, 0.0), (0.0, 0.0, 1.0)), F, S0)
    x_ref, info = ogmres(op, b, None, tol=1e-10, restart=10, max_iter=500)
    x, its, rr, st = ctx.gmres(b, tol=1e-10, restart=10, max_iter=500, precision=ie.IE_PREC_FP64)
    assert st == ie.IE_OK and rr <= 1e-10
    assert abs(its - info.iterations) <= 1
    assert rel(x, x_ref) <= 1e-8
    # warm start from x0 (the paper's inner solves start from the previous sweep)
    x2, its2, rr2, _ = ctx.gmres(b, x0=x_ref, tol=1e-12, restart=10, max_iter=500, precision=ie.IE_PREC_FP64)
    assert its2 <= its and rr2 <= 1e-12
    ctx.close()


def test_gmres_complex64_reaches_single_precision_tolerance(ie):
    shape = (8, 8, 8)
    ctx, g, s6 = _ctx(ie, shape, seed=15)
    op = oop.FFTOperator(oop.contrast(s6, S0), g.h, F, S0)
    b = inputs.random_field((3,) + shape, 16)
    x, its, rr, st = ctx.gmres(b, tol=1e-5, restart=30, max_iter=500, precision=ie.IE_PREC_MIXED)
    assert st == ie.IE_OK and rr <= 1e-5
    true = np.linalg.norm(b - op(x)) / np.linalg.norm(b)
    assert true <= 2e-5
    ctx.close()
