"""Every FFT tile variant computes the same operator (eq. 10), bit for bit.

The autotuner keeps whichever variant of the y passes (P2, P4: three tiles) and of the z pass (P3:
twelve tiles, with and without TMA staging, with and without mirrored rows ky / Ly - ky) is fastest
for a shape, so the solves only ever exercise the winners. Here ie_debug_force_tile runs each variant
in turn on the same input and the outputs are compared with the autotuned one exactly, and the
autotuned one with the oracle's FFT operator. Shapes: a ragged box (33 x 24 x 20: pencils of 128, 64
and 64) and a tall column (7 x 5 x 300: z pencils of 1024, y rows of 16, so the mirrored tiles pair
rows of a short y axis).
"""
import numpy as np
import pytest

from oracle import contraction as oc
from oracle import operator as oop
from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu
F, S0, H = 2.0e6, 0.1, 0.25
P3_VARIANTS = 12
FLOAT_ONLY_P3 = (8, 9)  # mirrored 256-thread z tiles: built for complex64 only


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    yield _ie
    for p in (2, 3, 4):
        _ie.debug_force_tile(p, -1)


def _case(shape, seed):
    nz, ny, nx = shape
    g = inputs.Grid(nx, ny, nz, H, (-nx * H / 2 + 0.05, -ny * H / 2 - 0.02, -nz * H / 2 + 0.07))
    s6 = inputs.random_contrast_sigma6(shape, seed, S0, 1.2)
    x = inputs.random_field((3,) + shape, seed + 1)
    return g, s6, x


@pytest.mark.parametrize("shape", [(20, 24, 33), (300, 5, 7)])
def test_every_tile_variant_gives_the_same_operator(ie, shape):
    g, s6, x = _case(shape, 31)
    ref = oop.FFTOperator(oop.contrast(s6, S0), H, F, S0)(x)
    refc = oc.ContractionOperator(s6, H, F, S0)(x)
    precs = ((ie.IE_PREC_MIXED, 1e-5), (ie.IE_PREC_FP64, 1e-11), (ie.IE_PREC_DFLOAT, 1e-11))
    with ie.Context(g, H, S0, F) as ctx:
        ctx.set_contrast(s6)
        for p in (2, 3, 4):
            ie.debug_force_tile(p, -1)
        auto = {prec: ctx.matvec(x, precision=prec) for prec, _ in precs}
        autoc = ctx.matvec_contraction(x, precision=ie.IE_PREC_MIXED)
        for prec, tol in precs:
            assert np.linalg.norm(auto[prec] - ref) <= tol * np.linalg.norm(ref), prec
        assert np.linalg.norm(autoc - refc) <= 1e-5 * np.linalg.norm(refc)
        try:
            for v in range(P3_VARIANTS):
                ie.debug_force_tile(3, v)
                for prec, _ in precs:
                    if v in FLOAT_ONLY_P3 and prec != ie.IE_PREC_MIXED:
                        continue
                    assert np.array_equal(ctx.matvec(x, precision=prec), auto[prec]), (v, prec)
                assert np.array_equal(ctx.matvec_contraction(x, precision=ie.IE_PREC_MIXED), autoc), v
            ie.debug_force_tile(3, -1)
            for p in (2, 4):
                for v in range(3):
                    ie.debug_force_tile(p, v)
                    for prec, _ in precs:
                        assert np.array_equal(ctx.matvec(x, precision=prec), auto[prec]), (p, v, prec)
                ie.debug_force_tile(p, -1)
        finally:
            for p in (2, 3, 4):
                ie.debug_force_tile(p, -1)


def test_force_tile_rejects_out_of_range(ie):
    for p, v in ((1, 0), (5, 0), (3, 12), (2, 3), (4, -2)):
        with pytest.raises(ie.IEError):
            ie.debug_force_tile(p, v)
    ie.debug_force_tile(3, -1)
