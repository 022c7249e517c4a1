"""Operator parity at the longest pencils the library runs (eq. 10 with the padded FFT lengths that the
large workloads need): L = 512 along x and y (slabs 256 cells wide, as in the 256^3 logging window and the
256x256x512 model's sub-domains) and L = 1024 along z (the whole-grid residual of a 512-cell-high model).

Every precision the solves use is covered: complex64 (GMRES operator, conventional and contraction
form), complex128 and double-float (the FP64-accurate whole-grid residual). References:
  * 256 x 256 slabs: the oracle's direct summation at sampled cells (a full oracle FFT of the padded
    512 x 512 grid per component is too large for a test);
  * 512-cell-high columns: the oracle's FFT operator on the whole output, itself pinned to direct
    summation, plus sampled direct sums;
  * 512-cell-long x or y extents (the largest the ABI accepts: pencils of 1024) and a ragged 300 x 257
    cross-section: the oracle's FFT operator on the whole output.
Tolerances: 1e-5 relative (complex64), 1e-11 relative (complex128, double-float).
"""
import numpy as np
import pytest

from oracle import contraction as oc
from oracle import operator as oop
from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu
F, S0, H = 2.0e6, 0.1, 0.25


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    return _ie


def sampled_reference(s6, x, picks, contraction):
    """(M)u - sum_j K(i - j) dsigma_j (M u)_j at the sampled flat cell indices, by direct summation."""
    nz, ny, nx = s6.shape[:3]
    w = oop.apply_contrast(oc.scaling_tensor(s6, S0), x) if contraction else x
    J = oop.apply_contrast(oop.contrast(s6, S0), w).reshape(3, -1)
    iz, iy, ix = [v.ravel() for v in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")]
    out = []
    for p in picks:
        K = oop.kernel_at_offsets(iz[p] - iz, iy[p] - iy, ix[p] - ix, H, F, S0)
        out.append(w.reshape(3, -1)[:, p] - np.einsum("jpq,qj->p", K, J))
    return np.array(out)


def picks_for(n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([[0, n - 1], rng.integers(0, n, 8)])


@pytest.fixture(scope="module")
def wide_slab():
    g = inputs.centred_grid(256, 256, 16, H)
    s6 = inputs.dipping_ti_with_ellipsoids(g, 3, n_layers=7, n_ellipsoids=5)
    x = inputs.random_field((3, 16, 256, 256), 4)
    picks = picks_for(g.n, 5)
    refs = {form: sampled_reference(s6, x, picks, form == "contraction") for form in ("conventional", "contraction")}
    return g, s6, x, picks, refs


@pytest.mark.parametrize("form,precision,tol", [("conventional", "MIXED", 1e-5), ("contraction", "MIXED", 1e-5),
                                                ("conventional", "FP64", 1e-11), ("conventional", "DFLOAT", 1e-11),
                                                ("contraction", "FP64", 1e-11)])
def test_xy_pencils_512(ie, wide_slab, form, precision, tol):
    g, s6, x, picks, refs = wide_slab
    prec = getattr(ie, "IE_PREC_" + precision)
    with ie.Context(g, H, S0, F) as ctx:
        assert ctx.fft_dims()[:2] == (512, 512)
        ctx.set_contrast(s6)
        y = ctx.matvec_contraction(x, precision=prec) if form == "contraction" else ctx.matvec(x, precision=prec)
    ref = refs[form]
    got = y.reshape(3, -1)[:, picks].T
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@pytest.fixture(scope="module")
def tall_column():
    g = inputs.centred_grid(12, 10, 512, H)
    s6 = inputs.dipping_ti_with_ellipsoids(g, 6, n_layers=7, n_ellipsoids=5)
    x = inputs.random_field((3, 512, 10, 12), 7)
    ref = oop.FFTOperator(oop.contrast(s6, S0), H, F, S0)(x)
    refc = oc.ContractionOperator(s6, H, F, S0)(x)
    return g, s6, x, ref, refc


@pytest.mark.parametrize("form,precision,tol", [("conventional", "MIXED", 1e-5), ("contraction", "MIXED", 1e-5),
                                                ("conventional", "FP64", 1e-11), ("conventional", "DFLOAT", 1e-11)])
def test_z_pencils_1024(ie, tall_column, form, precision, tol):
    g, s6, x, ref, refc = tall_column
    prec = getattr(ie, "IE_PREC_" + precision)
    with ie.Context(g, H, S0, F) as ctx:
        assert ctx.fft_dims()[2] == 1024
        ctx.set_contrast(s6)
        y = ctx.matvec_contraction(x, precision=prec) if form == "contraction" else ctx.matvec(x, precision=prec)
    r = refc if form == "contraction" else ref
    assert np.linalg.norm(y - r) <= tol * np.linalg.norm(r)
    picks = picks_for(g.n, 8)
    direct = sampled_reference(s6, x, picks, form == "contraction")
    assert np.max(np.abs(y.reshape(3, -1)[:, picks].T - direct)) <= max(tol, 1e-10) * np.max(np.abs(direct))


@pytest.mark.parametrize("shape", [(6, 9, 512), (5, 512, 7), (3, 300, 257)])
def test_longest_xy_pencils_and_ragged_sizes(ie, shape):
    # the ABI's largest x and y extents (512 cells: padded pencils of 1024) and a ragged 300/257 case
    # (pencils of 1024 and 512 with most of the padding), all precisions, against the oracle's FFT
    # operator on the whole output
    nz, ny, nx = shape
    g = inputs.Grid(nx, ny, nz, H, (-nx * H / 2 + 0.03, -ny * H / 2 - 0.07, -nz * H / 2 + 0.11))
    s6 = inputs.random_contrast_sigma6(shape, 21, S0, 1.5)
    x = inputs.random_field((3,) + shape, 22)
    ref = oop.FFTOperator(oop.contrast(s6, S0), H, F, S0)(x)
    refc = oc.ContractionOperator(s6, H, F, S0)(x)
    pad = lambda n: 1 << (2 * n - 1).bit_length()
    with ie.Context(g, H, S0, F) as ctx:
        assert ctx.fft_dims() == (pad(nx), pad(ny), pad(nz))
        ctx.set_contrast(s6)
        for prec, tol in ((ie.IE_PREC_MIXED, 1e-5), (ie.IE_PREC_FP64, 1e-11), (ie.IE_PREC_DFLOAT, 1e-11)):
            y = ctx.matvec(x, precision=prec)
            assert np.linalg.norm(y - ref) <= tol * np.linalg.norm(ref), prec
        yc = ctx.matvec_contraction(x, precision=ie.IE_PREC_MIXED)
        assert np.linalg.norm(yc - refc) <= 1e-5 * np.linalg.norm(refc)
