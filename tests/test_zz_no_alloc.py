"""The no-allocation sub-domain operator (ie_matvec_dev_noalloc).

Some callers cannot let a library call allocate device memory: an application that owns the GPU's
memory and gives the library a fixed budget (a cudaMalloc inside the call could fail at an arbitrary
point), or a latency-bound loop where cudaMalloc/cudaFree may synchronise the device. For them this
entry point keeps its FFT intermediates in a fixed library-owned device array.

Checked here, through the C ABI: its output against the allocating entry point ie_matvec_dev (1e-5
relative, the complex64 operator tolerance of the other tests) and against the FP64 oracle operator
(1e-5), on two calls in a row that share the array; that the device's free memory does not change
across calls; a sub-slab (z0 > 0, nz < the grid height) after ie_matvec_dev prepared its spectra;
IE_ESTATE for a height without spectra; IE_EINVAL beyond the array's size. The sizes change from test
to test (a large slab, then a small one), so stale contents of the shared array would show.

This file is collected last on purpose, and passes both alone and after the rest of the suite.
"""
import numpy as np
import pytest

from oracle import operator as oop
from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu

F, S0 = 1.0e5, 0.1


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    return _ie


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 12, 20), (5, 7, 3)])
def test_noalloc_matches_allocating_operator_and_oracle_twice(ie, shape):
    import torch

    nz, ny, nx = shape
    g = inputs.centred_grid(nx, ny, nz, 0.5)
    s6 = inputs.random_contrast_sigma6(shape, 7, S0, 0.5)
    xh = inputs.random_field((3,) + shape, 8).astype(np.complex64)
    oracle = oop.FFTOperator(oop.contrast(s6, S0), g.h, F, S0)(xh.astype(np.complex128))
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        x = torch.from_numpy(xh.ravel()).cuda()
        y_ref = torch.empty_like(x)
        ctx.matvec_dev(x, y_ref)
        ys = [torch.full_like(x, float("nan")) for _ in range(3)]
        ctx.matvec_dev_noalloc(x, ys[0])  # first call on the device may look up the array's address
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for y in ys[1:]:  # two more calls in a row share (and reuse) the array
            ctx.matvec_dev_noalloc(x, y)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = y_ref.cpu().numpy().reshape(oracle.shape)
    for y in ys:
        got = y.cpu().numpy().reshape(oracle.shape)
        assert rel(got, ref) <= 1e-5
        assert rel(got, oracle) <= 1e-5


def test_noalloc_sub_slab_after_spectra_prepared(ie):
    import torch

    shape = (24, 10, 14)
    z0, nz = 9, 11
    g = inputs.centred_grid(shape[2], shape[1], shape[0], 0.5)
    s6 = inputs.random_contrast_sigma6(shape, 17, S0, 1.0)
    xh = inputs.random_field((3, nz) + shape[1:], 18).astype(np.complex64)
    oracle = oop.FFTOperator(oop.contrast(s6[z0:z0 + nz], S0), g.h, F, S0)(xh.astype(np.complex128))
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        x = torch.from_numpy(xh.ravel()).cuda()
        y = torch.full_like(x, float("nan"))
        with pytest.raises(ie.IEError) as e:  # no spectra for this height yet
            ctx.matvec_dev_noalloc(x, y, z0=z0, nz=nz)
        assert e.value.status == ie.IE_ESTATE
        y_ref = torch.empty_like(x)
        ctx.matvec_dev(x, y_ref, z0=z0, nz=nz)  # prepares the spectra of an 11-plane slab
        outs = []
        for _ in range(2):
            y = torch.full_like(x, float("nan"))
            ctx.matvec_dev_noalloc(x, y, z0=z0, nz=nz)
            outs.append(y)
        torch.cuda.synchronize()
    ref = y_ref.cpu().numpy().reshape(oracle.shape)
    for y in outs:
        got = y.cpu().numpy().reshape(oracle.shape)
        assert rel(got, ref) <= 1e-5 and rel(got, oracle) <= 1e-5


def test_noalloc_rejects_slabs_beyond_its_scratch(ie):
    import torch

    g = inputs.centred_grid(64, 64, 64, 0.5)  # needs 24*64*128*(64+128) bytes > 16 MiB
    s6 = np.zeros((64, 64, 64, 6))
    s6[..., :3] = 0.2
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        x = torch.zeros(3 * g.n, dtype=torch.complex64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(ie.IEError) as e:
            ctx.matvec_dev_noalloc(x, y)
        assert e.value.status == ie.IE_EINVAL and "limit" in str(e.value)
