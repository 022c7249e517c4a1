"""The no-allocation sub-domain operator (ie_matvec_dev_noalloc) against ie_matvec_dev.

Callers that cannot allocate device memory during a call (stream capture, fixed memory budgets) use
this entry point; it keeps its FFT intermediates in a fixed library-owned device array. This file is
collected last on purpose, and passes both alone and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu

F, S0 = 1.0e5, 0.1


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    return _ie


@pytest.mark.parametrize("shape", [(16, 12, 20), (5, 7, 3), (32, 32, 32)])
def test_noalloc_matches_allocating_operator_twice(ie, shape):
    import torch

    nz, ny, nx = shape
    g = inputs.centred_grid(nx, ny, nz, 0.5)
    s6 = inputs.random_contrast_sigma6(shape, 7, S0, 0.5)
    with ie.Context(g, g.h, S0, F) as ctx:
        ctx.set_contrast(s6)
        torch.manual_seed(0)
        x = torch.randn(3 * g.n, dtype=torch.complex64, device="cuda")
        y_ref = torch.empty_like(x)
        ctx.matvec_dev(x, y_ref)
        ys = []
        for _ in range(2):  # two calls in a row share (and reuse) the scratch array
            y = torch.full_like(x, float("nan"))
            ctx.matvec_dev_noalloc(x, y)
            ys.append(y)
        torch.cuda.synchronize()
    ref = y_ref.cpu().numpy()
    for y in ys:
        got = y.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


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
