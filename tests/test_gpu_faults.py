"""Host-side fault injection and out-of-bounds-write checks (no GPU fault is ever caused).

* Allocation failure: ie_debug_fail_allocation makes one device allocation report out-of-memory
  without calling cudaMalloc. A solve that meets it must return IE_ENOMEM, and the same context must
  then solve the same problem correctly (compared with a fresh context). The failure is placed at
  every point of the allocation sequence of a solve on new sub-domain heights (spectra, convolution
  workspaces, Krylov basis, contraction tensors).
* Guard regions (a host-side stand-in for a memory checker): device outputs of the device-pointer
  entry points are written into the middle of a larger buffer filled with a sentinel; the sentinel
  before and after must be untouched, and read-only inputs unchanged.
"""
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


def _solve(ie, ctx, wl, split, contraction):
    opts = ie.make_opts(z_split=split, restart=20, max_inner=3000, max_outer=40, contraction=contraction)
    return ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, wl.tol, opts)


def _mild_workload():
    """16 x 16 x 32 cells with a moderate random anisotropic contrast (every split converges quickly in
    both operator forms), the coaxial tool at the centre."""
    wl = inputs.config2(0, scale=8)
    wl.sigma6 = inputs.random_contrast_sigma6((32, 16, 16), 21, wl.sigma0, 0.7)
    return wl


@pytest.mark.parametrize("contraction", [False, True])
def test_injected_allocation_failure_returns_enomem_and_context_stays_usable(ie, contraction):
    wl = _mild_workload()
    g = wl.grid
    splits = [[0, 10, 32], [0, 7, 20, 32], [0, 5, 32], [0, 12, 25, 32], [0, 3, 29, 32], [0, 9, 32], [0, 14, 32]]
    fired = 0
    try:
        with ie.Context(g, g.h, wl.sigma0, wl.freq) as ctx:
            ctx.set_contrast(wl.sigma6)
            H_base, _, _ = _solve(ie, ctx, wl, wl.z_split, contraction)
            for after, split in zip([0, 1, 2, 3, 4, 6, 9], splits):
                ie.debug_fail_allocation(after)
                try:
                    _solve(ie, ctx, wl, split, contraction)
                except ie.IEError as e:
                    assert e.status == ie.IE_ENOMEM, str(e)
                    fired += 1
                ie.debug_fail_allocation(-1)
                H, info, st = _solve(ie, ctx, wl, split, contraction)  # the same context, same problem
                assert st == ie.IE_OK and info.final_rel_residual <= wl.tol
                with ie.Context(g, g.h, wl.sigma0, wl.freq) as fresh:
                    fresh.set_contrast(wl.sigma6)
                    H_ref, _, _ = _solve(ie, fresh, wl, split, contraction)
                assert np.max(np.abs(H - H_ref)) <= 1e-5 * np.max(np.abs(H_ref))
                # every split solves the same discrete system (e <= 1e-6)
                assert np.max(np.abs(H - H_base)) <= 1e-4 * np.max(np.abs(H_base))
    finally:
        ie.debug_fail_allocation(-1)
    assert fired >= 3  # the injected failure was met at several points of the sequence


def test_injected_failure_in_create(ie):
    wl = inputs.config2(0, scale=8)
    g = wl.grid
    try:
        for after in range(4):
            ie.debug_fail_allocation(after)
            with pytest.raises(ie.IEError) as e:
                ie.Context(g, g.h, wl.sigma0, wl.freq)
            assert e.value.status == ie.IE_ENOMEM
    finally:
        ie.debug_fail_allocation(-1)
    with ie.Context(g, g.h, wl.sigma0, wl.freq) as ctx:  # and creation works again
        ctx.set_contrast(wl.sigma6)


GUARD = 4096  # complex elements of sentinel on each side


def _guarded(torch, n, dtype):
    buf = torch.full((n + 2 * GUARD,), complex(1.25e30, -7.5e29), dtype=dtype, device="cuda")
    return buf, buf[GUARD:GUARD + n]


def _guards_intact(torch, buf, n):
    sent = torch.tensor(complex(1.25e30, -7.5e29), dtype=buf.dtype, device="cuda")
    return bool(torch.all(buf[:GUARD] == sent)) and bool(torch.all(buf[GUARD + n:] == sent))


@pytest.mark.parametrize("shape", [(16, 12, 20), (7, 5, 3), (32, 16, 8)])
def test_device_outputs_stay_inside_their_buffers(ie, shape):
    import torch

    nz, ny, nx = shape
    g = inputs.centred_grid(nx, ny, nz, 0.5)
    s6 = inputs.random_contrast_sigma6(shape, 3, 0.1, 0.5)
    n = 3 * g.n
    with ie.Context(g, g.h, 0.1, 1e5) as ctx:
        ctx.set_contrast(s6)
        xbuf, x = _guarded(torch, n, torch.complex64)
        x.copy_(torch.randn(n, dtype=torch.complex64, device="cuda"))
        x_before = xbuf.clone()
        for call in (ctx.matvec_dev, ctx.matvec_dev_noalloc):
            ybuf, y = _guarded(torch, n, torch.complex64)
            call(x, y)
            torch.cuda.synchronize()
            assert _guards_intact(torch, ybuf, n)
            assert torch.all(torch.isfinite(torch.view_as_real(y)))
        z0, nzs = nz // 3, max(1, nz // 2)
        ns = 3 * nzs * ny * nx
        ybuf, y = _guarded(torch, ns, torch.complex64)
        ctx.matvec_dev(x[:ns], y, z0=z0, nz=nzs)
        torch.cuda.synchronize()
        assert _guards_intact(torch, ybuf, ns)
        assert torch.equal(xbuf, x_before)
        src = inputs.Dipole((0.1, 0.05, 0.13), (0.0, 0.0, 1.0))  # off every cell centre
        ebuf, e = _guarded(torch, n, torch.complex128)
        ctx.incident_field_dev(src, e)
        ctx.solve([src], np.array([[0.13, 0.07, 1.1]]), ie.IE_DD_NONE, 1e-6, ie.make_opts(restart=20, max_inner=2000))
        fbuf, f = _guarded(torch, n, torch.complex128)
        ctx.get_field_dev(f)
        torch.cuda.synchronize()
        assert _guards_intact(torch, ebuf, n) and _guards_intact(torch, fbuf, n)
