"""Parity at the benchmark's full size (128x128x256, two 128^3 sub-domains, block Gauss-Seidel with the
adaptive tolerance, complex64 + FP64-accurate refinement), in the launch configuration bench.py times,
for both operator forms: the contraction form (the benchmark's headline solve) and the paper's
conventional form (timed beside it).

The oracle cannot solve this system in reasonable time, so it checks what it can compute directly:
  * the sub-domain operator at sampled cells by direct summation over all 2.1 M source cells
    (relative error of the sampled outputs <= 1e-5, the complex64 per-matvec bound): for the
    contraction form y = M u - sum_j K(i - j) dsigma_j (M u)_j with M = 2 sigma0 (sigma + sigma0 I)^-1;
  * the whole-grid FP64 relative residual of the returned field with its own FFT operator
    (must be <= the 1e-6 target, and agree with the value the GPU reports);
  * the receiver fields of the returned field (FP64 closed forms, <= 1e-10 relative).
"""
import numpy as np
import pytest

from oracle import contraction as oc
from oracle import operator as oop
from oracle import physics
from oracle import solve as osolve
from paper_2306_17537_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ie():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie as _ie

    return _ie


@pytest.fixture(scope="module", params=["contraction", "conventional"])
def solved(ie, request):
    form = request.param
    contraction = form == "contraction"
    wl = inputs.config2(0)
    g = wl.grid
    nz = g.nz // 2
    rng = np.random.default_rng(5)
    x = (rng.normal(size=(3, nz, g.ny, g.nx)) + 1j * rng.normal(size=(3, nz, g.ny, g.nx))).astype(np.complex64)
    with ie.Context(g, g.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        opts = ie.make_opts(z_split=wl.z_split, restart=wl.restart, precision=ie.IE_PREC_MIXED, max_inner=4000,
                            max_outer=60, contraction=contraction)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, wl.tol, opts)
        E = ctx.get_field()
        # sampled operator outputs on sub-domain 0 (the launch configuration of the GMRES matvec)
        if contraction:
            y = ctx.matvec_contraction(x.astype(np.complex128), z0=0, nz=nz, precision=ie.IE_PREC_MIXED)
        else:
            import torch

            xd = torch.from_numpy(x.ravel()).cuda()
            yd = torch.empty_like(xd)
            ctx.matvec_dev(xd, yd, z0=0, nz=nz)
            torch.cuda.synchronize()
            y = yd.cpu().numpy().reshape(x.shape)
    return form, wl, H, info, st, E, x, y


def test_full_size_solve_converged(ie, solved):
    _, wl, H, info, st, E, _, _ = solved
    assert st == ie.IE_OK and info.final_rel_residual <= wl.tol


def test_full_size_operator_sampled_against_direct_summation(solved):
    form, wl, _, _, _, _, x, y = solved
    g = wl.grid
    nz = g.nz // 2
    s6 = wl.sigma6[:nz]
    dsig = oop.contrast(s6, wl.sigma0)
    u = x.astype(np.complex128)
    w = oop.apply_contrast(oc.scaling_tensor(s6, wl.sigma0), u) if form == "contraction" else u
    J = oop.apply_contrast(dsig, w).reshape(3, -1)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    iz, iy, ix = iz.ravel(), iy.ravel(), ix.ravel()
    rng = np.random.default_rng(9)
    picks = np.concatenate([[0, len(iz) - 1], rng.integers(0, len(iz), 10)])
    errs, refs = [], []
    for p in picks:
        K = oop.kernel_at_offsets(iz[p] - iz, iy[p] - iy, ix[p] - ix, g.h, wl.freq, wl.sigma0)  # (n, 3, 3)
        ref = w[:, iz[p], iy[p], ix[p]] - np.einsum("jpq,qj->p", K, J)
        errs.append(np.abs(y[:, iz[p], iy[p], ix[p]] - ref))
        refs.append(np.abs(ref))
    assert np.max(errs) <= 1e-5 * np.max(refs)


def test_full_size_residual_checked_by_oracle(solved):
    _, wl, _, info, _, E, _, _ = solved
    g = wl.grid
    E0 = osolve.incident_field_on_grid(g, wl.sources[0], wl.freq, wl.sigma0)
    op = oop.FFTOperator(oop.contrast(wl.sigma6, wl.sigma0), g.h, wl.freq, wl.sigma0)
    e = float(np.linalg.norm(E0 - op(E)) / np.linalg.norm(E0))
    assert e <= wl.tol
    assert abs(e - info.final_rel_residual) <= 1e-3 * e


def test_full_size_receivers_checked_by_oracle(solved):
    _, wl, H, _, _, E, _, _ = solved
    dsig = oop.contrast(wl.sigma6, wl.sigma0)
    ref = osolve.receiver_fields(wl.grid, dsig, E, wl.sources[0], wl.receivers, wl.freq, wl.sigma0)
    assert np.max(np.abs(H[0] - ref)) <= 1e-10 * np.max(np.abs(ref))
    # the scattered part is a visible fraction of the total at the near receiver
    H0 = physics.incident_H(wl.receivers, wl.sources[0].pos, wl.sources[0].moment, wl.freq, wl.sigma0)
    assert np.abs(H[0, 0, 2] - H0[0, 2]) > 1e-3 * np.abs(H0[0, 2])
