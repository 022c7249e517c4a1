"""Pins for the FNO reference (oracle/fno.py): the truncated transforms against numpy.fft, the
spectral convolution against an explicit mode-filtered FFT, and every gradient against central
finite differences on a tiny network."""
import numpy as np
import pytest

from oracle import fno


def test_truncated_transform_matches_numpy_fft():
    rng = np.random.default_rng(0)
    n, m = 8, 3
    v = rng.normal(size=(2, n, n, n, 2))
    Fxy, Fz, cz = fno.dft_matrices(n, m)
    V = fno.T(v, Fxy, Fz)
    full = np.fft.fftn(v, axes=(1, 2, 3))
    kxy, kz = fno.kept_modes(n, m)
    assert np.allclose(V, full[:, kz][:, :, kxy][:, :, :, kxy], atol=1e-12)


def test_spectral_convolution_equals_mode_filtered_rfft():
    # with R = identity per mode, S(T(v)) keeps the retained modes of the half spectrum (z the halved
    # axis) and inverts it with the real-output inverse transform, which numpy computes directly
    rng = np.random.default_rng(1)
    n, m = 8, 3
    v = rng.normal(size=(1, n, n, n, 1))
    Fxy, Fz, cz = fno.dft_matrices(n, m)
    k = fno.S(fno.T(v, Fxy, Fz), Fxy, Fz, cz, n)
    half = np.fft.rfftn(v, axes=(2, 3, 1))  # (1, n//2+1, n, n, 1): axis 1 (z) is the halved axis
    kxy, kz = fno.kept_modes(n, m)
    mask = np.zeros(half.shape[1:4], bool)
    mask[np.ix_(kz, kxy, kxy)] = True
    ref = np.fft.irfftn(np.where(mask[None, :, :, :, None], half, 0), s=(n, n, n), axes=(2, 3, 1))
    assert np.allclose(k, ref, atol=1e-12)


def test_gelu_gradient():
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    assert np.allclose(fno.gelu_grad(x), (fno.gelu(x + h) - fno.gelu(x - h)) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("which", ["P", "p", "W", "w", "R", "Q1", "q1", "Q2", "q2"])
def test_backward_matches_finite_differences(which):
    rng = np.random.default_rng(2)
    n, m = 6, 2
    prm = fno.init_params(3, cin=3, width=4, cout=2, hidden=5, layers=2, n=n, modes=m)
    prm.p = rng.normal(size=prm.p.shape) * 0.1
    prm.w = [rng.normal(size=w.shape) * 0.1 for w in prm.w]
    a = rng.normal(size=(2, n, n, n, 3))
    t = rng.normal(size=(2, n, n, n, 2))
    u, cache = fno.forward(prm, a, keep=True)
    loss, du = fno.rel_l2_loss(u, t)
    g = fno.backward(prm, cache, du)
    tgt = getattr(prm, which)
    grads = getattr(g, which)
    arrs = tgt if isinstance(tgt, list) else [tgt]
    garrs = grads if isinstance(grads, list) else [grads]
    for arr, garr in zip(arrs, garrs):
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(3)]:
            for part in ([1.0, 1j] if np.iscomplexobj(arr) else [1.0]):
                h = 1e-6
                old = arr[idx]
                arr[idx] = old + h * part
                lp, _ = fno.rel_l2_loss(fno.forward(prm, a), t)
                arr[idx] = old - h * part
                lm, _ = fno.rel_l2_loss(fno.forward(prm, a), t)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                an = garr[idx].real if part == 1.0 else garr[idx].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (which, idx, part, fd, an)
