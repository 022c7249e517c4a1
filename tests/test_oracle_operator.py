"""Pins for the oracle's discrete operator (eqs. 8 and 10): FFT form == direct summation == dense."""
import numpy as np
import pytest

from oracle import operator as op
from paper_2306_17537_gb300 import inputs

H_CELL, F, S0 = 0.5, 1.0e5, 0.1


def _case(shape, seed):
    s6 = inputs.random_contrast_sigma6(shape, seed, S0)
    dsig = op.contrast(s6, S0)
    E = inputs.random_field((3,) + tuple(shape), seed + 100)
    return dsig, E


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 7), (4, 4, 4), (2, 3, 6), (5, 1, 2)])
def test_fft_operator_equals_direct_summation(shape):
    dsig, E = _case(shape, 7)
    y_direct = op.matvec_direct(E, dsig, H_CELL, F, S0)
    y_fft = op.FFTOperator(dsig, H_CELL, F, S0)(E)
    assert np.linalg.norm(y_fft - y_direct) <= 1e-13 * np.linalg.norm(y_direct)


def test_fft_operator_pad_independence():
    shape = (3, 4, 5)
    dsig, E = _case(shape, 11)
    y2n = op.FFTOperator(dsig, H_CELL, F, S0)(E)
    for pad in [(5, 7, 9), (8, 8, 16), (7, 12, 10)]:
        y = op.FFTOperator(dsig, H_CELL, F, S0, pad=pad)(E)
        assert np.linalg.norm(y - y2n) <= 1e-13 * np.linalg.norm(y2n)


def test_dense_matrix_equals_direct_summation():
    shape = (2, 3, 2)
    dsig, E = _case(shape, 5)
    A = op.dense_matrix(dsig, H_CELL, F, S0)
    y = (A @ E.ravel()).reshape(E.shape)
    assert np.allclose(y, op.matvec_direct(E, dsig, H_CELL, F, S0), rtol=1e-13, atol=1e-13)


def test_kernel_translation_invariance_and_symmetry():
    # K(d) = K(-d) and K_pq = K_qp: the discrete operator G is a symmetric matrix
    shape = (2, 2, 3)
    dsig = op.contrast(np.tile(np.array([S0 + 1, S0 + 1, S0 + 1, 0, 0, 0]), shape + (1,)), S0)
    A = op.dense_matrix(dsig, H_CELL, F, S0)
    G = (np.eye(A.shape[0]) - A)  # = K * 1 (unit isotropic contrast)
    assert np.allclose(G, G.T, rtol=1e-13, atol=1e-15)


def test_padded_kernel_parity_per_axis():
    # The octant compression of the Green spectra relies on these parities of the 2n embedding:
    # K_pp even in every axis; K_xy odd in x and y; K_xz odd in x and z; K_yz odd in y and z.
    shape = (3, 4, 5)
    K = op.padded_kernel(shape, H_CELL, F, S0)  # (3, 3, pz, py, px)
    flip = lambda a, ax: np.roll(np.flip(a, axis=ax), 1, axis=ax)  # index m -> (-m) mod p
    par = {(0, 0): (1, 1, 1), (1, 1): (1, 1, 1), (2, 2): (1, 1, 1), (0, 1): (1, -1, -1),
           (0, 2): (-1, 1, -1), (1, 2): (-1, -1, 1)}  # signs along (z, y, x)
    for (p, q), sg in par.items():
        for ax, s in zip((0, 1, 2), sg):
            assert np.allclose(flip(K[p, q], ax), s * K[p, q], rtol=0, atol=1e-15)


def test_contrast_definition():
    s6 = np.array([[[[1.0, 2.0, 3.0, 0.1, 0.2, 0.3]]]])
    d = op.contrast(s6, 0.5)[0, 0, 0]
    assert np.allclose(d, np.array([[0.5, 0.1, 0.2], [0.1, 1.5, 0.3], [0.2, 0.3, 2.5]]))
