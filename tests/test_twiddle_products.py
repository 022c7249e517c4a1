"""Accuracy of the float twiddle scheme of the register FFT.

In complex64 each butterfly loads only the power-of-two twiddles w, w^2, w^4, w^8 of its stage from
the table exp(-2 pi i k / 1024) (each entry correctly rounded to float) and forms every other w^r as
a product of the entries named by r's binary digits. This emulates that arithmetic in numpy float32,
with the table rounded the same way and each complex product rounded per operation. It checks, for
every stage shape the FFTs use (radix 2 to 16, stride 1 to 512), that no twiddle is more than a few
float ulps from exp(-2 pi i k r / (Ns R)). The FFT's own roundings are of the same size, so the
scheme adds no new error scale.
"""
import numpy as np

TWN = 1024


def _table():
    k = np.arange(TWN)
    return np.exp(-2j * np.pi * k / TWN).astype(np.complex64)


def _cmul32(a, b):
    # complex product with every real operation rounded to float32
    ar, ai = np.float32(a.real), np.float32(a.imag)
    br, bi = np.float32(b.real), np.float32(b.imag)
    re = np.float32(np.float32(ar * br) - np.float32(ai * bi))
    im = np.float32(np.float32(ar * bi) + np.float32(ai * br))
    return np.complex64(complex(re, im))


def _twiddles(tab, q, R):
    p = {}
    b = 1
    while b < R:
        p[b] = tab[q * b]
        b <<= 1
    for r in range(3, R):
        if r & (r - 1):
            hb = 1 << (r.bit_length() - 1)
            p[r] = _cmul32(p[hb], p[r - hb])
    return p


def test_power_product_twiddles_stay_within_a_few_ulps():
    tab = _table()
    eps = np.finfo(np.float32).eps
    worst = 0.0
    for R in (2, 4, 8, 16):
        NS = 2  # every stage after the first: stride NS a power of two, NS * R <= 1024
        while NS * R <= TWN:
            for k in range(NS):
                q = k * (TWN // (NS * R))
                p = _twiddles(tab, q, R)
                for r in range(1, R):
                    exact = np.exp(-2j * np.pi * k * r / (NS * R))
                    worst = max(worst, abs(complex(p[r]) - exact))
            NS *= 2
    # table entries carry at most half an ulp per component, and up to four of them meet with three
    # roundings; the worst case over all stages comes to about 1.5 ulps of a unit-modulus number
    assert worst <= 4 * eps, worst / eps
    assert worst > 0.0
