"""CPU FP64 reference of the 3D Fourier neural operator used as a GMRES warm start. FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). This network is not part of the paper; it is
the learned initial guess of the sub-domain solves (an extension). The reference defines what the
GPU kernels must compute, forward and backward:

  input  a : (B, N, N, N, Cin) real, axes (z, y, x, channel)
  lift   v0 = a P + p                                   (Cin -> C)
  layer  v_{l+1} = act( v_l W_l + w_l + K_l(v_l) ),  act = GELU except after the last layer
         K_l(v) = S( R_l * T(v) )   (spectral convolution on the retained modes)
  head   u = GELU(v_L Q1 + q1) Q2 + q2                   (C -> H -> Cout)

T is the truncated DFT of a real field: kz in {0..M-1} (one half of the Hermitian spectrum),
ky, kx in {0..M-1} U {N-M..N-1}; T(v)[kz,ky,kx] = sum_{z,y,x} v e^{-2 pi i (kz z + ky y + kx x)/N}.
S is its truncated inverse with real output, S(W)[z,y,x] = N^-3 Re sum c_kz W e^{+2 pi i (...)/N},
c_0 = 1 and c_kz = 2 otherwise (the modes -kz are the conjugates of +kz). R_l holds one complex
C x C matrix per retained mode. GELU is x/2 (1 + erf(x / sqrt 2)).

Gradients are with respect to the real inner product (complex parameters: d/dRe + i d/dIm).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.special import erf


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def kept_modes(n: int, m: int):
    """Retained indices along x/y (both ends) and along z (lower half)."""
    kxy = np.concatenate([np.arange(m), np.arange(n - m, n)])
    return kxy, np.arange(m)


def dft_matrices(n: int, m: int):
    kxy, kz = kept_modes(n, m)
    r = np.arange(n)
    Fxy = np.exp(-2j * np.pi * np.outer(kxy, r) / n)  # (2m, n)
    Fz = np.exp(-2j * np.pi * np.outer(kz, r) / n)  # (m, n)
    cz = np.where(kz == 0, 1.0, 2.0)
    return Fxy, Fz, cz


@dataclass
class Params:
    P: np.ndarray
    p: np.ndarray
    W: list
    w: list
    R: list  # complex (m, 2m, 2m, C, C): [kz, ky, kx, in, out]
    Q1: np.ndarray
    q1: np.ndarray
    Q2: np.ndarray
    q2: np.ndarray

    def flat(self):
        return [self.P, self.p] + self.W + self.w + self.R + [self.Q1, self.q1, self.Q2, self.q2]


def init_params(seed: int, cin=12, width=32, cout=6, hidden=128, layers=4, n=64, modes=12, dtype=np.float64):
    rng = np.random.default_rng(seed)

    def lin(i, o):
        return rng.uniform(-1, 1, (i, o)) / np.sqrt(i)

    sc = 1.0 / (width * width)
    shp = (modes, 2 * modes, 2 * modes, width, width)
    return Params(P=lin(cin, width), p=np.zeros(width), W=[lin(width, width) for _ in range(layers)],
                  w=[np.zeros(width) for _ in range(layers)],
                  R=[sc * (rng.uniform(0, 1, shp) + 1j * rng.uniform(0, 1, shp)) for _ in range(layers)],
                  Q1=lin(width, hidden), q1=np.zeros(hidden), Q2=lin(hidden, cout), q2=np.zeros(cout))


def T(v, Fxy, Fz):
    """(B, N, N, N, C) real -> (B, m, 2m, 2m, C) complex."""
    t = np.einsum("kz,bzyxc->bkyxc", Fz, v)
    t = np.einsum("jy,bkyxc->bkjxc", Fxy, t)
    return np.einsum("ix,bkjxc->bkjic", Fxy, t)


def S(W, Fxy, Fz, cz, n):
    """(B, m, 2m, 2m, C) complex -> (B, N, N, N, C) real."""
    t = np.einsum("ix,bkjic->bkjxc", np.conj(Fxy), W)
    t = np.einsum("jy,bkjxc->bkyxc", np.conj(Fxy), t)
    t = np.einsum("kz,bkyxc->bzyxc", cz[:, None] * np.conj(Fz), t)
    return np.real(t) / n**3


def forward(prm: Params, a: np.ndarray, keep: bool = False):
    n = a.shape[1]
    m = prm.R[0].shape[0]
    Fxy, Fz, cz = dft_matrices(n, m)
    L = len(prm.W)
    v = a @ prm.P + prm.p
    cache = {"a": a, "v": [], "pre": [], "V": []}
    for l in range(L):
        V = T(v, Fxy, Fz)
        k = S(np.einsum("bkjic,kjico->bkjio", V, prm.R[l]), Fxy, Fz, cz, n)
        pre = v @ prm.W[l] + prm.w[l] + k
        cache["v"].append(v)
        cache["V"].append(V)
        cache["pre"].append(pre)
        v = gelu(pre) if l < L - 1 else pre
    hp = v @ prm.Q1 + prm.q1
    h = gelu(hp)
    u = h @ prm.Q2 + prm.q2
    cache.update(vL=v, hp=hp, h=h)
    return (u, cache) if keep else u


def backward(prm: Params, cache, du: np.ndarray) -> Params:
    """Gradient of a scalar loss with dL/du = du, for every parameter (same layout as Params)."""
    a = cache["a"]
    n = a.shape[1]
    m = prm.R[0].shape[0]
    Fxy, Fz, cz = dft_matrices(n, m)
    L = len(prm.W)
    red = tuple(range(a.ndim - 1))
    g = {}
    g["Q2"] = np.tensordot(cache["h"], du, axes=(red, red))
    g["q2"] = du.sum(axis=red)
    dhp = (du @ prm.Q2.T) * gelu_grad(cache["hp"])
    g["Q1"] = np.tensordot(cache["vL"], dhp, axes=(red, red))
    g["q1"] = dhp.sum(axis=red)
    dv = dhp @ prm.Q1.T
    gW, gw, gR = [None] * L, [None] * L, [None] * L
    for l in reversed(range(L)):
        dpre = dv * gelu_grad(cache["pre"][l]) if l < L - 1 else dv
        v, V = cache["v"][l], cache["V"][l]
        gW[l] = np.tensordot(v, dpre, axes=(red, red))
        gw[l] = dpre.sum(axis=red)
        # adjoint of S: a forward transform of the real dpre with the weights c_kz, scaled by N^-3
        dWm = T(dpre, Fxy, Fz) * cz[None, :, None, None, None] / n**3
        gR[l] = np.einsum("bkjio,bkjic->kjico", dWm, np.conj(V))
        dV = np.einsum("kjico,bkjio->bkjic", np.conj(prm.R[l]), dWm)
        # adjoint of T (real input): real part of the conjugate-transposed transform
        t = np.einsum("ix,bkjic->bkjxc", np.conj(Fxy), dV)
        t = np.einsum("jy,bkjxc->bkyxc", np.conj(Fxy), t)
        t = np.einsum("kz,bkyxc->bzyxc", np.conj(Fz), t)
        dv = dpre @ prm.W[l].T + np.real(t)
    gP = np.tensordot(a, dv, axes=(red, red))
    gp = dv.sum(axis=red)
    return Params(P=gP, p=gp, W=gW, w=gw, R=gR, Q1=g["Q1"], q1=g["q1"], Q2=g["Q2"], q2=g["q2"])


def rel_l2_loss(u, target):
    """Mean over the batch of ||u - t|| / ||t|| (per sample), and its gradient."""
    B = u.shape[0]
    d = (u - target).reshape(B, -1)
    t = target.reshape(B, -1)
    nd = np.linalg.norm(d, axis=1)
    nt = np.linalg.norm(t, axis=1)
    loss = float(np.mean(nd / nt))
    grad = (d / (nd * nt)[:, None] / B).reshape(u.shape)
    return loss, grad
