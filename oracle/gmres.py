"""Restarted GMRES (Saad & Schultz 1986), as used for every linear solve in the paper (Section 2.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Stopping rule: the relative residual of eq. 9, ||b - A x|| / ||b||. Reading: the paper ran MATLAB's
gmres, which measures the residual relative to ||b|| (not to ||b - A x0||); restart length is a
parameter (10 in Section 3.1). Arnoldi uses modified Gram-Schmidt and the small least-squares
problem is solved with Givens rotations, all in FP64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class GmresInfo:
    iterations: int = 0  # Arnoldi steps (= operator applications inside the Krylov loop)
    rel_residual: float = 0.0  # true ||b - A x|| / ||b|| at exit
    converged: bool = False
    history: list = field(default_factory=list)  # residual estimate after every Arnoldi step


def gmres(A, b: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-6, restart: int = 30,
          max_iter: int = 1000):
    """Solve A x = b. ``A`` is a callable on arrays shaped like ``b``."""
    shape = b.shape
    bv = b.ravel()
    nb = np.linalg.norm(bv)
    x = np.zeros_like(bv) if x0 is None else x0.ravel().astype(np.complex128).copy()
    info = GmresInfo()
    if nb == 0.0:
        return np.zeros(shape, dtype=np.complex128), GmresInfo(0, 0.0, True, [])

    def Av(v):
        return A(v.reshape(shape)).ravel()

    r = bv - Av(x) if x0 is not None else bv.copy()
    beta = np.linalg.norm(r)
    info.rel_residual = beta / nb
    if info.rel_residual <= tol:
        info.converged = True
        return x.reshape(shape), info
    while info.iterations < max_iter:
        m = restart
        V = np.zeros((m + 1, bv.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        j_done = 0
        for j in range(m):
            w = Av(V[j])
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # apply previous rotations to the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            # New rotation [[cs, sn], [-conj(sn), conj(cs)]] mapping (a, c) to (|(a, c)|, 0).
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = np.conj(a) / den if den != 0 else 1.0
            sn[j] = np.conj(c) / den if den != 0 else 0.0
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            info.iterations += 1
            j_done = j + 1
            est = abs(g[j + 1]) / nb
            info.history.append(est)
            if est <= tol or breakdown or info.iterations >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        r = bv - Av(x)
        beta = np.linalg.norm(r)
        info.rel_residual = beta / nb
        if info.rel_residual <= tol:
            info.converged = True
            break
    return x.reshape(shape), info
