"""Domain decomposition of the IE (Section 2.3, eqs. 11-23, Appendix A, Algorithm 1). FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The domain is split along z into M non-overlapping slabs (the drilling axis of Section 3.3). The
block system A E~ = E~(0) (eqs. 13-15) has diagonal blocks A_ii = I - G^(ii) dsigma^(i) and
off-diagonal blocks A_ij = -G^(ij) dsigma^(j). One outer sweep of Algorithm 1:

  Gauss-Seidel (eq. 21):  b_i = E^(i,0) + sum_{j<i} G^(ij) dsigma^(j) E^(j),k+1
                                        + sum_{j>i} G^(ij) dsigma^(j) E^(j),k
  Jacobi (eq. 23):        b_i = E^(i,0) + sum_{j != i} G^(ij) dsigma^(j) E^(j),k
  then E^(i),k+1 = GMRES(A_ii, b_i, x0 = E^(i),k, tol), tol = e/10 (adaptive, "-A") or fixed ("-F").

Readings:
  * Algorithm 1 never refreshes e inside its loop; e is recomputed on the whole (anomalous) domain
    after every full sweep, by eq. 9.
  * Algorithm 1's Jacobi line sums over all j including j = i; eq. 23 excludes j = i, which is the
    consistent form and the one used.
  * The interaction sum of block i is evaluated as the whole-domain convolution (eq. 10 on the union
    of the sub-domains) of the contrast current with block i's own current set to zero, restricted
    to block i. This is the definition of sum_{j != i} G^(ij) dsigma^(j) E^(j) written out.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .gmres import gmres
from .operator import FFTOperator, apply_contrast


@dataclass
class DDInfo:
    outer_iters: int = 0
    gmres_iters: list = field(default_factory=list)  # per sweep: list of per-block iteration counts
    residuals: list = field(default_factory=list)  # e before the first sweep and after each sweep
    converged: bool = False

    @property
    def gmres_total(self) -> int:
        return int(sum(sum(s) for s in self.gmres_iters))


def full_relative_residual(full: FFTOperator, E0: np.ndarray, E: np.ndarray) -> float:
    """e = ||E(0) - (I - G dsigma) E|| / ||E(0)|| on the whole domain (eq. 9)."""
    return float(np.linalg.norm(E0 - full(E)) / np.linalg.norm(E0))


def dd_solve(dsig: np.ndarray, E0: np.ndarray, z_split, h: float, freq: float, sigma0: float,
             mode: str = "gs", eps: float = 1e-6, adaptive: bool = True, fixed_tol: float = 1e-6,
             restart: int = 30, max_outer: int = 50, max_inner: int = 600, full: FFTOperator | None = None):
    """Algorithm 1. ``mode`` is "gs" (block Gauss-Seidel) or "jacobi". Returns (E, DDInfo)."""
    assert mode in ("gs", "jacobi")
    full = full if full is not None else FFTOperator(dsig, h, freq, sigma0)
    blocks = [(z_split[i], z_split[i + 1]) for i in range(len(z_split) - 1)]
    A = [FFTOperator(dsig[z0:z1], h, freq, sigma0) for z0, z1 in blocks]
    E = E0.astype(np.complex128).copy()
    info = DDInfo()
    e = full_relative_residual(full, E0, E)
    info.residuals.append(e)
    while e > eps and info.outer_iters < max_outer:
        E_k = E.copy()
        counts = []
        for i, (z0, z1) in enumerate(blocks):
            src = E if mode == "gs" else E_k  # GS: blocks j < i already hold E^(j),k+1
            J = apply_contrast(dsig, src)
            J[:, z0:z1] = 0.0
            b = E0[:, z0:z1] + full.G(J)[:, z0:z1]
            tol = e / 10.0 if adaptive else fixed_tol
            Ei, gi = gmres(A[i], b, x0=E[:, z0:z1], tol=tol, restart=restart, max_iter=max_inner)
            E[:, z0:z1] = Ei
            counts.append(gi.iterations)
        info.gmres_iters.append(counts)
        info.outer_iters += 1
        e = full_relative_residual(full, E0, E)
        info.residuals.append(e)
    info.converged = e <= eps
    return E, info


@dataclass
class FGMRESInfo:
    outer_iters: int = 0  # preconditioner applications (one DD sweep each)
    gmres_iters: list = field(default_factory=list)  # per outer iteration: per-block inner iterations
    residuals: list = field(default_factory=list)  # e at the start and after every restart cycle
    converged: bool = False

    @property
    def gmres_total(self) -> int:
        return int(sum(sum(s) for s in self.gmres_iters))


def dd_sweep_from_zero(dsig, v, blocks, A, full, mode, inner_tol, inner_restart, max_inner):
    """One sweep of Algorithm 1 on A z = v started from z = 0: the block right-hand sides of eq. 21 (GS,
    blocks j < i already updated) or eq. 23 (Jacobi, all other blocks at zero, so only v_i) with v in
    place of E^(0), each block solved by GMRES to the relative tolerance inner_tol."""
    z = np.zeros_like(v)
    counts = []
    for i, (z0, z1) in enumerate(blocks):
        J = apply_contrast(dsig, z if mode == "gs" else np.zeros_like(z))
        J[:, z0:z1] = 0.0
        b = v[:, z0:z1] + full.G(J)[:, z0:z1]
        zi, gi = gmres(A[i], b, x0=None, tol=inner_tol, restart=inner_restart, max_iter=max_inner)
        z[:, z0:z1] = zi
        counts.append(gi.iterations)
    return z, counts


def fgmres_dd(dsig: np.ndarray, E0: np.ndarray, z_split, h: float, freq: float, sigma0: float, mode: str = "gs",
              eps: float = 1e-6, restart: int = 10, inner_tol: float = 0.1, inner_restart: int = 30,
              max_inner: int = 600, max_outer: int = 50, full: FFTOperator | None = None):
    """Flexible GMRES on the whole-domain system (I - G dsigma) E = E^(0) (eq. 8), right-preconditioned by
    one sweep of Algorithm 1 (the Krylov outer iteration the paper's conclusion proposes in place of the
    fixed-point sweeps). Starts from E = E^(0); the Arnoldi basis is orthogonalised by modified
    Gram-Schmidt and the small least-squares problem is solved directly at every step."""
    assert mode in ("gs", "jacobi")
    full = full if full is not None else FFTOperator(dsig, h, freq, sigma0)
    blocks = [(z_split[i], z_split[i + 1]) for i in range(len(z_split) - 1)]
    A = [FFTOperator(dsig[z0:z1], h, freq, sigma0) for z0, z1 in blocks]
    x = E0.astype(np.complex128).copy()
    n0 = np.linalg.norm(E0)
    r = E0 - full(x)
    info = FGMRESInfo()
    e = float(np.linalg.norm(r) / n0)
    info.residuals.append(e)
    while e > eps and info.outer_iters < max_outer:
        beta = np.linalg.norm(r)
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        y = np.zeros(0)
        for j in range(restart):
            z, counts = dd_sweep_from_zero(dsig, V[j], blocks, A, full, mode, inner_tol, inner_restart, max_inner)
            info.gmres_iters.append(counts)
            info.outer_iters += 1
            Z.append(z)
            w = full(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            g = np.zeros(j + 2, dtype=np.complex128)
            g[0] = beta
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], g, rcond=None)
            res = np.linalg.norm(g - H[: j + 2, : j + 1] @ y)
            if H[j + 1, j] == 0 or res / n0 <= eps or info.outer_iters >= max_outer:
                break
            V.append(w / H[j + 1, j])
        for k in range(len(y)):
            x = x + y[k] * Z[k]
        r = E0 - full(x)
        e = float(np.linalg.norm(r) / n0)
        info.residuals.append(e)
    info.converged = e <= eps
    return x, info
