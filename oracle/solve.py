"""The full forward model: incident field, IE solve, receiver fields (eqs. 3-4, 8). FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For every transmitter: E^(0) on the cell centres, solve (I - G dsigma) E = E^(0) either on the whole
domain (GMRES, or dense LU on tiny grids) or by Algorithm 1 (``dd.py``), then the total magnetic
field at each receiver H = H^(0) + H^s (eq. 4). Outputs are (n_src, n_rx, 3) complex.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import physics
from .dd import DDInfo, dd_solve, full_relative_residual
from .gmres import gmres
from .operator import FFTOperator, apply_contrast, contrast, dense_matrix


def cell_centres(grid) -> np.ndarray:
    """Cell centres as an (n, 3) array in (z, y, x) memory order (x fastest)."""
    x, y, z = grid.centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=-1)


def incident_field_on_grid(grid, src, freq: float, sigma0: float) -> np.ndarray:
    """E^(0) of one dipole on the cell centres, shaped (3, nz, ny, nx)."""
    E = physics.incident_E(cell_centres(grid), src.pos, src.moment, freq, sigma0)
    return E.T.reshape(3, grid.nz, grid.ny, grid.nx).copy()


def receiver_fields(grid, dsig, E, src, receivers, freq: float, sigma0: float) -> np.ndarray:
    """Total H = H^(0) + H^s at the receivers (eq. 4), (n_rx, 3)."""
    J = apply_contrast(dsig, E).reshape(3, -1).T
    Hs = physics.scattered_H(receivers, cell_centres(grid), J, grid.h**3, freq, sigma0)
    H0 = physics.incident_H(receivers, src.pos, src.moment, freq, sigma0)
    return H0 + Hs


@dataclass
class SolveInfo:
    method: str = ""
    gmres_iters: int = 0
    outer_iters: int = 0
    rel_residual: float = 0.0
    dd: list = field(default_factory=list)  # DDInfo per source


def forward(grid, sigma6, sigma0: float, freq: float, sources, receivers, method: str = "gmres",
            tol: float = 1e-6, restart: int = 30, z_split=None, adaptive: bool = True,
            max_inner: int = 2000, max_outer: int = 50, return_E: bool = False):
    """Forward model. ``method``: "lu" (dense, tiny grids), "gmres" (whole domain), "gs" or "jacobi"
    (Algorithm 1 with the sub-domain boundaries ``z_split``)."""
    dsig = contrast(np.asarray(sigma6, dtype=np.float64), sigma0)
    receivers = np.asarray(receivers, dtype=np.float64)
    H = np.zeros((len(sources), len(receivers), 3), dtype=np.complex128)
    info = SolveInfo(method=method)
    Es = []
    full = FFTOperator(dsig, grid.h, freq, sigma0) if method != "lu" else None
    Adense = dense_matrix(dsig, grid.h, freq, sigma0) if method == "lu" else None
    for s, src in enumerate(sources):
        E0 = incident_field_on_grid(grid, src, freq, sigma0)
        if method == "lu":
            E = np.linalg.solve(Adense, E0.ravel()).reshape(E0.shape)
            Ax = (Adense @ E.ravel()).reshape(E0.shape)
            info.rel_residual = max(info.rel_residual,
                                    float(np.linalg.norm(E0 - Ax) / np.linalg.norm(E0)))
        elif method == "gmres":
            # Reading: the whole-domain solve starts from E = E^(0), as Algorithm 1 does.
            E, gi = gmres(full, E0, x0=E0, tol=tol, restart=restart, max_iter=max_inner)
            info.gmres_iters += gi.iterations
            info.rel_residual = max(info.rel_residual, full_relative_residual(full, E0, E))
        else:
            E, di = dd_solve(dsig, E0, z_split, grid.h, freq, sigma0, mode=method, eps=tol,
                             adaptive=adaptive, restart=restart, max_outer=max_outer,
                             max_inner=max_inner, full=full)
            info.dd.append(di)
            info.gmres_iters += di.gmres_total
            info.outer_iters += di.outer_iters
            info.rel_residual = max(info.rel_residual, di.residuals[-1])
        H[s] = receiver_fields(grid, dsig, E, src, receivers, freq, sigma0)
        Es.append(E)
    if return_E:
        return H, info, Es
    return H, info


__all__ = ["forward", "incident_field_on_grid", "receiver_fields", "cell_centres", "SolveInfo",
           "DDInfo"]
