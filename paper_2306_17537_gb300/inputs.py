"""Seeded synthetic earth models and tool layouts (shared by the oracle, the tests and the bench).

This module only *describes inputs*: voxel grids, absolute conductivity tensors, magnetic-dipole
sources and receiver positions. It contains none of the integral-equation arithmetic (no Green's
functions, no operator, no solver), so the CPU oracle and the CUDA path can both consume it
without sharing any of the method's code.

Conventions (stated once, used everywhere):
  * A grid is ``(nx, ny, nz, h, origin)``; ``origin`` is the minimum corner, cell centres sit at
    ``origin + (i + 1/2) h`` and x varies fastest in memory (Section 2.2 of the paper: uniform
    grid blocks with centroids r^j and volume h^3).
  * The tool origin (0, 0, 0) is placed on a cell *vertex* so that transmitters and receivers at
    multiples of h never coincide with a cell centre (where the scalar Green's function is
    singular).
  * Conductivity is the absolute tensor sigma (not the contrast), stored per voxel as the six
    unique components ``(xx, yy, zz, xy, xz, yz)`` of the symmetric 3x3 tensor (Appendix C), array
    shape ``(nz, ny, nx, 6)``, float64.
  * Transversely isotropic layers are rotated into the tool frame by Appendix C: with the layer
    normal n = (sin t cos p, sin t sin p, cos t) the rotated tensor is
    ``sigma_h I + (sigma_v - sigma_h) n n^T``.

The paper's own formations exist only in figures that are not available, so every workload here
is a seeded stand-in with the shapes and value ranges of the paper's examples (Section 3).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

COMPONENTS6 = ("xx", "yy", "zz", "xy", "xz", "yz")


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    h: float
    origin: tuple  # (x0, y0, z0): minimum corner of the voxel grid, metres

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def centres(self):
        """Cell-centre coordinates as three 1-D arrays (x, y, z)."""
        x = self.origin[0] + (np.arange(self.nx) + 0.5) * self.h
        y = self.origin[1] + (np.arange(self.ny) + 0.5) * self.h
        z = self.origin[2] + (np.arange(self.nz) + 0.5) * self.h
        return x, y, z


@dataclass
class Dipole:
    pos: tuple
    moment: tuple  # magnetic moment, A m^2


@dataclass
class Workload:
    name: str
    grid: Grid
    sigma0: float  # background conductivity, S/m
    freq: float  # Hz
    sigma6: np.ndarray  # (nz, ny, nx, 6) absolute conductivity
    sources: list
    receivers: np.ndarray  # (n_rx, 3)
    z_split: list = field(default_factory=list)  # sub-domain boundaries along z (voxel index)
    tol: float = 1e-6
    restart: int = 30


def centred_grid(nx: int, ny: int, nz: int, h: float) -> Grid:
    """A grid whose centre is the tool origin (0,0,0), which then lies on a cell vertex (even n)."""
    return Grid(nx, ny, nz, h, (-nx * h / 2.0, -ny * h / 2.0, -nz * h / 2.0))


def ti_tensor(sigma_h, sigma_v, theta, phi):
    """Transversely isotropic conductivity rotated into the tool frame (Appendix C).

    Returns the six components (xx, yy, zz, xy, xz, yz) with a trailing axis of length 6.
    """
    sigma_h = np.asarray(sigma_h, dtype=np.float64)
    sigma_v = np.asarray(sigma_v, dtype=np.float64)
    nvec = (np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta))
    d = sigma_v - sigma_h
    out = np.empty(np.broadcast(sigma_h, sigma_v).shape + (6,))
    out[..., 0] = sigma_h + d * nvec[0] * nvec[0]
    out[..., 1] = sigma_h + d * nvec[1] * nvec[1]
    out[..., 2] = sigma_h + d * nvec[2] * nvec[2]
    out[..., 3] = d * nvec[0] * nvec[1]
    out[..., 4] = d * nvec[0] * nvec[2]
    out[..., 5] = d * nvec[1] * nvec[2]
    return out


def sigma6_to_matrix(s6: np.ndarray) -> np.ndarray:
    """(…, 6) -> (…, 3, 3) symmetric tensor."""
    m = np.empty(s6.shape[:-1] + (3, 3), dtype=s6.dtype)
    m[..., 0, 0] = s6[..., 0]
    m[..., 1, 1] = s6[..., 1]
    m[..., 2, 2] = s6[..., 2]
    m[..., 0, 1] = m[..., 1, 0] = s6[..., 3]
    m[..., 0, 2] = m[..., 2, 0] = s6[..., 4]
    m[..., 1, 2] = m[..., 2, 1] = s6[..., 5]
    return m


def _log_uniform(rng, lo_exp, hi_exp, size=None):
    return 10.0 ** rng.uniform(lo_exp, hi_exp, size)


def _random_rotation(rng) -> np.ndarray:
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def layered_vti(grid: Grid, seed: int, n_layers: int = 3, ratio_max: float = 5.0) -> np.ndarray:
    """Horizontal VTI layers: interfaces at sorted seeded uniform z inside the grid's z-extent,
    sigma_h log-uniform in [0.01, 10] S/m, anisotropy ratio r ~ U(1, ratio_max), sigma_v = sigma_h / r.
    """
    rng = np.random.default_rng(seed)
    z0 = grid.origin[2]
    z1 = z0 + grid.nz * grid.h
    iface = np.sort(rng.uniform(z0, z1, n_layers - 1))
    sh = _log_uniform(rng, -2.0, 1.0, n_layers)
    ratio = rng.uniform(1.0, ratio_max, n_layers)
    sv = sh / ratio
    _, _, zc = grid.centres()
    layer = np.searchsorted(iface, zc)  # (nz,)
    s6 = np.zeros((grid.nz, grid.ny, grid.nx, 6))
    s6[..., 0] = sh[layer][:, None, None]
    s6[..., 1] = sh[layer][:, None, None]
    s6[..., 2] = sv[layer][:, None, None]
    return s6


def dipping_ti_with_ellipsoids(grid: Grid, seed: int, n_layers: int = 5, ratio_max: float = 10.0,
                               dip_max_deg: float = 30.0, n_ellipsoids: int = 2, eval_grid: Grid | None = None) -> np.ndarray:
    """Dipping TI layers (common dip/azimuth, Appendix C rotation) plus isotropic ellipsoids.

    The model is drawn for ``grid``; ``eval_grid`` (default ``grid``) is where it is evaluated, so a
    sub-grid of ``grid`` gives exactly the corresponding crop of the full model."""
    rng = np.random.default_rng(seed)
    theta = np.deg2rad(rng.uniform(0.0, dip_max_deg))
    phi = rng.uniform(0.0, 2.0 * np.pi)
    nrm = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    xc, yc, zc = (eval_grid or grid).centres()
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    dist = X * nrm[0] + Y * nrm[1] + Z * nrm[2]
    half = 0.5 * grid.h * np.array([grid.nx, grid.ny, grid.nz])
    reach = float(np.abs(nrm) @ half)
    iface = np.sort(rng.uniform(-0.8 * reach, 0.8 * reach, n_layers - 1))
    sh = _log_uniform(rng, -2.0, 1.0, n_layers)
    ratio = rng.uniform(1.0, ratio_max, n_layers)
    sv = sh / ratio
    layer = np.searchsorted(iface, dist)
    s6 = ti_tensor(sh[layer], sv[layer], theta, phi)
    lo = np.array(grid.origin)
    ext = grid.h * np.array([grid.nx, grid.ny, grid.nz])
    for _ in range(n_ellipsoids):
        c = lo + ext * rng.uniform(0.1, 0.9, 3)
        ax = rng.uniform(1.0, 4.0, 3)
        rot = _random_rotation(rng)
        sig = _log_uniform(rng, -2.0, 1.0)
        d = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1) @ rot  # body-frame coordinates
        inside = np.sum((d / ax) ** 2, axis=-1) <= 1.0
        s6[inside, :3] = sig
        s6[inside, 3:] = 0.0
    return s6


def coaxial_tool(spacings=(0.5, 1.0, 2.0)):
    """z-directed unit magnetic dipole at the origin, receivers on the tool (z) axis."""
    src = [Dipole((0.0, 0.0, 0.0), (0.0, 0.0, 1.0))]
    rx = np.array([[0.0, 0.0, s] for s in spacings], dtype=np.float64)
    return src, rx


def config1(seed: int = 0) -> Workload:
    """Plain full-domain IE: 16^3 voxels of 0.5 m, 3 horizontal VTI layers (ratio 1-5),
    coaxial z-dipole with receivers at 0.5/1/2 m, f = 100 kHz, sigma0 = 0.1 S/m, GMRES(30), tol 1e-8."""
    g = centred_grid(16, 16, 16, 0.5)
    src, rx = coaxial_tool()
    return Workload("full-domain IE 16x16x16 @0.5 m, 3 VTI layers, 100 kHz", g, 0.1, 1.0e5,
                    layered_vti(g, seed), src, rx, z_split=[0, 16], tol=1e-8, restart=30)


def config2(seed: int = 0, scale: int = 1) -> Workload:
    """Plain DD: 128x128x256 voxels of 0.25 m split into 2 sub-domains along z, 5 dipping TI layers
    (ratio 1-10) plus 2 isotropic ellipsoids, coaxial z-dipole at the domain centre, f = 400 kHz,
    sigma0 = 0.1 S/m, block Gauss-Seidel with adaptive tolerance, tol 1e-6.

    ``scale`` > 1 divides every grid dimension (same physical cell size), giving the same kind of
    model on a smaller box for tests.
    """
    nx, ny, nz = 128 // scale, 128 // scale, 256 // scale
    g = centred_grid(nx, ny, nz, 0.25)
    src, rx = coaxial_tool()
    name = f"DD {nx}x{ny}x{nz} @0.25 m, 2 blocks GS-A, 5 dipping TI layers + 2 ellipsoids, 400 kHz"
    # restart 40: the fastest of a measured sweep over 8..80 on this workload (fewer, longer cycles)
    return Workload(name, g, 0.1, 4.0e5, dipping_ti_with_ellipsoids(g, seed), src, rx,
                    z_split=[0, nz // 2, nz], tol=1e-6, restart=40)


def faulted_ti_with_ellipsoids(grid: Grid, seed: int, n_layers: int = 7, ratio_max: float = 10.0,
                               dip_max_deg: float = 30.0, n_ellipsoids: int = 5) -> np.ndarray:
    """Dipping TI layers offset by a planar fault, plus isotropic ellipsoids (the large configuration).

    The layer stack has a common seeded dip theta ~ U(0, 30) deg and azimuth phi, per layer
    sigma_h = 10^U(-1.5, 0.3) S/m (0.03 - 2 S/m, the range of the logging formation of Section 3.3) and
    anisotropy ratio r ~ U(1, 10) with sigma_v = sigma_h / r, rotated into the tool frame by Appendix C.
    A fault plane (dip U(50, 80) deg, random strike, through a point in the inner half of the grid)
    offsets the stack: on its hanging-wall side the layers are displaced vertically by a throw U(2, 8) m.
    Ellipsoids: centres uniform in the inner 80 %, semi-axes U(1, 4) m, random orientation, isotropic
    sigma = 10^U(-2, 0.3) S/m. (At 2 MHz a 10 S/m layer has a skin depth of 0.11 m, under half a
    0.25 m cell: the conductivities stop at 2 S/m, where it is 0.25 m.)
    """
    rng = np.random.default_rng(seed)
    theta = np.deg2rad(rng.uniform(0.0, dip_max_deg))
    phi = rng.uniform(0.0, 2.0 * np.pi)
    nrm = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    half = 0.5 * grid.h * np.array([grid.nx, grid.ny, grid.nz])
    reach = float(np.abs(nrm) @ half)
    iface = np.sort(rng.uniform(-0.8 * reach, 0.8 * reach, n_layers - 1))
    sh = _log_uniform(rng, -1.5, 0.3, n_layers)
    sv = sh / rng.uniform(1.0, ratio_max, n_layers)
    fdip, fstrike = np.deg2rad(rng.uniform(50.0, 80.0)), rng.uniform(0.0, 2.0 * np.pi)
    fnrm = np.array([np.sin(fdip) * np.cos(fstrike), np.sin(fdip) * np.sin(fstrike), np.cos(fdip)])
    lo = np.array(grid.origin)
    ext = grid.h * np.array([grid.nx, grid.ny, grid.nz])
    fpt = lo + ext * rng.uniform(0.25, 0.75, 3)
    throw = rng.uniform(2.0, 8.0)
    xc, yc, zc = grid.centres()
    X, Y, Z = xc[None, None, :], yc[None, :, None], zc[:, None, None]
    hanging = ((X - fpt[0]) * fnrm[0] + (Y - fpt[1]) * fnrm[1] + (Z - fpt[2]) * fnrm[2]) > 0.0
    dist = X * nrm[0] + Y * nrm[1] + Z * nrm[2] - np.where(hanging, throw * nrm[2], 0.0)
    layer = np.searchsorted(iface, dist)
    del dist, hanging
    s6 = ti_tensor(sh[layer], sv[layer], theta, phi)
    del layer
    for _ in range(n_ellipsoids):
        c = lo + ext * rng.uniform(0.1, 0.9, 3)
        ax = rng.uniform(1.0, 4.0, 3)
        rot = _random_rotation(rng)
        sig = _log_uniform(rng, -2.0, 0.3)
        # only the bounding box of the ellipsoid is evaluated
        i0 = [max(0, int(np.floor((c[a] - ax.max() - lo[a]) / grid.h))) for a in range(3)]
        i1 = [min(n, int(np.ceil((c[a] + ax.max() - lo[a]) / grid.h)) + 1)
              for a, n in enumerate((grid.nx, grid.ny, grid.nz))]
        Zb, Yb, Xb = np.meshgrid(zc[i0[2]:i1[2]], yc[i0[1]:i1[1]], xc[i0[0]:i1[0]], indexing="ij")
        d = np.stack([Xb - c[0], Yb - c[1], Zb - c[2]], axis=-1) @ rot  # body-frame coordinates
        inside = np.sum((d / ax) ** 2, axis=-1) <= 1.0
        box = s6[i0[2]:i1[2], i0[1]:i1[1], i0[0]:i1[0]]
        box[inside, :3] = sig
        box[inside, 3:] = 0.0
    return s6


_C5_CACHE: dict = {}


def config5(seed: int = 0, position: int = 0, n_positions: int = 16, scale: int = 1) -> Workload:
    """Large DD: 256x256x512 voxels of 0.25 m (33.5 M cells, 100.7 M complex unknowns) split into 8
    sub-domains of 256x256x64 along z, block Jacobi; 7 dipping TI layers offset by a fault plus 5
    ellipsoids (faulted_ti_with_ellipsoids); coaxial z-dipole tool at one of 16 positions along the z
    axis, 2 m apart and centred on the grid (receivers 0.5/1/2 m above the transmitter); f = 2 MHz,
    sigma0 = 0.1 S/m, tol 1e-6. The model is the same for every position (one set_contrast serves the
    16 solves). ``scale`` > 1 divides every grid dimension and the position spacing (same cell size)."""
    nx, ny, nz = 256 // scale, 256 // scale, 512 // scale
    g = centred_grid(nx, ny, nz, 0.25)
    key = (seed, scale)
    if key not in _C5_CACHE:
        _C5_CACHE.clear()
        _C5_CACHE[key] = faulted_ti_with_ellipsoids(g, seed)
    spacing = 2.0 / scale
    zt = spacing * (position - 0.5 * (n_positions - 1))
    src = [Dipole((0.0, 0.0, zt), (0.0, 0.0, 1.0))]
    rx = np.array([[0.0, 0.0, zt + s] for s in (0.5, 1.0, 2.0)], dtype=np.float64)
    split = [k * (nz // 8) for k in range(9)]
    name = (f"DD {nx}x{ny}x{nz} @0.25 m, 8 blocks Jacobi, 7 faulted TI layers + 5 ellipsoids, "
            f"position {position}/{n_positions}, 2 MHz")
    return Workload(name, g, 0.1, 2.0e6, _C5_CACHE[key], src, rx, z_split=split, tol=1e-6, restart=40)


@dataclass
class Formation:
    """A layered earth model in global coordinates (z up) in the style of the paper's logging example
    (Section 3.3): anisotropic shale layers around isotropic sand layers, a fault offsetting the stack,
    and the exponential perturbation of the sand conductivity
    sigma_sand = sigma_u (1 + alpha exp(-|r - r_c| / gamma))."""
    normal: np.ndarray  # unit layer normal (global)
    interfaces: np.ndarray  # sorted offsets of the layer boundaries along the normal, metres
    sigma_h: np.ndarray
    sigma_v: np.ndarray
    is_sand: np.ndarray
    fault_point: np.ndarray
    fault_normal: np.ndarray
    fault_throw: float  # offset of the layer stack (along the layer normal) across the fault plane
    r_c: np.ndarray  # centre of the sand perturbation
    alpha: float
    gamma: float


def formation(seed: int, n_layers: int = 7, extent: float = 80.0) -> Formation:
    """Seeded logging formation: layers dipping U(0, 30) deg, alternately shale (TI, sigma_h
    10^U(-0.5, 0.3) S/m, anisotropy ratio U(2, 5)) and sand (isotropic 10^U(-2, -1) S/m) with the
    exponential perturbation (alpha = 4, gamma = 50 m, as in Section 3.3), and a planar fault."""
    rng = np.random.default_rng(seed)
    th, ph = np.deg2rad(rng.uniform(0.0, 30.0)), rng.uniform(0.0, 2.0 * np.pi)
    nrm = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    iface = np.sort(rng.uniform(-extent / 4, extent / 4, n_layers - 1))
    sand = (np.arange(n_layers) % 2) == 1
    sh = np.where(sand, 10.0 ** rng.uniform(-2.0, -1.0, n_layers), 10.0 ** rng.uniform(-0.5, 0.3, n_layers))
    sv = np.where(sand, sh, sh / rng.uniform(2.0, 5.0, n_layers))
    fth, fph = np.deg2rad(rng.uniform(50.0, 80.0)), rng.uniform(0.0, 2.0 * np.pi)
    fn = np.array([np.sin(fth) * np.cos(fph), np.sin(fth) * np.sin(fph), np.cos(fth)])
    return Formation(nrm, iface, sh, sv, sand, rng.uniform(-5.0, 5.0, 3), fn, float(rng.uniform(1.0, 4.0)),
                     rng.uniform(-extent / 3, extent / 3, 3), 4.0, 50.0)


def window_sigma6(form: Formation, grid: Grid, tool_pos, rot) -> np.ndarray:
    """Conductivity of ``form`` on a tool-aligned window grid: the columns of ``rot`` are the tool
    axes in global coordinates (tool z along the well), the window origin is relative to ``tool_pos``.
    Layer tensors are rotated into the tool frame by Appendix C using the tool-frame layer normal."""
    xc, yc, zc = grid.centres()
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    loc = np.stack([X, Y, Z], axis=-1)
    glob = np.asarray(tool_pos) + loc @ rot.T
    side = np.sign((glob - form.fault_point) @ form.fault_normal)
    dist = glob @ form.normal + 0.5 * form.fault_throw * side
    layer = np.searchsorted(form.interfaces, dist)
    pert = 1.0 + form.alpha * np.exp(-np.linalg.norm(glob - form.r_c, axis=-1) / form.gamma)
    factor = np.where(form.is_sand[layer], pert, 1.0)
    n_tool = rot.T @ form.normal
    theta = np.arccos(np.clip(n_tool[2], -1.0, 1.0))
    phi = np.arctan2(n_tool[1], n_tool[0])
    return ti_tensor(form.sigma_h[layer] * factor, form.sigma_v[layer] * factor, theta, phi)


def trajectory(seed: int, n_positions: int, spacing: float = 0.5):
    """Seeded deviated well: inclination U(60, 85) deg from vertical, random azimuth; returns tool
    positions and the tool-frame rotation (columns: tool x, y, z axes in global coordinates)."""
    rng = np.random.default_rng(seed + 1000)
    inc, az = np.deg2rad(rng.uniform(60.0, 85.0)), rng.uniform(0.0, 2.0 * np.pi)
    d = np.array([np.sin(inc) * np.cos(az), np.sin(inc) * np.sin(az), np.cos(inc)])
    ex = np.cross([0.0, 0.0, 1.0], d)
    ex /= np.linalg.norm(ex)
    ey = np.cross(d, ex)
    rot = np.stack([ex, ey, d], axis=1)
    start = -0.5 * spacing * (n_positions - 1) * d
    return [start + k * spacing * d for k in range(n_positions)], rot


# Tool-aligned windows of the batched logging workload: (shape (nz, ny, nx), sub-domain split along z)
LOGGING_WINDOWS = {
    2.0e6: ((160, 64, 64), [0, 64, 160]),     # 64^3 + 64x64x96 sub-domains
    1.0e5: ((320, 128, 128), [0, 128, 320]),  # 128^3 + 128x128x192 sub-domains
}


def config3_item(seed: int, position: int, freq: float, n_positions: int = 64, scale: int = 1) -> Workload:
    """One (tool position, frequency) problem of the batched logging workload: a window of the seeded
    formation around position ``position`` of the seeded trajectory, coaxial z-dipole tool, block
    Jacobi over two uneven sub-domains along the tool axis, tol 1e-6. ``scale`` > 1 shrinks the window."""
    (nz, ny, nx), split = LOGGING_WINDOWS[freq]
    nz, ny, nx = nz // scale, ny // scale, nx // scale
    split = [v // scale for v in split]
    g = centred_grid(nx, ny, nz, 0.25)
    pos, rot = trajectory(seed, n_positions)
    s6 = window_sigma6(formation(seed), g, pos[position], rot)
    src, rx = coaxial_tool()
    name = f"logging window {nx}x{ny}x{nz} @0.25 m, position {position}, {freq:g} Hz"
    return Workload(name, g, 0.1, freq, s6, src, rx, z_split=split, tol=1e-6, restart=40)


def paper_logging_formation() -> Formation:
    """The logging formation of Section 3.3 as its text describes it (its figure is not available): a
    2.5-D stack (layer normal in the x-z plane, 3 deg dip) of anisotropic shale layers around isotropic
    sand layers spanning the well's climb from z = 0 to 79 m, offset by a fault near x = 450 m, with the
    sand perturbation sigma_u (1 + alpha exp(-|r - r_c| / gamma)) at r_c = (500, 0, 40) m, alpha = 4,
    gamma = 50 m. Layer conductivities are fixed values in the ranges of that section."""
    dip = np.deg2rad(3.0)
    nrm = np.array([-np.sin(dip), 0.0, np.cos(dip)])
    iface = np.array([-10.0, 6.0, 18.0, 30.0, 44.0, 58.0, 70.0, 86.0])
    sand = np.array([False, True, False, True, False, True, False, True, False])
    sh = np.array([1.2, 0.05, 0.8, 0.03, 1.5, 0.04, 1.0, 0.06, 0.9])
    ratio = np.array([3.0, 1.0, 4.0, 1.0, 2.5, 1.0, 3.5, 1.0, 3.0])
    fault_n = np.array([np.cos(np.deg2rad(70.0)), 0.0, np.sin(np.deg2rad(70.0))])
    return Formation(nrm, iface, sh, sh / ratio, sand, np.array([450.0, 0.0, 40.0]), fault_n, 6.0,
                     np.array([500.0, 0.0, 40.0]), 4.0, 50.0)


PAPER_LOGGING_WINDOWS = {
    1: ((256, 128, 128), [0, 128, 256]),                  # 32 x 32 x 64 m, two sub-domains
    2: ((256, 256, 256), [32 * k for k in range(9)]),     # 64 x 64 x 64 m, eight sub-domains
}


def paper_logging_item(position: int, n_positions: int = 64, window: int = 1, scale: int = 1) -> Workload:
    """One position of the logging simulation of Section 3.3: the well runs at 85 deg from (0, 0, 0) to
    (900, 0, 78.74) m; a tool-aligned window (window 1: 128 x 128 x 256 cells, two sub-domains; window 2:
    256^3 cells, eight) of 0.25 m cells centred on the transmitter; z-directed magnetic dipole at 24 kHz
    with receivers 7, 15 and 30 m ahead on the tool axis; sigma0 = 0.1 S/m; GS-A to e = 1e-3."""
    (nz, ny, nx), split = PAPER_LOGGING_WINDOWS[window]
    nz, ny, nx = nz // scale, ny // scale, nx // scale
    split = [v // scale for v in split]
    g = centred_grid(nx, ny, nz, 0.25)
    end = np.array([900.0, 0.0, 78.74])
    d = end / np.linalg.norm(end)
    ex = np.cross([0.0, 1.0, 0.0], d)
    ex /= np.linalg.norm(ex)
    ey = np.cross(d, ex)
    rot = np.stack([ex, ey, d], axis=1)
    pos = end * (position / max(n_positions - 1, 1))
    s6 = window_sigma6(paper_logging_formation(), g, pos, rot)
    src = [Dipole((0.0, 0.0, 0.0), (0.0, 0.0, 1.0))]
    rx = np.array([[0.0, 0.0, 7.0], [0.0, 0.0, 15.0], [0.0, 0.0, 30.0]])
    name = f"Section 3.3 logging, window {window} ({nx}x{ny}x{nz} @0.25 m), position {position}/{n_positions}, 24 kHz"
    return Workload(name, g, 0.1, 2.4e4, s6, src, rx, z_split=split, tol=1e-3, restart=10)


def isolated_blocks(n: int = 128) -> Workload:
    """The isolated sub-domains model of Section 3.1: an n^3 grid of 0.25 m cells (32 m for n = 128) in a
    0.1 S/m background with two resistive (0.01 S/m) slabs of 30 x 30 x 7.5 m centred on the tool axis,
    10 m apart along z; x-directed magnetic dipole at the origin, 24 kHz. Sub-domains along z: the two
    anomalous slabs and the background around and between them (which the DD sweeps leave out).
    Receivers at the slab centres, in the gap and beside it. ``n`` < 128 shrinks every length by n/128."""
    h = 0.25
    scale = n / 128.0
    g = centred_grid(n, n, n, h)
    s6 = np.zeros((n, n, n, 6))
    s6[..., :3] = 0.1
    half_xy = int(round(60 * scale))   # 30 m lateral extent = 120 cells at full size
    thick = int(round(30 * scale))     # 7.5 m = 30 cells
    gap = int(round(40 * scale))       # 10 m = 40 cells
    z0 = n // 2 - gap // 2 - thick
    z1 = n // 2 + gap // 2
    c = n // 2
    for za in (z0, z1):
        s6[za:za + thick, c - half_xy:c + half_xy, c - half_xy:c + half_xy, :3] = 0.01
    src = [Dipole((0.0, 0.0, 0.0), (1.0, 0.0, 0.0))]
    zc = (z0 + thick / 2 - n / 2) * h
    rx = np.array([[0.0, 0.0, zc], [0.0, 0.0, -zc], [2.0, 0.0, 0.0], [4.0, 1.0, 0.0]])
    split = [0, z0, z0 + thick, z1, z1 + thick, n]
    name = f"isolated sub-domains {n}^3 @{h} m, two 0.01 S/m slabs in 0.1 S/m, 24 kHz x-dipole"
    return Workload(name, g, 0.1, 2.4e4, s6, src, rx, z_split=split, tol=1e-6, restart=10)


def config4_item(seed: int, n: int = 64) -> Workload:
    """One training/evaluation sample of the learned warm start: a model of the 128x128x256 @0.25 m
    dipping-TI-plus-ellipsoids generator (the tool at the centre of the full model, 400 kHz, sigma0
    0.1 S/m) cropped to an n^3 block at a seeded offset, solved as one sub-domain (no receivers).
    The tool may lie inside or outside the block; it always sits on a cell vertex."""
    full = centred_grid(128, 128, 256, 0.25)
    rng = np.random.default_rng([seed, 4])
    off = (int(rng.integers(0, full.nx - n + 1)), int(rng.integers(0, full.ny - n + 1)),
           int(rng.integers(0, full.nz - n + 1)))
    crop = Grid(n, n, n, full.h, tuple(full.origin[k] + off[k] * full.h for k in range(3)))
    src, _ = coaxial_tool()
    s6 = dipping_ti_with_ellipsoids(full, seed, eval_grid=crop)
    name = f"warm-start block {n}^3 @0.25 m cropped at cells {off} of the 128x128x256 model, 400 kHz"
    return Workload(name, crop, 0.1, 4.0e5, s6, src, np.zeros((0, 3)), z_split=[0, n], tol=1e-6, restart=40)


def random_contrast_sigma6(shape, seed: int, sigma0: float, spread: float = 0.5) -> np.ndarray:
    """Random symmetric positive-definite conductivity around sigma0 (for operator parity tests)."""
    rng = np.random.default_rng(seed)
    a = rng.normal(scale=spread, size=tuple(shape) + (3, 3))
    m = sigma0 * (np.eye(3) + 0.5 * (a @ np.swapaxes(a, -1, -2)))
    return np.stack([m[..., 0, 0], m[..., 1, 1], m[..., 2, 2], m[..., 0, 1], m[..., 0, 2],
                     m[..., 1, 2]], axis=-1)


def random_field(n3_shape, seed: int) -> np.ndarray:
    """Random complex field of shape (3, nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=n3_shape) + 1j * rng.normal(size=n3_shape)
