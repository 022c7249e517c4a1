"""Direct physical pins of the oracle's off-diagonal weight dv * G^E(d h) (Section 2.2 discretisation).

The other operator pins (FFT vs direct sum vs dense matrix) all call ``kernel_at_offsets``, so they
cannot see a wrong weight. These checks use static lattice sums whose values follow from number
theory and symmetry alone, not from the kernel code:

* a single-layer square plate of M x M cells (static limit k0 -> 0): for the centre cell,
  sum_j K_zz(i - j) = -1/(3 sigma0) - S/(4 pi sigma0) and K_xx = K_yy = -1/(3 sigma0) + S/(8 pi sigma0),
  where S = sum over the square lattice points (a, b) != 0 with |a|, |b| <= M/2 of 1/(a^2 + b^2)^{3/2}
  = 4 zeta(3/2) beta(3/2) - 4 sqrt(2)/(M/2 + 1/2) + O(M^-3) (Riemann zeta, Dirichlet beta, and the
  integral of r^-3 outside the square). A wrong cell volume, a missing factor or a flipped sign of
  the R_hat R_hat term changes these sums by O(1).
* a cube (static limit): by cubic symmetry the dipole kernel sums to zero over the cube around its
  centre cell, and its volume average is isotropic and traceless, so both the centre-cell sum and the
  cell-averaged sum equal the static self term -I/(3 sigma0) (the textbook depolarisation 1/3).
"""
import numpy as np
import pytest
from scipy.special import zeta

from oracle import operator as oop

H, S0, F_STATIC = 0.5, 0.2, 1e-6  # at 1 uHz |k0 h| ~ 1e-7: the static limit to ~1e-12


def lattice_constant():
    """sum over (a, b) != 0 of (a^2 + b^2)^{-3/2} on the square lattice = 4 zeta(3/2) beta(3/2)."""
    s = 1.5
    beta = 4.0**(-s) * (zeta(s, 0.25) - zeta(s, 0.75))  # Dirichlet beta from Hurwitz zeta
    return 4.0 * zeta(s, 1.0) * beta


@pytest.mark.parametrize("half", [30, 60])
def test_plate_lattice_sum(half):
    a = np.arange(-half, half + 1)
    dy, dx = np.meshgrid(a, a, indexing="ij")
    K = oop.kernel_at_offsets(np.zeros_like(dx), dy, dx, H, F_STATIC, S0)
    tot = K.reshape(-1, 3, 3).sum(axis=0)
    S = lattice_constant() - 4.0 * np.sqrt(2.0) / (half + 0.5)
    zz = -1.0 / (3 * S0) - S / (4 * np.pi * S0)
    xx = -1.0 / (3 * S0) + S / (8 * np.pi * S0)
    assert abs(tot[2, 2] - zz) <= 2e-5 * abs(zz)
    assert abs(tot[0, 0] - xx) <= 2e-4 * abs(xx)
    assert abs(tot[1, 1] - tot[0, 0]) <= 1e-12 * abs(xx)
    off = tot - np.diag(np.diag(tot))
    assert np.max(np.abs(off)) <= 1e-12 * abs(zz)


def test_plate_sum_scales_with_cell_volume():
    # dv G^E(d h) is scale-free in the static limit: the same lattice sum for any cell size
    a = np.arange(-20, 21)
    dy, dx = np.meshgrid(a, a, indexing="ij")
    t1 = oop.kernel_at_offsets(np.zeros_like(dx), dy, dx, 0.25, F_STATIC, S0).reshape(-1, 3, 3).sum(0)
    t2 = oop.kernel_at_offsets(np.zeros_like(dx), dy, dx, 2.0, F_STATIC, S0).reshape(-1, 3, 3).sum(0)
    assert np.max(np.abs(t1 - t2)) <= 1e-8 * np.max(np.abs(t1))


@pytest.mark.parametrize("n", [5, 7])
def test_cube_depolarisation(n):
    iz, iy, ix = [v.ravel() for v in np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")]
    K = oop.kernel_at_offsets(iz[:, None] - iz[None, :], iy[:, None] - iy[None, :], ix[:, None] - ix[None, :],
                              H, F_STATIC, S0)  # (n^3, n^3, 3, 3)
    per_cell = K.sum(axis=1)
    target = -np.eye(3) / (3 * S0)
    centre = (n // 2) * (n * n + n + 1)
    assert np.max(np.abs(per_cell[centre] - target)) <= 1e-9 / S0
    assert np.max(np.abs(per_cell.mean(axis=0) - target)) <= 1e-9 / S0
    # away from the centre the sum is not isotropic (the body's shape acts), but its trace is
    # always that of the self term: the dipole kernel is traceless
    tr = np.trace(per_cell, axis1=1, axis2=2)
    assert np.max(np.abs(tr + 1.0 / S0)) <= 1e-9 / S0
    assert np.max(np.abs(per_cell[0] - target)) > 1e-2 / S0
