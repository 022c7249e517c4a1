"""Pins for the seeded input generators (Appendix C tensor rotation, grid placement, determinism)."""
import numpy as np

from paper_2306_17537_gb300 import inputs


def test_ti_rotation_invariants():
    rng = np.random.default_rng(0)
    for _ in range(20):
        sh, sv = 10 ** rng.uniform(-2, 1, 2)
        th, ph = rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)
        m = inputs.sigma6_to_matrix(inputs.ti_tensor(sh, sv, th, ph))
        ev = np.sort(np.linalg.eigvalsh(m))
        assert np.allclose(ev, np.sort([sh, sh, sv]), rtol=1e-12)
        n = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        assert np.allclose(m @ n, sv * n, rtol=1e-12, atol=1e-14)  # symmetry axis = layer normal
        assert abs(np.trace(m) - (2 * sh + sv)) < 1e-12 * sh


def test_ti_rotation_unrotated_is_diagonal():
    m = inputs.sigma6_to_matrix(inputs.ti_tensor(0.2, 0.1, 0.0, 1.3))
    assert np.allclose(m, np.diag([0.2, 0.2, 0.1]), atol=1e-15)


def test_grid_puts_tool_on_a_vertex():
    for wl in (inputs.config1(0), inputs.config2(0, scale=8)):
        x, y, z = wl.grid.centres()
        for pts in [wl.receivers] + [np.array([s.pos]) for s in wl.sources]:
            for p in pts:
                d = np.min(np.abs(z - p[2])) + np.min(np.abs(x - p[0])) + np.min(np.abs(y - p[1]))
                assert d >= 0.49 * wl.grid.h


def test_generators_are_seeded_and_physical():
    a, b = inputs.config2(3, scale=8), inputs.config2(3, scale=8)
    assert np.array_equal(a.sigma6, b.sigma6)
    assert not np.array_equal(a.sigma6, inputs.config2(4, scale=8).sigma6)
    m = inputs.sigma6_to_matrix(a.sigma6)
    assert np.all(np.linalg.eigvalsh(m) > 0)
    c1 = inputs.config1(0)
    assert c1.sigma6.shape == (16, 16, 16, 6) and np.all(c1.sigma6[..., 3:] == 0)
    assert np.all((c1.sigma6[..., 0] >= 0.01) & (c1.sigma6[..., 0] <= 10))


def test_isolated_blocks_layout():
    # Section 3.1: two anomalous slabs of 7.5 m (30 cells of 0.25 m) 10 m (40 cells) apart, 30 x 30 m wide
    wl = inputs.isolated_blocks(128)
    d = wl.sigma6.copy()
    d[..., :3] -= wl.sigma0
    planes = np.array([np.any(d[z] != 0) for z in range(128)])
    zs = wl.z_split
    assert zs == [0, 14, 44, 84, 114, 128]
    assert planes[zs[1]:zs[2]].all() and planes[zs[3]:zs[4]].all()
    assert not planes[:zs[1]].any() and not planes[zs[2]:zs[3]].any() and not planes[zs[4]:].any()
    assert np.count_nonzero(d[zs[1], :, :, 0]) == 120 * 120
    assert np.allclose(d[d != 0], 0.01 - 0.1)


def test_paper_logging_geometry():
    # Section 3.3: the well runs from (0,0,0) to (900,0,78.74) m, i.e. 85 deg from vertical; window 1 is
    # 128x128x256 cells of 0.25 m split in two, window 2 256^3 split in eight; receivers 7, 15, 30 m ahead
    wl = inputs.paper_logging_item(0, 64, 1)
    assert (wl.grid.nx, wl.grid.ny, wl.grid.nz) == (128, 128, 256) and wl.z_split == [0, 128, 256]
    assert np.allclose(wl.receivers[:, 2], [7.0, 15.0, 30.0]) and wl.freq == 2.4e4 and wl.tol == 1e-3
    w2 = inputs.paper_logging_item(0, 64, 2, scale=8)
    assert len(w2.z_split) == 9
    end = np.array([900.0, 0.0, 78.74])
    assert abs(np.degrees(np.arccos(end[2] / np.linalg.norm(end))) - 85.0) < 0.01
    # the sand perturbation peaks at r_c with factor 1 + alpha
    f = inputs.paper_logging_formation()
    assert np.allclose(f.r_c, [500.0, 0.0, 40.0]) and f.alpha == 4.0 and f.gamma == 50.0
