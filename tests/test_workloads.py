"""CPU checks of the seeded input generators: the sizes of the synthetic
workloads, their determinism, a brute-force 2:1 balance check on the finest
grid, and admissible initial states (positive density and pressure)."""
import numpy as np
import pytest

from paper_2607_06045_b300 import workloads as W


def level_map(m):
    """Level of the leaf covering each cell of the finest grid."""
    L = int(m.level.max())
    lm = -np.ones((m.nx0 << L, m.ny0 << L), dtype=np.int64)
    for lev, ix, iy in zip(m.level, m.ix, m.iy):
        f = 1 << (L - int(lev))
        cell = lm[ix * f:(ix + 1) * f, iy * f:(iy + 1) * f]
        assert (cell == -1).all(), "leaves overlap"
        cell[...] = lev
    assert (lm >= 0).all(), "leaves leave a gap"
    return lm


def assert_balanced(m):
    lm = level_map(m)
    dx = np.abs(np.diff(lm, axis=0))
    dy = np.abs(np.diff(lm, axis=1))
    assert dx.max(initial=0) <= 1 and dy.max(initial=0) <= 1
    px, py = m.periodic()
    if px:
        assert np.abs(lm[0] - lm[-1]).max() <= 1
    if py:
        assert np.abs(lm[:, 0] - lm[:, -1]).max() <= 1


def pressure(u, gamma=1.4):
    return (gamma - 1) * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0])


def test_refined_square():
    m = W.square_mesh()
    assert m.n_elems == 304 and m.nx0 == m.ny0 == 16
    assert_balanced(m)
    u = W.disc_wave_state(m, 3)
    assert u.shape == (4, 304, 4, 4)
    assert u[0].min() > 0 and pressure(u).min() > 0
    assert u[0].max() == pytest.approx(2.0)   # the disc


def test_dmr_mesh_size_and_states():
    m = W.dmr_mesh()
    assert m.n_elems == 60139 and 54000 <= m.n_elems <= 66000
    assert (m.nx0, m.ny0) == (256, 64) and int(m.level.max()) == 3
    assert_balanced(m)
    assert (W.dmr_mesh().level == m.level).all()   # seeded
    u = W.dmr_state(m, 3)
    rho = np.unique(np.round(u[0], 12))
    assert set(rho) == {1.4, 8.0}
    p = pressure(u)
    assert np.isclose(p[u[0] == 8.0], 116.5).all() and np.isclose(p[u[0] == 1.4], 1.0).all()


def test_dmr_sample_mesh():
    m = W.dmr_sample_mesh()
    assert 3400 <= m.n_elems <= 4100 and (m.nx0, m.ny0) == (64, 16)
    assert_balanced(m)


def test_batch_meshes():
    ms = W.batch_meshes(256, seed=0)
    assert len(ms) == 256 and sum(m.n_elems for m in ms) == 1806581
    sides = [m.nx0 for m in ms]
    assert 8 <= min(sides) and max(sides) <= 128
    for m in ms[::37]:
        assert_balanced(m)
    again = W.batch_meshes(256, seed=0)
    assert all((a.level == b.level).all() and a.nx0 == b.nx0 for a, b in zip(ms, again))
    other = W.batch_meshes(256, seed=1)
    assert sum(m.n_elems for m in other) != 1806581
    rng = np.random.default_rng(1)
    u = W.riemann4_state(ms[0], 3, rng)
    assert u[0].min() >= 0.1 - 1e-12 and u[0].max() <= 10 + 1e-12
    assert pressure(u).min() >= 0.1 * (1 - 1e-12)


def test_blast_mesh_and_state():
    m, c = W.blast_mesh()
    assert m.n_elems == 386035 and (m.nx0, m.ny0) == (512, 512)
    assert 0.3 <= c[0] <= 0.7 and 0.3 <= c[1] <= 0.7
    small, c2 = W.blast_mesh(n0=64)
    assert_balanced(small)
    u = W.blast_state(small, 5, c2)
    assert u[0].min() == pytest.approx(1e-6) and u[0].max() == pytest.approx(1.0)
    p = pressure(u)
    assert p.min() == pytest.approx(1e-9, rel=1e-6) and p.max() == pytest.approx(1e3, rel=1e-12)


def test_jet_mesh_and_state():
    m = W.jet_mesh()
    assert m.n_elems == 53632 and (m.nx0, m.ny0) == (64, 64)
    assert_balanced(m)
    u = W.jet_state(m, 3, W.JET_GAMMA, seed=3)
    assert u[0].min() > 0 and pressure(u, W.JET_GAMMA).min() > 0
