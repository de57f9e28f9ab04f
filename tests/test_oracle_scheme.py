"""Pins of the oracle's whole-scheme behaviour against what the paper fixes.

- Eq. evolutionformula and Eq. fluxdifferencingform give the same residual.
- Free-stream preservation on a nonconforming mesh (high order, low order,
  limited); a wall at rest keeps a uniform state at rest.
- Discrete conservation: sum_i m_i du_i/dt = 0 on periodic meshes, and
  sum_i m_i u_i constant over 100 limited SSP-RK3 steps.
- Metric identities sum_j c_ij = 0 (Eq. metric_identity) and c_ji = -c_ij,
  also across mortars (Remark re:Equivalence_mortarFlux_cdForm).
- The bar-state form (Eq. barstateform) equals the c/d form.
- Under the IDP step restriction (Eq. timestep_restriction) the low-order
  update is a convex combination (Eq. convex_combination): the density stays
  within its bar-state range and pressure stays positive.
- Smooth data far from the bounds: positivity limiting is inactive and the
  limited residual equals the high-order one (Sec. 3.1).
- Local bounds hold after limited stages; mirror and transpose symmetry.
- Mortar fluxes: conservation (Eq. conservationProperty) and consistency.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import rel_err, rhs_scale
from paper_2607_06045_b300 import workloads as W

G = 1.4


@pytest.fixture(scope="module")
def square():
    m = W.square_mesh()
    return m, oracle.Oracle(m, 3), W.disc_wave_state(m, 3)


def euler_flux(u, n):
    rho, m1, m2, E = u
    p = (G - 1) * (E - 0.5 * (m1 * m1 + m2 * m2) / rho)
    vn = (m1 * n[0] + m2 * n[1]) / rho
    return np.array([rho * vn, m1 * vn + p * n[0], m2 * vn + p * n[1], (E + p) * vn])


def test_evolution_equals_flux_differencing(square):
    m, o, u = square
    r1 = o.dg_residual(u)
    r2 = o.dg_residual(u, form="fd")
    assert np.abs(r1 - r2).max() <= 1e-13 * np.abs(r1).max()
    u2 = W.smooth_random_state(m, 3, seed=4)
    r1, r2 = o.dg_residual(u2), o.dg_residual(u2, form="fd")
    assert np.abs(r1 - r2).max() <= 1e-13 * np.abs(r1).max()


def test_free_stream_nonconforming(square):
    m, o, _ = square
    sh = (m.n_elems, 4, 4)
    u = W.conserved(1.3 * np.ones(sh), 0.4 * np.ones(sh), -0.7 * np.ones(sh), 2.0 * np.ones(sh), G)
    mm = o.masses()
    scale = 3.0 / mm.min()
    assert np.abs(o.rhs(u, dt=0.0)).max() < 1e-13 * scale
    assert np.abs(o.fv_residual(u)[0]).max() < 1e-15 * scale * mm.min() * 10
    dt = o.dt(u, cfl=0.5)
    assert np.abs(o.rhs(u, dt=dt, limiting=2)).max() < 1e-13 * scale


def test_wall_at_rest():
    mesh = W.uniform_mesh(4, 3, (0.0, 0.0, 2.0, 1.0), bc=(W.BC_WALL,) * 4)
    o = oracle.Oracle(mesh, 3)
    sh = (mesh.n_elems, 4, 4)
    u = W.conserved(np.ones(sh), np.zeros(sh), np.zeros(sh), np.ones(sh), G)
    assert np.abs(o.rhs(u, dt=0.0)).max() < 1e-12
    dt = o.dt(u, cfl=0.5)
    assert np.abs(o.rhs(u, dt=dt, limiting=2)).max() < 1e-12


def test_dirichlet_free_stream():
    prim = np.array([1.1, 0.3, 0.2, 0.9])
    mesh = W.uniform_mesh(3, 3, (0.0, 0.0, 1.0, 1.0), bc=(W.BC_DIRICHLET,) * 4)
    mesh.bc_prim = np.tile(prim, (4, 1))
    o = oracle.Oracle(mesh, 3)
    sh = (mesh.n_elems, 4, 4)
    u = W.conserved(prim[0] * np.ones(sh), prim[1] * np.ones(sh), prim[2] * np.ones(sh), prim[3] * np.ones(sh), G)
    assert np.abs(o.rhs(u, dt=0.0)).max() < 1e-12


@pytest.mark.parametrize("limiting", [0, 1, 2])
def test_conservation_of_residual(square, limiting):
    m, o, u = square
    mm = o.masses()
    dt = o.dt(u, cfl=0.5)
    r = o.rhs(u, dt=dt if limiting else 0.0, limiting=limiting)
    for v in range(4):
        tot = (mm * r[v]).sum()
        scale = (mm * np.abs(r[v])).sum()
        assert abs(tot) <= 1e-13 * scale, (v, tot, scale)


def test_conservation_100_steps(square):
    m, o, u = square
    I0 = o.integrals(u)
    un, t, dts, st = o.step(u, 100, cfl=0.5, limiting=2)
    I1 = o.integrals(un)
    mm = o.masses()
    for v in range(4):
        scale = (mm * np.abs(u[v])).sum()
        assert abs(I1[v] - I0[v]) <= 1e-13 * scale
    assert st["viol_rho"] == 0 and st["viol_p"] == 0 and st["nonpositive"] == 0
    assert st["dt_exceed"] == 0
    assert np.all(dts > 0)


def test_metric_identities(square):
    m, o, _ = square
    off, j, cx, cy = o.graph()
    nn = len(off) - 1
    sx = np.add.reduceat(cx, off[:-1])
    sy = np.add.reduceat(cy, off[:-1])
    assert np.abs(sx).max() < 1e-15 and np.abs(sy).max() < 1e-15
    # c_ji = -c_ij for every node pair
    lookup = {}
    for i in range(nn):
        for k in range(off[i], off[i + 1]):
            lookup[(i, int(j[k]))] = (cx[k], cy[k])
    for (a, b), c in lookup.items():
        assert b >= 0
        d = lookup[(b, a)]
        assert abs(c[0] + d[0]) < 1e-18 and abs(c[1] + d[1]) < 1e-18


def bar_state_residual(o, u, mesh):
    """m_i du_i/dt = sum_j 2 d_ij (ubar_ij - u_i) from the graph (Eq. barstateform)."""
    off, jj, cx, cy = o.graph()
    K, np_ = mesh.n_elems, o.np
    U = u.reshape(4, -1)
    res = np.zeros_like(U)
    for i in range(U.shape[1]):
        ui = U[:, i]
        for k in range(off[i], off[i + 1]):
            uj = U[:, jj[k]]
            c = np.array([cx[k], cy[k]])
            nrm = np.hypot(*c)
            n = c / nrm
            def lam(q):
                rho = q[0]; p = (G - 1) * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / rho)
                return abs((q[1] * n[0] + q[2] * n[1]) / rho) + math.sqrt(G * p / rho)
            d = nrm * max(lam(ui), lam(uj))
            cdf = cx[k] * (euler_flux(uj, (1, 0)) - euler_flux(ui, (1, 0))) + cy[k] * (euler_flux(uj, (0, 1)) - euler_flux(ui, (0, 1)))
            ubar = 0.5 * (ui + uj) - cdf / (2 * d)
            res[:, i] += 2 * d * (ubar - ui)
    return res.reshape(u.shape)


def test_bar_state_form(square):
    m, o, u = square
    r_cd, _ = o.fv_residual(u)
    r_bar = bar_state_residual(o, u, m)
    assert np.abs(r_cd - r_bar).max() <= 1e-12 * np.abs(r_cd).max()


def test_low_order_step_is_convex():
    m = W.square_mesh()
    o = oracle.Oracle(m, 3)
    u = W.random_state(m, 3, seed=3, rho_range=(0.01, 10.0), p_range=(0.01, 10.0), vmax=3.0)
    dt = o.dt(u, cfl=1.0)
    r, ds = o.fv_residual(u)
    mm = o.masses()
    assert np.all(dt * ds / mm <= 1.0 + 1e-14)
    ufv = u + dt * r / mm[None]
    p = (G - 1) * (ufv[3] - 0.5 * (ufv[1] ** 2 + ufv[2] ** 2) / ufv[0])
    assert ufv[0].min() > 0 and p.min() > 0


def test_smooth_data_no_limiting():
    # density wave far from the positivity bounds: the limited and unlimited
    # residuals coincide (Sec. 3.1: results without limiting are identical)
    m = W.density_wave_mesh(3)
    o = oracle.Oracle(m, 3)
    u = W.density_wave_state(m, 3)
    dt = o.dt(u, cfl=0.95)
    st = np.zeros(16); oracle.lib().orc_stats_init(oracle._d(st))
    r_lim = o.rhs(u, dt=dt, limiting=1, stats=st)
    r_dg = o.rhs(u, dt=0.0)
    s = oracle.stats_dict(st)
    assert s["n_vol_active"] == 0 and s["n_mort_active"] == 0
    assert rel_err(r_lim, r_dg, rhs_scale(u, o.dt(u, cfl=1.0))) <= 1e-12
    assert np.abs(o.rhs(u, dt=dt, limiting=0) - r_dg).max() == 0.0


def test_local_bounds_after_stage(square):
    m, o, u = square
    dt = o.dt(u, cfl=0.5)
    st = np.zeros(16); oracle.lib().orc_stats_init(oracle._d(st))
    _, ut = o.stage(u, 0.0, dt, limiting=2, stats=st)
    s = oracle.stats_dict(st)
    assert s["viol_rho"] == 0 and s["viol_p"] == 0 and s["nonpositive"] == 0
    assert s["n_vol_active"] > 0      # the disc jump is limited
    # positivity only on the same data admits more antidiffusion
    st2 = np.zeros(16); oracle.lib().orc_stats_init(oracle._d(st2))
    o.stage(u, 0.0, dt, limiting=1, stats=st2)
    s2 = oracle.stats_dict(st2)
    assert s2["alpha_vol_m"] < s["alpha_vol_m"]


def _mirror_maps(mesh, np_):
    key = {(int(l), int(x), int(y)): e for e, (l, x, y) in enumerate(zip(mesh.level, mesh.ix, mesh.iy))}
    mx, tr = np.zeros(mesh.n_elems, int), np.zeros(mesh.n_elems, int)
    for e, (l, x, y) in enumerate(zip(mesh.level, mesh.ix, mesh.iy)):
        n = mesh.nx0 << int(l)
        mx[e] = key[(int(l), n - 1 - int(x), int(y))]
        tr[e] = key[(int(l), int(y), int(x))]
    return mx, tr


def test_mirror_and_transpose_symmetry():
    m = W.square_mesh()
    o = oracle.Oracle(m, 3)
    X, Y = W.node_coords(m, 3)
    # symmetric under x -> 1 - x and under x <-> y
    rho = 1 + 0.3 * np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y) + 0.5 * ((X - .5) ** 2 + (Y - .5) ** 2 < 0.02)
    p = 1 + 0.2 * np.cos(2 * np.pi * X) + 0.2 * np.cos(2 * np.pi * Y)
    v1 = 0.2 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    v2 = 0.2 * np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * X)
    u = W.conserved(rho, v1, v2, p, G)
    mx, tr = _mirror_maps(m, 4)
    dt = o.dt(u, cfl=0.5)
    for dtt in (0.0, dt):
        r = o.rhs(u, dt=dtt, limiting=2)
        sc = np.abs(r).max(axis=(1, 2, 3))
        rm = r[:, mx][:, :, :, ::-1]                  # mirrored in x
        sgn = np.array([1, -1, 1, 1])[:, None, None, None]
        assert np.abs(rm * sgn - r).max(axis=(1, 2, 3)).max() <= 1e-11 * sc.max()
        rt = r[:, tr].transpose(0, 1, 3, 2)[[0, 2, 1, 3]]   # transposed
        assert np.abs(rt - r).max() <= 1e-11 * sc.max()


def test_mortar_sparse_conservation_consistency():
    rng = np.random.default_rng(0)
    for N in (2, 3, 4, 5):
        np_ = N + 1
        uL = np.array([W.conserved(rng.uniform(.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(.5, 2), G) for _ in range(np_)])
        us = np.array([W.conserved(rng.uniform(.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(.5, 2), G) for _ in range(2 * np_)])
        F = oracle.mortar_sparse(N, uL, us)
        assert np.abs(F[:np_].sum(0) + F[np_:].sum(0)).max() < 1e-13
        # a constant state: F_i^- = w_i f.n and F_j^+ = -(w_j / 2) f.n
        c = uL[0]
        F = oracle.mortar_sparse(N, np.tile(c, (np_, 1)), np.tile(c, (2 * np_, 1)))
        _, w = oracle.lgl(N)
        f = euler_flux(c, (1, 0))
        np.testing.assert_allclose(F[:np_], w[:, None] * f[None], atol=1e-14)
        np.testing.assert_allclose(F[np_:], -np.concatenate([w, w])[:, None] / 2 * f[None], atol=1e-14)


def test_near_vacuum_positivity():
    # Cheng-Shu isentropic flow (Sec. 3.2) at low resolution, gamma = 3
    n = 8
    L = math.sqrt(2)
    m = W.box_refined_mesh(n, n, (-L, -L, L, L), (-L / 2, -L / 2, 0.0, L / 2))
    o = oracle.Oracle(m, 3, gamma=3.0)
    X, Y = W.node_coords(m, 3)
    xp = X * math.cos(math.pi / 4) + Y * math.sin(math.pi / 4)
    rho = 1 + 0.9999999 * np.sin(np.pi * xp)
    z = np.zeros_like(X)
    u = W.conserved(rho, z, z, rho ** 3, 3.0)
    un, t, dts, st = o.step(u, 5, cfl=0.5, dt_rule=1, limiting=1)
    p = 2.0 * (un[3] - 0.5 * (un[1] ** 2 + un[2] ** 2) / un[0])
    assert un[0].min() > 0 and p.min() > 0
    assert st["nonpositive"] == 0
