"""Oracle pins of the remaining local-limiting variants of Sec. 2.3:

- the modified specific entropy eta = p rho^-gamma / (gamma - 1) of
  Eq. Bounds_Barstates: its closed form on isentropic states p = rho^gamma
  (Sec. 3.2) and its scaling;
- the entropy factor (R21): feasible, and maximal against a brute-force scan;
- after a stage with the entropy bound, every node satisfies
  eta(u_i) >= min_j eta(ubar_(i,j)) with the bar states formed here from the
  graph coefficients (Eq. barstateform), independently of the oracle's
  limiter;
- the low-order-solution bounds (Eq. Bounds_LowOrder): after a stage every
  node lies within the density range and above the entropy minimum of the
  low-order states of itself and its graph neighbours, formed here from the
  oracle's low-order residual;
- positivity limiting ignores both options; the limiter stays conservative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2607_06045_b300 import workloads as W

G = 1.4


def eta(U, g=G):
    """eta over the last axis-0 component layout [4, ...]."""
    p = (g - 1) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
    return p * U[0] ** (-g) / (g - 1)


def euler_flux(u, n):
    rho, m1, m2, E = u
    p = (G - 1) * (E - 0.5 * (m1 * m1 + m2 * m2) / rho)
    vn = (m1 * n[0] + m2 * n[1]) / rho
    return np.array([rho * vn, m1 * vn + p * n[0], m2 * vn + p * n[1], (E + p) * vn])


@pytest.mark.parametrize("g", [1.4, 3.0])
def test_eta_closed_form(g):
    rng = np.random.default_rng(5)
    for _ in range(20):
        rho = rng.uniform(0.01, 10.0)
        v = rng.uniform(-2, 2, 2)
        p = rho ** g   # isentropic (Cheng-Shu data of Sec. 3.2)
        u = np.array([rho, rho * v[0], rho * v[1], p / (g - 1) + 0.5 * rho * (v @ v)])
        assert abs(oracle.entropy_eta(u, g) - 1.0 / (g - 1)) <= 1e-13 / (g - 1)
    # eta(lambda rho, p) = lambda^-gamma eta(rho, p) at rest
    u1 = np.array([2.0, 0.0, 0.0, 3.0 / (g - 1)])
    u2 = np.array([6.0, 0.0, 0.0, 3.0 / (g - 1)])
    assert abs(oracle.entropy_eta(u2, g) / oracle.entropy_eta(u1, g) - 3.0 ** (-g)) <= 1e-14


def test_theta_entropy_is_maximal_and_feasible():
    rng = np.random.default_rng(17)
    grid = np.linspace(0, 1, 20001)
    n_root = 0
    for _ in range(300):
        rho = rng.uniform(0.1, 5.0)
        v = rng.uniform(-1, 1, 2)
        p = rng.uniform(0.1, 5.0)
        u0 = np.array([rho, rho * v[0], rho * v[1], p / (G - 1) + 0.5 * rho * (v @ v)])
        a = rng.normal(0, 1, 4) * np.array([rho, abs(u0[1]) + 1, abs(u0[2]) + 1, u0[3]]) * rng.uniform(0.2, 3)
        K = eta(u0) * rng.uniform(0.3, 1.0)
        hi = rng.uniform(0.2, 1.0)
        # keep the density positive on [0, hi], as the pressure factor does
        if a[0] < 0:
            hi = min(hi, 0.5 * rho / -a[0])
        th = oracle.theta_entropy(u0, a, K, hi)
        assert 0 <= th <= hi
        w = u0 + th * a
        assert w[0] > 0 and eta(w) >= K * (1 - 1e-12)
        ts = grid[grid <= th] if th > 0 else np.array([0.0])
        V = u0[:, None] + a[:, None] * ts[None, :]
        assert (V[0] > 0).all() and (eta(V) >= K * (1 - 1e-12)).all()
        if th < hi:
            # maximal up to the rounding margin of the target (1e-14 of the
            # terms of rho e - K rho^gamma)
            n_root += 1
            t2 = min(hi, th * (1 + 1e-6) + 1e-12)
            w2 = u0 + t2 * a
            assert not (w2[0] > 0 and eta(w2) >= K), (th, t2)
    assert n_root > 30


def _bar_state_eta_min(o, u):
    """min over the node itself and its bar states (Eq. barstateform) of eta,
    from the graph coefficients; ghosts come from the wall/outflow copies the
    meshes here do not have (periodic)."""
    off, jj, cx, cy = o.graph()
    U = u.reshape(4, -1)
    out = eta(U).copy()
    for i in range(U.shape[1]):
        ui = U[:, i]
        for k in range(off[i], off[i + 1]):
            assert jj[k] >= 0
            uj = U[:, jj[k]]
            c = np.array([cx[k], cy[k]])
            nrm = np.hypot(*c)
            n = c / nrm

            def lam(q):
                p = (G - 1) * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / q[0])
                return abs((q[1] * n[0] + q[2] * n[1]) / q[0]) + math.sqrt(G * p / q[0])
            d = nrm * max(lam(ui), lam(uj))
            cdf = cx[k] * (euler_flux(uj, (1, 0)) - euler_flux(ui, (1, 0))) + \
                cy[k] * (euler_flux(uj, (0, 1)) - euler_flux(ui, (0, 1)))
            ub = 0.5 * (ui + uj) - cdf / (2 * d)
            out[i] = min(out[i], eta(ub))
    return out


@pytest.fixture(scope="module")
def disc():
    m = W.square_mesh()
    return m, oracle.Oracle(m, 3), W.disc_wave_state(m, 3)


def _stage(o, u, dt, **kw):
    st = np.zeros(16)
    oracle.lib().orc_stats_init(oracle._d(st))
    _, ut = o.stage(u, 0.0, dt, stats=st, **kw)
    return ut, oracle.stats_dict(st)


def test_entropy_bound_holds_after_stage(disc):
    m, o, u = disc
    dt = o.dt(u, cfl=0.5)
    ut, s = _stage(o, u, dt, limiting=2, entropy=1)
    assert s["viol_rho"] == 0 and s["viol_p"] == 0 and s["viol_eta"] == 0 and s["nonpositive"] == 0
    emin = _bar_state_eta_min(o, u)
    # the low-order state widens the bound (it lies above it in exact arithmetic)
    r, _ = o.fv_residual(u)
    ufv = (u + dt * r / o.masses()[None]).reshape(4, -1)
    emin = np.minimum(emin, eta(ufv))
    e_t = eta(ut.reshape(4, -1))
    assert (e_t >= emin * (1 - 1e-11)).all()
    # without the entropy bound the same stage goes below it somewhere, and
    # the entropy bound costs limiting
    ut0, s0 = _stage(o, u, dt, limiting=2)
    assert (eta(ut0.reshape(4, -1)) < emin * (1 - 1e-9)).any()
    assert s["alpha_vol_m"] > s0["alpha_vol_m"]


def _low_order_bounds(o, u, dt, beta=0.1):
    off, jj, _, _ = o.graph()
    r, _ = o.fv_residual(u)
    ufv = (u + dt * r / o.masses()[None]).reshape(4, -1)
    e_fv = eta(ufv)
    nn = ufv.shape[1]
    lo, hi, el = ufv[0].copy(), ufv[0].copy(), e_fv.copy()
    for i in range(nn):
        js = [int(j) for j in jj[off[i]:off[i + 1]] if j >= 0]
        if js:
            lo[i] = min(lo[i], ufv[0, js].min())
            hi[i] = max(hi[i], ufv[0, js].max())
            el[i] = min(el[i], e_fv[js].min())
    return np.maximum(lo, beta * ufv[0]), hi, el


@pytest.mark.parametrize("entropy", [0, 1])
def test_low_order_bounds_hold_after_stage(disc, entropy):
    m, o, u = disc
    dt = o.dt(u, cfl=0.5)
    ut, s = _stage(o, u, dt, limiting=2, bounds=1, entropy=entropy)
    assert s["viol_rho"] == 0 and s["viol_p"] == 0 and s["viol_eta"] == 0 and s["nonpositive"] == 0
    assert s["n_vol_active"] > 0
    lo, hi, el = _low_order_bounds(o, u, dt)
    q = ut.reshape(4, -1)
    assert (q[0] >= lo - 1e-13 * np.abs(lo)).all() and (q[0] <= hi + 1e-13 * np.abs(hi)).all()
    if entropy:
        assert (eta(q) >= el * (1 - 1e-11)).all()
    # the bar-state and low-order kinds are different bounds
    ut0, _ = _stage(o, u, dt, limiting=2, bounds=0, entropy=entropy)
    assert not np.array_equal(ut, ut0)


def test_positivity_ignores_local_options(disc):
    m, o, u = disc
    dt = 0.5 * o.dt(u, cfl=1.0)
    r = o.rhs(u, dt=dt, limiting=1)
    for b, e in ((1, 0), (0, 1), (1, 1)):
        assert np.array_equal(o.rhs(u, dt=dt, limiting=1, bounds=b, entropy=e), r)


@pytest.mark.parametrize("bounds", [0, 1])
def test_entropy_limited_steps_conserve(disc, bounds):
    m, o, u = disc
    mm = o.masses()
    I0 = (mm[None] * u).reshape(4, -1).sum(axis=1)
    u1, _, _, st = o.step(u, 20, cfl=0.5, limiting=2, bounds=bounds, entropy=1)
    I1 = (mm[None] * u1).reshape(4, -1).sum(axis=1)
    scale = (mm[None] * np.abs(u)).reshape(4, -1).sum(axis=1)
    assert (np.abs(I1 - I0) / scale).max() <= 1e-13
    assert st["viol_rho"] == 0 and st["viol_p"] == 0 and st["viol_eta"] == 0 and st["nonpositive"] == 0
