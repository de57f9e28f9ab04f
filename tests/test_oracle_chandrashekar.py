"""Pins of the oracle's Chandrashekar volume flux (reading R23) and of the
high-Mach jet setup (gamma = 5/3, reading R24):

- consistency with the Euler flux, symmetry, exact Tadmor entropy
  conservation (w_R - w_L) . f* = psi_R - psi_L with the textbook entropy
  variables, for gamma = 1.4 and 5/3;
- kinetic-energy-preserving momentum form: the tangential momentum flux is
  f_rho times the mean tangential velocity, and the normal part adds a
  pressure average lying between p_L and p_R;
- the flux-differencing form equals the evolution form and free stream is
  preserved on a nonconforming mesh with this volume flux;
- the jet's boundary: the total mass-weighted residual equals the sum of the
  LLF boundary fluxes against the inflow band and the ambient state, formed
  here; limited steps of the jet keep positivity and bounds.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2607_06045_b300 import workloads as W


def euler_flux(u, n, g):
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (g - 1) * (E - 0.5 * rho * (v1 * v1 + v2 * v2))
    vn = v1 * n[0] + v2 * n[1]
    return np.array([rho * vn, m1 * vn + p * n[0], m2 * vn + p * n[1], (E + p) * vn])


def rand_state(rng, g):
    rho = rng.uniform(0.1, 10)
    v = rng.uniform(-2, 2, 2)
    p = rng.uniform(0.1, 10)
    return np.array([rho, rho * v[0], rho * v[1], p / (g - 1) + 0.5 * rho * (v @ v)])


def entropy_vars(u, g):
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (g - 1) * (E - 0.5 * rho * (v1 * v1 + v2 * v2))
    s = math.log(p) - g * math.log(rho)
    return np.array([(g - s) / (g - 1) - rho * (v1 * v1 + v2 * v2) / (2 * p), rho * v1 / p, rho * v2 / p, -rho / p])


def pres(u, g):
    return (g - 1) * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0])


@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0])
@pytest.mark.parametrize("d", [0, 1])
def test_consistent_symmetric(d, g):
    rng = np.random.default_rng(2 + d)
    n = (1.0, 0.0) if d == 0 else (0.0, 1.0)
    for _ in range(200):
        a, b = rand_state(rng, g), rand_state(rng, g)
        np.testing.assert_allclose(oracle.chandrashekar(a, a, d, g), euler_flux(a, n, g), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(oracle.chandrashekar(a, b, d, g), oracle.chandrashekar(b, a, d, g),
                                   rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0])
@pytest.mark.parametrize("d", [0, 1])
def test_entropy_conservative(d, g):
    rng = np.random.default_rng(5 + d)
    for _ in range(500):
        a, b = rand_state(rng, g), rand_state(rng, g)
        f = oracle.chandrashekar(a, b, d, g)
        lhs = (entropy_vars(b, g) - entropy_vars(a, g)) @ f
        rhs = b[1 + d] - a[1 + d]   # psi = rho v_n
        scale = np.abs(entropy_vars(b, g) - entropy_vars(a, g)) @ np.abs(f) + abs(a[1 + d]) + abs(b[1 + d])
        assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


def test_kinetic_energy_preserving_form():
    rng = np.random.default_rng(9)
    g = 1.4
    for _ in range(200):
        a, b = rand_state(rng, g), rand_state(rng, g)
        for d in (0, 1):
            f = oracle.chandrashekar(a, b, d, g)
            vm = 0.5 * (a[1:3] / a[0] + b[1:3] / b[0])
            t = 1 - d   # tangential momentum component
            np.testing.assert_allclose(f[1 + t], f[0] * vm[t], rtol=1e-13, atol=1e-14)
            ph = f[1 + d] - f[0] * vm[d]
            lo, hi = sorted((pres(a, g), pres(b, g)))
            assert lo * (1 - 1e-13) <= ph <= hi * (1 + 1e-13)
    # it differs from Ranocha's flux away from equal states
    a, b = rand_state(rng, g), rand_state(rng, g)
    assert np.abs(oracle.chandrashekar(a, b, 0, g) - oracle.ranocha(a, b, 0, g)).max() > 1e-6


def test_scheme_forms_and_free_stream():
    m = W.square_mesh()
    o = oracle.Oracle(m, 3, volume_flux=1)
    u = W.smooth_random_state(m, 3, seed=4)
    r1, r2 = o.dg_residual(u), o.dg_residual(u, form="fd")
    assert np.abs(r1 - r2).max() <= 1e-13 * np.abs(r1).max()
    # differs from the Ranocha residual
    assert np.abs(r1 - oracle.Oracle(m, 3).dg_residual(u)).max() > 1e-8 * np.abs(r1).max()
    sh = (m.n_elems, 4, 4)
    uf = W.conserved(1.3 * np.ones(sh), 0.4 * np.ones(sh), -0.7 * np.ones(sh), 2.0 * np.ones(sh), 1.4)
    scale = 3.0 / o.masses().min()
    assert np.abs(o.rhs(uf, dt=0.0)).max() < 1e-13 * scale
    dt = o.dt(uf, cfl=0.5)
    assert np.abs(o.rhs(uf, dt=dt, limiting=3)).max() < 1e-13 * scale


def _jet_boundary_flux_sum(o, m, u, N, g):
    """sum over the boundary face nodes of w_t |face|/2 * LLF(interior, ghost)
    along the outward normal, the ghost being the jet inflow for |y| <= 0.05
    on the -x side and the ambient state elsewhere on the x sides."""
    xi, w = oracle.lgl(N)
    x0, y0, x1, y1 = m.box
    nx0 = m.nx0
    ft, _ = o.faces()
    tot = np.zeros(4)
    for e in range(m.n_elems):
        h = (x1 - x0) / (nx0 << int(m.level[e]))
        yc = y0 + (m.iy[e] + 0.5) * h
        for s, n in ((0, (-1.0, 0.0)), (1, (1.0, 0.0))):
            if ft[e, s] != 1:
                continue
            i = 0 if s == 0 else N
            for t in range(N + 1):
                y = yc + 0.5 * h * xi[t]
                prim = W.JET_IN if (s == 0 and abs(y) <= 0.05) else W.JET_AMBIENT
                q = W.conserved(*(np.array([v]) for v in prim), g)[:, 0]
                ui = u[:, e, t, i]
                tot -= w[t] * h / 2 * oracle.llf(ui, q, n, g)
    return tot


def test_jet_boundary_and_steps():
    g = W.JET_GAMMA
    m = W.jet_mesh(n0=8, levels=2)
    N = 3
    o = oracle.Oracle(m, N, gamma=g, volume_flux=1)
    u = W.jet_state(m, N, g, seed=3)
    # total residual = boundary fluxes (interior fluxes cancel, y periodic)
    r = o.rhs(u, dt=0.0)
    mm = o.masses()
    tot = (mm[None] * r).reshape(4, -1).sum(axis=1)
    ref = _jet_boundary_flux_sum(o, m, u, N, g)
    assert np.abs(tot - ref).max() <= 1e-11 * np.abs(ref).max(), (tot, ref)
    assert ref[0] > 0   # mass enters through the band
    # limited steps (combined limiting, as for the paper's jet) stay admissible
    u1, t1, _, st = o.step(u, 5, cfl=0.5, limiting=3)
    assert st["nonpositive"] == 0 and st["viol_rho"] == 0 and st["viol_p"] == 0
    assert u1[0].max() > 1.0   # the jet's density has entered
