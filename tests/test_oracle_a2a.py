"""Pins of the oracle's all-to-all low-order mortar flux (Eqs.
interfaceflux_nonlocal, nonlocal_weight; reading R25: the weights are
integrated with the LGL quadrature of the small face):

- the weights equal w_j |S|/2 phi_i(x_j), with the large face's Lagrange
  basis evaluated here by numpy, and satisfy Eq. sum_weights (rows sum to the
  large node's LGL weight, columns to the small node's);
- some weights are negative for N >= 2, so sum_j |omega_ij| exceeds the LGL
  weight: the graph viscosity at mortar nodes grows (the diffusive behaviour
  the paper reports);
- metric identities sum_j c_ij = 0 and c_ji = -c_ij, conservation of the
  residual, free stream, and the convexity of the low-order step under the
  IDP time step with these weights.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as Pn

import oracle
from paper_2607_06045_b300 import workloads as W

G = 1.4


def lagrange(xs, i, x):
    others = [xk for k, xk in enumerate(xs) if k != i]
    return np.prod([(x - xk) / (xs[i] - xk) for xk in others], axis=0)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_weights_closed_form_and_sums(N):
    m = W.square_mesh()
    o = oracle.Oracle(m, N, mortar_low=1)
    wa = o.mortar_weights()
    xi, w = oracle.lgl(N)
    np_ = N + 1
    ref = np.zeros((np_, 2 * np_))
    for p in range(2):
        xs = (xi + (2 * p - 1)) / 2.0    # small-face nodes in the large face's coordinate
        for l in range(np_):
            for k in range(np_):
                ref[k, p * np_ + l] = 0.5 * w[l] * lagrange(xi, k, xs[l])
    ref[np.abs(ref) < 1e-13] = 0.0
    np.testing.assert_allclose(wa, ref, atol=1e-14)
    # Eq. sum_weights: rows sum to w_k, each small face's columns to w_l / 2
    np.testing.assert_allclose(wa.sum(axis=1), w, atol=1e-14)
    np.testing.assert_allclose(wa.sum(axis=0), np.concatenate([w, w]) / 2.0, atol=1e-14)
    if N >= 2:
        assert wa.min() < 0.0
        assert (np.abs(wa).sum(axis=1) > w * (1 + 1e-6)).any()
    # the sparse weights are what mortar_low = 0 uses
    assert np.array_equal(oracle.Oracle(m, N).mortar_weights(), oracle.operators(N)[4])


def test_graph_identities_and_conservation():
    m = W.square_mesh()
    o = oracle.Oracle(m, 3, mortar_low=1)
    off, j, cx, cy = o.graph()
    sx, sy = np.add.reduceat(cx, off[:-1]), np.add.reduceat(cy, off[:-1])
    assert np.abs(sx).max() < 1e-15 and np.abs(sy).max() < 1e-15
    lookup = {}
    for i in range(len(off) - 1):
        for k in range(off[i], off[i + 1]):
            lookup[(i, int(j[k]))] = (cx[k], cy[k])
    for (a, b), c in lookup.items():
        d = lookup[(b, a)]
        assert abs(c[0] + d[0]) < 1e-18 and abs(c[1] + d[1]) < 1e-18
    # more graph edges than the sparse weights
    assert len(j) > len(oracle.Oracle(m, 3).graph()[1])
    u = W.disc_wave_state(m, 3)
    mm = o.masses()
    dt = o.dt(u, cfl=0.5)
    for lim in (0, 2):
        r = o.rhs(u, dt=dt if lim else 0.0, limiting=lim)
        for v in range(4):
            assert abs((mm * r[v]).sum()) <= 1e-13 * (mm * np.abs(r[v])).sum()


def test_free_stream_and_convexity():
    m = W.square_mesh()
    o = oracle.Oracle(m, 3, mortar_low=1)
    sh = (m.n_elems, 4, 4)
    uf = W.conserved(1.3 * np.ones(sh), 0.4 * np.ones(sh), -0.7 * np.ones(sh), 2.0 * np.ones(sh), G)
    scale = 3.0 / o.masses().min()
    assert np.abs(o.rhs(uf, dt=0.0)).max() < 1e-13 * scale
    assert np.abs(o.rhs(uf, dt=o.dt(uf, cfl=0.5), limiting=2)).max() < 1e-13 * scale
    u = W.random_state(m, 3, seed=3, rho_range=(0.01, 10.0), p_range=(0.01, 10.0), vmax=3.0)
    dt = o.dt(u, cfl=1.0)
    r, ds = o.fv_residual(u)
    mm = o.masses()
    assert np.all(dt * ds / mm <= 1.0 + 1e-14)
    ufv = u + dt * r / mm[None]
    p = (G - 1) * (ufv[3] - 0.5 * (ufv[1] ** 2 + ufv[2] ** 2) / ufv[0])
    assert ufv[0].min() > 0 and p.min() > 0
    # the all-to-all graph viscosity sum_j 2 d_ij is larger in total and at
    # most mortar nodes (the wave speeds of the pairs differ, so not at each)
    _, ds0 = oracle.Oracle(m, 3).fv_residual(u)
    assert ds.sum() > ds0.sum() and (ds > ds0 * (1 + 1e-3)).sum() > 100
    assert dt <= oracle.Oracle(m, 3).dt(u, cfl=1.0)
    st = np.zeros(16); oracle.lib().orc_stats_init(oracle._d(st))
    o.stage(u, 0.0, 0.5 * dt, limiting=2, stats=st)
    s = oracle.stats_dict(st)
    assert s["viol_rho"] == 0 and s["viol_p"] == 0 and s["nonpositive"] == 0
