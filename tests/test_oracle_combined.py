"""Oracle pins of the combined limiting (Sec. 3.5, Eq. combination_posLim_local)
and of its shock indicator (reading R20: Hennemann et al.'s modal energy
indicator applied to the pressure):

- the indicator of a polynomial of degree <= N - 2 in each variable is 0, of a
  pure highest mode 1, and at the energy fraction E = T exactly 1/2 (the
  logistic map's midpoint);
- where the indicator is 0 everywhere (smooth data) the combined scheme is the
  positivity-limited scheme bit for bit, and where it is 1 everywhere (N = 1,
  whose highest-but-one energy fraction is always 1) the locally limited one;
- in between it keeps positivity and conservation over many steps.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle
from paper_2607_06045_b300 import workloads as W


def _modal_field(N, coeff):
    """p(x_i, y_j) = sum m_kl Lt_k(x_i) Lt_l(y_j), Lt the orthonormal Legendre
    polynomials, as [j][i]."""
    xi, _ = oracle.lgl(N)
    V = np.array([[np.sqrt((2 * k + 1) / 2.0) * Lg.legval(x, [0] * k + [1]) for k in range(N + 1)] for x in xi])
    return V @ coeff @ V.T   # [i][j] -> transpose to [j][i]


@pytest.mark.parametrize("N", [2, 3, 5])
def test_indicator_closed_forms(N):
    rng = np.random.default_rng(N)
    # degree <= N - 2 in each variable: all energy in e0
    m = np.zeros((N + 1, N + 1))
    m[:N - 1, :N - 1] = rng.uniform(-1, 1, (N - 1, N - 1))
    m[0, 0] = 3.0
    assert oracle.indicator(N, _modal_field(N, m).T) == 0.0
    # a pure highest mode
    m = np.zeros((N + 1, N + 1))
    m[N, 1] = 1.0
    assert oracle.indicator(N, _modal_field(N, m).T) == 1.0
    # E = T exactly: m00 = 1, m_N0 = sqrt(T / (1 - T))
    T = 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)
    m = np.zeros((N + 1, N + 1))
    m[0, 0] = 1.0
    m[N, 0] = np.sqrt(T / (1.0 - T))
    p = _modal_field(N, m)
    assert abs(oracle.indicator(N, p.T) - 0.5) < 1e-8
    # transposing the element (x <-> y) does not change it
    assert abs(oracle.indicator(N, p) - 0.5) < 1e-8


def test_combined_reduces_to_positivity_on_smooth_data():
    m = W.density_wave_mesh(2)
    u = W.density_wave_state(m, 3)
    o = oracle.Oracle(m, 3)
    dt = 0.5 * o.dt(u, cfl=1.0)
    r3 = o.rhs(u, dt=dt, limiting=3)
    r1 = o.rhs(u, dt=dt, limiting=1)
    assert np.array_equal(r3, r1)


def test_combined_reduces_to_local_at_degree_one():
    m = W.square_mesh()
    u = W.disc_wave_state(m, 1)
    o = oracle.Oracle(m, 1)
    dt = 0.5 * o.dt(u, cfl=1.0)
    assert np.array_equal(o.rhs(u, dt=dt, limiting=3), o.rhs(u, dt=dt, limiting=2))


def test_combined_positivity_and_conservation():
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    o = oracle.Oracle(m, 3)
    # the blend is active: neither of the two pure schemes
    dt = 0.5 * o.dt(u, cfl=1.0)
    r3 = o.rhs(u, dt=dt, limiting=3)
    assert not np.array_equal(r3, o.rhs(u, dt=dt, limiting=1))
    assert not np.array_equal(r3, o.rhs(u, dt=dt, limiting=2))
    mm = o.masses()
    I0 = (mm[None] * u).reshape(4, -1).sum(axis=1)
    u1, t1, _, st = o.step(u, 30, cfl=0.5, limiting=3)
    I1 = (mm[None] * u1).reshape(4, -1).sum(axis=1)
    scale = (mm[None] * np.abs(u)).reshape(4, -1).sum(axis=1)
    assert (np.abs(I1 - I0) / scale).max() <= 1e-13
    assert st["nonpositive"] == 0 and st["viol_rho"] == 0 and st["viol_p"] == 0, st
    assert u1[0].min() > 0.0
