"""Convergence pins of the oracle on smooth problems with exact solutions.

- Density wave (Sec. 3.1, Eq. entropywave2D) on the periodic box [-1,1]^2
  with the refined box [-0.5,0] x [-0.5,0.5], positivity limiting, CFL 0.95
  with the IDP time step, to T = 1: the L2 errors of all four conserved
  variables equal the paper's printed values (Table
  ConvergenceTestPositivity for N = 3, Table ConvergenceTest_polydeg4 (a) for
  N = 4; `tests/golden/density_wave_positivity_N*.txt`) to their three
  printed digits. The error norm (reading R29): the solution polynomial of
  each element interpolated to the 2N+1 LGL nodes, the squared difference
  from the exact solution there summed with the LGL weights and the element
  Jacobian, divided by the domain area, square root. No limiting is active,
  so this pins the high-order scheme absolutely: the volume flux (R1), the
  LLF surface flux with its wave speed (R3), the L2 mortar (R5), SSP-RK3
  and the IDP time step.
- The same pin fails on a planted mistake in the volume flux.
- Isentropic vortex (exact solution: the advected initial state) on a
  nonconforming periodic mesh: EOC above 2.5.
"""
import os

import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2607_06045_b300 import workloads as W

G = 1.4
SRC = os.path.join(os.path.dirname(oracle.__file__), "idp_oracle.c")


def run_to(o, u, T, cfl, limiting):
    t = 0.0
    while t < T - 1e-14:
        dt = min(o.dt(u, t, cfl=cfl), T - t)
        _, u1 = o.stage(u, t, dt, limiting=limiting)
        _, ut = o.stage(u1, t + dt, dt, limiting=limiting)
        u2 = 0.75 * u + 0.25 * ut
        _, ut = o.stage(u2, t + 0.5 * dt, dt, limiting=limiting)
        u = u / 3.0 + 2.0 / 3.0 * ut
        t += dt
    return u


def l2(o, a, b):
    return float(np.sqrt((o.masses() * (a - b) ** 2).sum()))


def lagrange_matrix(xs, x):
    """L[a][j] = l_j(x_a), the Lagrange basis on the nodes xs (numpy only)."""
    L = np.ones((len(x), len(xs)))
    for j in range(len(xs)):
        for k in range(len(xs)):
            if k != j:
                L[:, j] *= (x - xs[k]) / (xs[j] - xs[k])
    return L


def analysis_l2(mesh, N, u, exact, area):
    """R29: per-variable L2 error of the nodal solution u [4][K][N+1][N+1]
    against exact(X, Y) -> [4][...], by interpolation to the 2N+1 LGL
    nodes, normalised by the domain area."""
    xi, _ = oracle.lgl(N)
    xa, wa = oracle.lgl(2 * N)
    I = lagrange_matrix(xi, xa)
    x0, y0, x1, y1 = mesh.box
    lev = mesh.level.astype(np.int64)
    hx = (x1 - x0) / (mesh.nx0 * (1 << lev))
    hy = (y1 - y0) / (mesh.ny0 * (1 << lev))
    cx = x0 + (mesh.ix + 0.5) * hx
    cy = y0 + (mesh.iy + 0.5) * hy
    X = cx[:, None, None] + 0.5 * hx[:, None, None] * xa[None, None, :]
    Y = cy[:, None, None] + 0.5 * hy[:, None, None] * xa[None, :, None]
    na = len(xa)
    X = np.broadcast_to(X, (mesh.n_elems, na, na))
    Y = np.broadcast_to(Y, (mesh.n_elems, na, na))
    ua = np.einsum("bj,ai,veji->veba", I, I, u)
    wgt = wa[None, :, None] * wa[None, None, :] * (hx * hy / 4.0)[:, None, None]
    d = ua - exact(X, Y)
    return np.sqrt((wgt[None] * d * d).sum(axis=(1, 2, 3)) / area)


def density_wave_exact(T):
    def f(X, Y):
        rho = 2.0 + 0.98 * np.sin(2 * np.pi * ((X - 0.1 * T) + (Y - 0.2 * T)))
        return W.conserved(rho, 0.1 * np.ones_like(X), 0.2 * np.ones_like(X), 20.0 * np.ones_like(X), G)
    return f


_ERRS = {}


def density_wave_errors(N, level, T=1.0):
    key = (N, level, T, oracle.lib()._name)
    if key not in _ERRS:
        _ERRS[key] = _density_wave_errors(N, level, T)
    return _ERRS[key]


def _density_wave_errors(N, level, T):
    m = W.density_wave_mesh(level)
    o = oracle.Oracle(m, N)
    u = run_to(o, W.density_wave_state(m, N), T, 0.95, limiting=1)
    return analysis_l2(m, N, u, density_wave_exact(T), 4.0)


def printed(N, level):
    for row in read_golden(f"density_wave_positivity_N{N}.txt"):
        if row[0] == level:
            return np.array(row[1:5])
    raise KeyError(level)


def three_digits_agree(ours, table):
    """|ours - printed| within 0.6 units of the printed value's last digit."""
    unit = 10.0 ** (np.floor(np.log10(table)) - 2)
    return np.abs(ours - table) <= 0.6 * unit


@pytest.mark.parametrize("N,level", [(3, 2), (3, 3), (4, 2)])
def test_density_wave_matches_paper_table(N, level):
    e = density_wave_errors(N, level)
    assert np.all(three_digits_agree(e, printed(N, level))), (e, printed(N, level))


def test_density_wave_order_N3():
    # the EOC between levels 2 and 3 the paper prints (3.11) follows from the
    # two rows; checked here from the oracle's own errors
    e2, e3 = density_wave_errors(3, 2)[0], density_wave_errors(3, 3)[0]
    assert abs(np.log2(e2 / e3) - 3.11) < 0.01


def test_density_wave_pin_catches_planted_mistake(tmp_path):
    # the logarithmic density mean of Ranocha's flux replaced by the
    # arithmetic mean: still consistent and symmetric, but no longer the
    # paper's volume flux (the wave has constant velocity and pressure, so
    # the density flux is the term it tests)
    src = open(SRC).read()
    old = "    double rho_ln = orc_logmean(rL, rR);\n"
    assert src.count(old) == 1
    lib = oracle.compile_source(src.replace(old, "    double rho_ln = 0.5 * (rL + rR);\n"),
                                str(tmp_path / "lib_flux.so"))
    with oracle.using(lib):
        e = density_wave_errors(3, 2)
    assert not np.all(three_digits_agree(e, printed(3, 2))), e


def test_vortex_order_N3():
    errs = []
    for n in (8, 16):
        m = W.box_refined_mesh(n, n, (-5.0, -5.0, 5.0, 5.0), (-2.5, -2.5, 0.0, 2.5))
        o = oracle.Oracle(m, 3)
        u = run_to(o, W.vortex_state(m, 3), 0.25, 0.9, limiting=1)
        errs.append(l2(o, u[0], W.vortex_state(m, 3, t=0.25)[0]))
    eoc = np.log2(errs[0] / errs[1])
    assert eoc > 2.5, (errs, eoc)
