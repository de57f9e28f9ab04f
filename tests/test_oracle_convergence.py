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
- With local limiting (density and entropy bounds; Table
  ConvergenceTestLocalLimiting) the errors lie within 25% of the printed
  ones and the EOC within 0.2 of 1.68: a band, not the digits, since the
  limiter details the paper defers set the amount of low-order flux (parity
  unpinned in those digits).
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


def run_to(o, u, T, cfl, limiting, entropy=0):
    t = 0.0
    while t < T - 1e-14:
        dt = min(o.dt(u, t, cfl=cfl), T - t)
        _, u1 = o.stage(u, t, dt, limiting=limiting, entropy=entropy)
        _, ut = o.stage(u1, t + dt, dt, limiting=limiting, entropy=entropy)
        u2 = 0.75 * u + 0.25 * ut
        _, ut = o.stage(u2, t + 0.5 * dt, dt, limiting=limiting, entropy=entropy)
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


def _density_wave_errors(N, level, T, limiting=1, entropy=0):
    m = W.density_wave_mesh(level)
    o = oracle.Oracle(m, N)
    u = run_to(o, W.density_wave_state(m, N), T, 0.95, limiting=limiting, entropy=entropy)
    return analysis_l2(m, N, u, density_wave_exact(T), 4.0)


def printed(N, level, table="positivity"):
    for row in read_golden(f"density_wave_{table}_N{N}.txt"):
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


def test_density_wave_local_limiting_band():
    """Table ConvergenceTestLocalLimiting (N = 3) within a band, not to its
    digits. Local limiting as Sec. 3 defines it: the density bounds and the
    entropy bound from the bar states (readings R6, R21). The limiter details
    the paper defers to a cited paper (readings R7-R9, R15, R21) set how much
    low-order flux it admits on this smooth wave, and the oracle's errors
    come out 16% and 11% below the printed ones at levels 2 and 3 (parity
    unpinned in those digits; with the low-order-solution bounds instead of
    the bar states they come out 10% above and 3% below). What the band
    pins: local limiting is active (the errors are some 6 and 16 times the
    positivity table's) with the paper's amount of dissipation within 25%,
    the momentum and energy errors in the wave's ratios to the density error
    (0.1, 0.2, 0.025), and an EOC within 0.2 of the printed 1.68."""
    e2 = _density_wave_errors(3, 2, 1.0, limiting=2, entropy=1)
    e3 = _density_wave_errors(3, 3, 1.0, limiting=2, entropy=1)
    for e, lv in ((e2, 2), (e3, 3)):
        ratio = e / printed(3, lv, "local")
        assert np.all((ratio > 0.75) & (ratio < 1.25)), (lv, e, ratio)
        assert np.allclose(e[1:] / e[0], [0.1, 0.2, 0.025], rtol=0.02), (lv, e)
        assert e[0] > 5 * printed(3, lv)[0]   # far above the positivity-limited error
    eoc = np.log2(e2[0] / e3[0])
    assert abs(eoc - 1.68) < 0.2, eoc


def test_local_limiting_band_catches_planted_mistake(tmp_path):
    # the entropy factor formed at the left end of each interface only (the
    # right end keeps its pressure factor): still admissible at one end,
    # but not the entropy bound of Eq. Bounds_Barstates at every node
    src = open(SRC).read()
    old = "                    if (ent) th_r = orc_theta_entropy(gm, u0, av, emin[gr], th_r);\n"
    assert src.count(old) == 1
    lib = oracle.compile_source(src.replace(old, "\n"), str(tmp_path / "lib_ent.so"))
    with oracle.using(lib):
        e = _density_wave_errors(3, 2, 1.0, limiting=2, entropy=1)
    ratio = e / printed(3, 2, "local")
    assert not np.all((ratio > 0.75) & (ratio < 1.25)), (e, ratio)


def test_vortex_order_N3():
    errs = []
    for n in (8, 16):
        m = W.box_refined_mesh(n, n, (-5.0, -5.0, 5.0, 5.0), (-2.5, -2.5, 0.0, 2.5))
        o = oracle.Oracle(m, 3)
        u = run_to(o, W.vortex_state(m, 3), 0.25, 0.9, limiting=1)
        errs.append(l2(o, u[0], W.vortex_state(m, 3, t=0.25)[0]))
    eoc = np.log2(errs[0] / errs[1])
    assert eoc > 2.5, (errs, eoc)
