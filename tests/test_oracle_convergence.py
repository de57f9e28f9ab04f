"""Convergence pins of the oracle on smooth problems with exact solutions.

- Density wave (Sec. 3.1, Eq. entropywave2D) on the periodic box [-1,1]^2
  with the refined box [-0.5,0] x [-0.5,0.5]: with positivity limiting no
  limiting is active and the order approaches N+1 (the paper prints EOC
  3.11 and 3.77 for the first two refinements of N = 3, Table
  ConvergenceTestPositivity; the error norm is not stated, so only the order
  is pinned).
- Isentropic vortex (exact solution: the advected initial state) on a
  nonconforming periodic mesh.
"""
import numpy as np
import pytest

import oracle
from paper_2607_06045_b300 import workloads as W


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


def test_density_wave_order_N3():
    errs = []
    for lvl in (2, 3, 4):
        m = W.density_wave_mesh(lvl)
        o = oracle.Oracle(m, 3)
        u = run_to(o, W.density_wave_state(m, 3), 0.1, 0.95, limiting=1)
        errs.append(l2(o, u[0], W.density_wave_state(m, 3, t=0.1)[0]))
    eoc = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[0] > errs[1] > errs[2]
    assert eoc[-1] > 3.0, eoc


def test_vortex_order_N3():
    errs = []
    for n in (8, 16):
        m = W.box_refined_mesh(n, n, (-5.0, -5.0, 5.0, 5.0), (-2.5, -2.5, 0.0, 2.5))
        o = oracle.Oracle(m, 3)
        u = run_to(o, W.vortex_state(m, 3), 0.25, 0.9, limiting=1)
        errs.append(l2(o, u[0], W.vortex_state(m, 3, t=0.25)[0]))
    eoc = np.log2(errs[0] / errs[1])
    assert eoc > 2.5, (errs, eoc)
