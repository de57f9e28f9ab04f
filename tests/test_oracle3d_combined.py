"""Pins of the 3D oracle's combined limiting (limiting 3: Sec. 3.5,
Eq. combination_posLim_local with d = 3; reading R34 for the indicator).

- The shock indicator: on a pressure that does not depend on z it equals
  the 2D oracle's indicator of the x-y slice; a cyclic renaming of the axes
  leaves it unchanged; a polynomial of degree N - 2 gives 0 and the top
  Legendre mode alone gives 1.
- The blend: with every indicator forced to 0 the combined stage is the
  positivity-limited one bit for bit, forced to 1 the locally limited one,
  and at 0.3 each interface factor is 0.7 times its positivity-only factor
  plus 0.3 times its local one.
- A near-vacuum blast on an octree stays positive over 10 combined steps.
Each indicator pin fails on a mistake planted in a copy of the oracle.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import o3d
from paper_2607_06045_b300 import workloads as W

SRC = os.path.join(os.path.dirname(o3d.__file__), "idp_oracle3d.c")


def smooth_pressures(N, seed):
    """Pressures 1 + low modes + c P_N(x) with c set (by bisection on the 2D
    indicator) so that the indicator takes values near 0.2, 0.5 and 0.8."""
    rng = np.random.default_rng(seed)
    x = oracle.lgl(N)[0]
    X, Y = np.meshgrid(x, x, indexing="xy")
    top = np.polynomial.legendre.legval(X, [0] * N + [1])
    out = []
    for target in (0.2, 0.5, 0.8):
        a = rng.uniform(0.05, 0.3, 2)
        base = 1.0 + a[0] * X + a[1] * Y

        def alpha(lc):
            return oracle.indicator(N, base + 10.0 ** lc * top)
        lo, hi = -8.0, 0.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if alpha(mid) < target:
                lo = mid
            else:
                hi = mid
        out.append(base + 10.0 ** (0.5 * (lo + hi)) * top)
    return out


def check_indicator():
    bad = []
    seen_mid = 0
    for N in (2, 3, 4):
        x = oracle.lgl(N)[0]
        for p2 in smooth_pressures(N, N):
            a2 = oracle.indicator(N, p2)
            p3 = np.broadcast_to(p2[None], (N + 1,) * 3).copy()
            a3 = o3d.indicator3(N, p3)
            if abs(a3 - a2) > 1e-12:
                bad.append(f"N={N}: z-independent indicator {a3} differs from the 2D {a2}")
            seen_mid += 0.0 < a2 < 1.0
            # renamed axes (x, y, z) -> (y, z, x)
            ap = o3d.indicator3(N, np.ascontiguousarray(p3.transpose(1, 2, 0)))
            if abs(ap - a3) > 1e-12:
                bad.append(f"N={N}: indicator changes under a renaming of the axes ({ap} vs {a3})")
        X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
        low = 1.0 + 0.3 * X ** (N - 2) + (0.2 * Y * Z if N >= 3 else 0.0) + 0.1 * Z ** (N - 2)
        if o3d.indicator3(N, low.transpose(2, 1, 0)) != 0.0:
            bad.append(f"N={N}: a polynomial of degree N - 2 does not give 0")
        top = np.polynomial.legendre.legval(Z, [0] * N + [1])
        if o3d.indicator3(N, top.transpose(2, 1, 0)) != 1.0:
            bad.append(f"N={N}: the top mode alone does not give 1")
    if seen_mid < 4:
        bad.append("too few indicator values strictly between 0 and 1")
    return bad


def test_indicator_pins():
    assert check_indicator() == []


MUTATIONS = {
    # the top mode by the sum of the indices instead of their maximum
    "top_sum": ("        int top = i > j ? i : j;\n        if (k > top) top = k;",
                "        int top = i + j + k;"),
    # no transform along z
    "no_z": ("        for (int k = 0; k < np; ++k) s += Vi[m][k] * a[(k * np + j) * np + i];",
             "        s = a[(m * np + j) * np + i];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_indicator_pins_catch_planted_mistakes(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1
    lib = o3d.compile_source(src.replace(old, new), str(tmp_path / f"lib_{name}.so"))
    with o3d.using(lib):
        assert check_indicator(), name


def _case():
    m = W.box_refined_mesh3(3, 3, 3, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), (0.34, 0.34, 0.34, 0.66, 0.66, 0.66))
    N = 3
    X, Y, Z = W.node_coords3(m, N)
    inside = ((X - 1 / 3) ** 2 + (Y - 0.4) ** 2 + (Z - 0.45) ** 2) < 0.15 ** 2
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) + 2.0 * inside
    one = np.ones_like(X)
    return m, N, W.conserved3(rho, 0.3 * one, -0.2 * one, 0.25 * one, 1.0 + 4.0 * inside, 1.4)


def test_blend_reductions():
    m, N, u = _case()
    o = o3d.Oracle3D(m, N)
    dt = o.dt(u, cfl=0.5)
    try:
        o3d.set_force_alpha(0.0)
        r0 = o.rhs(u, dt=dt, limiting=3)
        o3d.set_force_alpha(1.0)
        r1 = o.rhs(u, dt=dt, limiting=3)
        o3d.set_force_alpha(0.3)
        d3 = o.stage_debug(u, dt, limiting=3)
    finally:
        o3d.set_force_alpha(-1.0)
    assert np.array_equal(r0, o.rhs(u, dt=dt, limiting=1))
    assert np.array_equal(r1, o.rhs(u, dt=dt, limiting=2))
    l1 = o.stage_debug(u, dt, limiting=1)["iface"][:, 6]
    l2 = o.stage_debug(u, dt, limiting=2)["iface"][:, 6]
    l3 = d3["iface"][:, 6]
    assert np.any(l1 != l2), "the case must separate the two limiters"
    assert np.array_equal(l3, 0.7 * l1 + 0.3 * l2)


def test_combined_near_vacuum_blast_on_octree():
    m = W.box_refined_mesh3(4, 4, 4, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), (0.3, 0.3, 0.3, 0.7, 0.7, 0.7))
    N = 3
    u = W.blast3_state(m, N, rho_bg=1e-5, p_bg=1e-6, rho_in=1.0, p_in=1e2, centre=(0.45, 0.5, 0.55), r0=0.2)
    o = o3d.Oracle3D(m, N)
    un, _, _, st = o.step(u, 10, cfl=0.9, limiting=3)
    q = un.reshape(5, -1)
    p = 0.4 * (q[4] - 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0])
    assert q[0].min() > 0.0 and p.min() > 0.0
    assert st["nonpositive"] == 0 and st["viol_p"] == 0 and st["viol_rho"] == 0
