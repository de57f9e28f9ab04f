"""Pins of the 3D oracle on 2:1 octrees (oracle/idp_oracle3d.c: the
nonconforming faces of Sec. 2.2 in 3D, readings R5, R9, R16 and R32).

- Mortar table: the list of mortars (direction, large element, its side, the
  four small elements by transverse offset) equals the one found from the
  leaf boxes alone.
- Reduction to 2D: on the z-extrusion of a 2:1 quadtree and a state that
  does not depend on z, the high-order residual (tensor-product mortar
  interpolation, LLF, L2 projection) and the low-order residual (sparse
  mortar pairs with product weights) equal the 2D oracle's node by node,
  and the z-momentum residual vanishes.
- Axis permutation on an octree: the residual of the cyclically renamed mesh
  and state is the renamed residual, so z-normal mortars are the x-normal
  ones.
- Free stream and discrete conservation of every residual and of 10 limited
  steps on octrees with small and with large elements inside.
- FCT assembly with mortars: every factor forced to 0 gives the low-order
  residual bit for bit, forced to 1 the high-order one.
- Mortar factor (R9 with the n_i budget): n_i counted from the mortar table,
  every node of a mortar admissible at l_S, and a node inadmissible just above
  l_S when l_S < 1, on meshes whose edge and corner nodes lie on two and
  three mortars.
- Consistency: the high-order residual of the smooth density wave converges
  on octrees (L2 order above N + 0.2, maximum-norm order above N - 0.5 at
  N = 3), which a wrong mortar interpolation, projection or area would
  break.
Each pin is checked to fail on a mistake planted in a copy of the oracle.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import o3d
from paper_2607_06045_b300 import workloads as W

G = 1.4
SRC = os.path.join(os.path.dirname(o3d.__file__), "idp_oracle3d.c")
TOL = 1e-14   # the relative slack of the bounds (R15)


def pressure(u):
    return (G - 1.0) * (u[..., 4] - 0.5 * (u[..., 1] ** 2 + u[..., 2] ** 2 + u[..., 3] ** 2) / u[..., 0])


# ----------------------------------------------------------------------------
# meshes and states
# ----------------------------------------------------------------------------

UNIT = (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
MID = (0.34, 0.34, 0.34, 0.66, 0.66, 0.66)


def small_inside():
    """3^3 periodic base grid, the centre element refined: six mortars whose
    small elements' edge and corner nodes lie on two and three of them."""
    return W.box_refined_mesh3(3, 3, 3, UNIT, MID)


def large_inside():
    """3^3 base grid, everything but the centre element refined: the centre's
    six faces are mortars with it as the large element (its edge and corner
    nodes on two and three mortars); walls in x, outflow in y, periodic in z."""
    return W.box_refined_mesh3(3, 3, 3, UNIT, MID, inside=False,
                               bc=(W.BC_WALL, W.BC_WALL, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_PERIODIC, W.BC_PERIODIC))


def sphere_state(m, N, centre=(1 / 3, 0.4, 0.45), r0=0.15):
    """A density and pressure jump on a sphere about a corner edge of the
    refined block, on a smooth background moving diagonally."""
    X, Y, Z = W.node_coords3(m, N)
    inside = ((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2) < r0 ** 2
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * Z) + 2.0 * inside
    one = np.ones_like(X)
    return W.conserved3(rho, 0.3 * one, -0.2 * one, 0.25 * one, 1.0 + 4.0 * inside, G)


def rough_state(m, N, seed, wide=False):
    if wide:
        return W.random3_state(m, N, seed=seed, rho_range=(0.1, 10.0), p_range=(0.1, 10.0), vmax=2.0)
    return W.random3_state(m, N, seed=seed, rho_range=(0.3, 3.0), p_range=(0.3, 3.0), vmax=1.0)


_CASES = None


def cases():
    """(mesh, N, state): the sphere on both meshes (N = 1..4 and N = 3), a
    rough seeded state (N = 2), and a rougher one whose large-side
    interpolation leaves the admissible set on some mortars (R16, N = 2)."""
    global _CASES
    if _CASES is None:
        a, b = small_inside(), large_inside()
        _CASES = [(a, N, sphere_state(a, N)) for N in (1, 2, 3, 4)]
        _CASES += [(b, 3, sphere_state(b, 3)), (a, 2, rough_state(a, 2, 5)), (b, 2, rough_state(b, 2, 6, wide=True))]
    return _CASES


# ----------------------------------------------------------------------------
# the mesh's own view of its mortars
# ----------------------------------------------------------------------------

def geometric_mortars(mesh):
    """{(d, large, large on the low side): [small p = p1 + 2 p2]} from the leaf
    boxes on the finest grid (p1, p2 the offsets along (d+1) % 3, (d+2) % 3)."""
    Lm = int(mesh.level.max())
    sh = Lm - mesh.level.astype(np.int64)
    lo = np.stack([mesh.ix.astype(np.int64) << sh, mesh.iy.astype(np.int64) << sh, mesh.iz.astype(np.int64) << sh], 1)
    size = np.int64(1) << sh
    n = [mesh.nx0 << Lm, mesh.ny0 << Lm, mesh.nz0 << Lm]
    per = [mesh.bc[2 * d] == W.BC_PERIODIC for d in range(3)]
    out = {}
    K = mesh.n_elems
    for L in range(K):
        for S in range(K):
            if mesh.level[S] != mesh.level[L] + 1:
                continue
            for d in range(3):
                t1, t2 = (d + 1) % 3, (d + 2) % 3
                if not (lo[L, t1] <= lo[S, t1] < lo[L, t1] + size[L] and lo[L, t2] <= lo[S, t2] < lo[L, t2] + size[L]):
                    continue
                for low in (1, 0):
                    a = lo[L, d] + size[L] if low else lo[L, d]
                    b = lo[S, d] if low else lo[S, d] + size[S]
                    if per[d]:
                        a, b = a % n[d], b % n[d]
                    if a == b:
                        p = (lo[S, t1] - lo[L, t1]) // size[S] + 2 * ((lo[S, t2] - lo[L, t2]) // size[S])
                        out.setdefault((d, L, low), [None] * 4)[int(p)] = S
    return out


def face_nodes(e, s, N):
    """Global nodes of side s (-x, +x, -y, +y, -z, +z) of element e, layout
    [e][k][j][i]."""
    np1 = N + 1
    d, hi = s // 2, s & 1
    r = range(np1)
    out = set()
    for k in r:
        for j in r:
            for i in r:
                if (i, j, k)[d] == (N if hi else 0):
                    out.add(((e * np1 + k) * np1 + j) * np1 + i)
    return out


def mortar_node_sets(tab, N):
    sets = []
    for d, L, low, *S in tab:
        sL = 2 * d + (1 if low else 0)
        st = set(face_nodes(L, sL, N))
        for e in S:
            st |= face_nodes(e, sL ^ 1, N)
        sets.append(st)
    return sets


# ----------------------------------------------------------------------------
# checks (each returns a list of failures)
# ----------------------------------------------------------------------------

def check_table(mesh, N=2):
    o = o3d.Oracle3D(mesh, N)
    geo = geometric_mortars(mesh)
    got = {(int(t[0]), int(t[1]), int(t[2])): [int(x) for x in t[3:]] for t in o.mortars()}
    bad = []
    if got != geo:
        bad.append(f"mortar table {sorted(got.items())} differs from the geometric {sorted(geo.items())}")
    if len(geo) == 0:
        bad.append("no mortar in the case")
    return bad


def check_reduction_2d(N, mesh2=None, seed=0):
    m2 = mesh2 or W.box_refined_mesh(4, 4, (0.0, 0.0, 1.0, 1.0), (0.3, 0.3, 0.7, 0.7))
    m3, e2 = W.extruded_mesh3(m2, 0.0, 0.5)
    u2 = W.random_state(m2, N, seed=seed)
    u3 = W.extrude_state(u2, e2, N)
    o2, o3 = oracle.Oracle(m2, N), o3d.Oracle3D(m3, N)
    np1 = N + 1
    bad = []
    if o3.M == 0:
        bad.append("no mortar in the extruded mesh")
    m2w = o2.masses().reshape(m2.n_elems, np1, np1)
    m3w = o3.masses().reshape(m3.n_elems, np1, np1, np1)
    for name in ("dg", "fv"):
        if name == "dg":
            r2 = o2.rhs(u2, dt=0.0).reshape(4, m2.n_elems, np1, np1)
            r3 = o3.rhs(u3, dt=0.0).reshape(5, m3.n_elems, np1, np1, np1)
        else:
            r2 = o2.fv_residual(u2)[0].reshape(4, m2.n_elems, np1, np1) / m2w
            r3 = o3.fv_residual(u3)[0].reshape(5, m3.n_elems, np1, np1, np1) / m3w
        for a, b in ((0, 0), (1, 1), (2, 2), (4, 3)):
            ref = np.broadcast_to(r2[b][e2][:, None], r3[a].shape)
            err = np.abs(r3[a] - ref).max() / np.abs(r2[b]).max()
            if not err <= 1e-13:
                bad.append(f"{name} residual of variable {a} differs from 2D by {err:.2e}")
        if not np.abs(r3[3]).max() <= 1e-13 * np.abs(r3[1:3]).max():
            bad.append(f"{name}: z momentum residual does not vanish")
    return bad


def permute_mesh3(m):
    """Axes renamed (x, y, z) -> (y, z, x): new x is old z, new y old x, new z
    old y; leaves keep their order."""
    x0, y0, z0, x1, y1, z1 = m.box
    bc = m.bc
    return W.Mesh3(m.nz0, m.nx0, m.ny0, (z0, x0, y0, z1, x1, y1), m.level.copy(), m.iz.copy(), m.ix.copy(),
                   m.iy.copy(), bc=(bc[4], bc[5], bc[0], bc[1], bc[2], bc[3]))


def permute_state3(u, K, N):
    np1 = N + 1
    U = np.asarray(u).reshape(5, K, np1, np1, np1)       # v, e, k, j, i
    V = U.transpose(0, 1, 3, 4, 2)                        # v, e, k'=j, j'=i, i'=k
    return np.ascontiguousarray(V[[0, 3, 1, 2, 4]].reshape(5, -1))


def check_free_stream_conservation(mesh, N):
    o = o3d.Oracle3D(mesh, N)
    bad = []
    one = np.ones((mesh.n_elems, N + 1, N + 1, N + 1))
    # no normal velocity through walls: their mirrored ghost state is then the state itself
    vel = [0.0 if W.BC_WALL in mesh.bc[2 * d:2 * d + 2] else v for d, v in enumerate((0.2, -0.1, 0.3))]
    uf = W.conserved3(1.3 * one, vel[0] * one, vel[1] * one, vel[2] * one, 2.0 * one, G)
    for lim in (0, 1, 2):
        dt = 0.0 if lim == 0 else o.dt(uf)
        e = np.abs(o.rhs(uf, dt=dt, limiting=lim)).max() / (np.abs(uf).max() / o.dt(uf))
        if not e <= 1e-12:
            bad.append(f"free stream residual {e:.2e} (limiting {lim})")
    periodic = all(b == W.BC_PERIODIC for b in mesh.bc)
    u = W.random3_state(mesh, N, seed=2)
    if periodic:
        for lim in (0, 1, 2):
            dt = 0.0 if lim == 0 else o.dt(u)
            r = o.stage(u, dt, limiting=lim)[0].reshape(5, -1)
            e = (np.abs(r.sum(axis=1)) / np.abs(r).sum(axis=1)).max()
            if not e <= 1e-13:
                bad.append(f"residual not conservative: {e:.2e} (limiting {lim})")
        un, _, _, st = o.step(u, 10, cfl=0.5, limiting=2)
        I0, I1 = o.integrals(u), o.integrals(un)
        if not (np.abs(I1 - I0) <= 1e-13 * np.abs(I0).max()).all():
            bad.append("totals drift over 10 steps")
        if st["viol_rho"] or st["viol_p"] or st["nonpositive"]:
            bad.append("bound violations over 10 steps")
        if st["n_mort_active"] == 0:
            bad.append("no mortar limited over 10 steps")
    return bad


def check_fct(mesh, N, u):
    o = o3d.Oracle3D(mesh, N)
    dt = 0.5 * o.dt(u, cfl=1.0)
    bad = []
    r0 = o.stage_debug(u, dt, limiting=2, force_ell=0.0)["res"]
    if not np.array_equal(r0, o.fv_residual(u)[0]):
        bad.append("factors 0: not the low-order residual")
    r1 = o.stage_debug(u, dt, limiting=2, force_ell=1.0)["res"]
    rdg = o.dg_residual(u)
    sc = np.abs(u).reshape(5, -1).max(axis=1)[:, None] * o.masses()[None, :] / o.dt(u, cfl=1.0)
    e = (np.abs(r1 - rdg).reshape(5, -1) / sc).max()
    if not e <= 1e-12:
        bad.append(f"factors 1: high-order residual missed by {e:.2e}")
    return bad


def _lagrange(xn, s):
    """[len(s)][len(xn)]: the Lagrange basis of the nodes xn at the points s."""
    out = np.ones((len(s), len(xn)))
    for j in range(len(xn)):
        for m in range(len(xn)):
            if m != j:
                out[:, j] *= (s - xn[m]) / (xn[j] - xn[m])
    return out


def interpolation_inadmissible(u, K, N, mortar):
    """R16 evaluated here: does the large side's face polynomial, sampled at
    the four small faces' nodes, give a non-positive density or pressure?"""
    d, L, low = int(mortar[0]), int(mortar[1]), int(mortar[2])
    np1 = N + 1
    U = np.asarray(u).reshape(5, K, np1, np1, np1)
    F = np.zeros((5, np1, np1))
    for a in range(np1):
        for b in range(np1):
            idx = [0, 0, 0]
            idx[d] = N if low else 0
            idx[(d + 1) % 3], idx[(d + 2) % 3] = a, b
            F[:, a, b] = U[:, L, idx[2], idx[1], idx[0]]
    x = W.lgl_points(N)
    bad = False
    for p1 in (0, 1):
        for p2 in (0, 1):
            I1, I2 = _lagrange(x, (x + 2 * p1 - 1) / 2), _lagrange(x, (x + 2 * p2 - 1) / 2)
            ui = np.einsum("la,mb,vab->lmv", I1, I2, F)
            bad |= bool((ui[..., 0] <= 0.0).any() or (pressure(ui) <= 0.0).any())
    return bad


def check_mortar_factor(mesh, N, u):
    o = o3d.Oracle3D(mesh, N)
    dt = o.dt(u, cfl=0.5)
    r = o.stage_debug(u, dt, limiting=2)
    node, rec, ell = r["node"], r["mortar"], r["mortar_ell"]
    mm = o.masses()
    bad = []
    sets = mortar_node_sets(o.mortars(), N)
    count = np.zeros(len(mm), int)
    for st in sets:
        for g in st:
            count[g] += 1
    if count.max() < 3:
        bad.append("no node lies on three mortars: the case does not exercise the n_i budget")
    n_limited = 0
    tab = o.mortars()
    for m, st in enumerate(sets):
        R = rec[m]
        if interpolation_inadmissible(u, mesh.n_elems, N, tab[m]):
            # R16: the mortar keeps its low-order flux
            if ell[m] != 0.0 or np.any(R[:, 15:20] != 0.0):
                bad.append(f"mortar {m}: inadmissible interpolation but l_S = {ell[m]}")
            n_limited += 1
            continue
        g = R[:, 0].astype(int)
        if set(g.tolist()) != st or len(g) != len(st):
            bad.append(f"mortar {m}: node list differs from the mesh's")
            continue
        ni = count[g]
        if not np.array_equal(R[:, 14].astype(int), ni):
            bad.append(f"mortar {m}: n_i differs from the count of incident mortars")
        a_expect = (ni * dt / mm[g])[:, None] * R[:, 15:20]
        if np.any(np.abs(R[:, 6:11] - a_expect) > 1e-14 * np.abs(a_expect).max() + 1e-300):
            bad.append(f"mortar {m}: correction not scaled by n_i dt / m_i")
        u0, av = R[:, 1:6], R[:, 6:11]
        rlo, rhi, pm = R[:, 11], R[:, 12], R[:, 13]
        tol = TOL * np.abs(node[g, 0])

        def feasible(l, slack):
            v = u0 + l * av
            ok_r = (v[:, 0] >= rlo - tol - slack * np.abs(rlo)) & (v[:, 0] <= rhi + tol + slack * np.abs(rhi))
            ok_p = pressure(v) >= pm - TOL * np.abs(pm) - slack * np.abs(pm)
            return ok_r & ok_p
        lS = ell[m]
        if not np.all(feasible(lS, 1e-13)):
            bad.append(f"mortar {m}: a node is inadmissible at l_S = {lS}")
        if lS < 1.0:
            n_limited += 1
            up = min(1.0, lS + max(1e-8 * lS, 1e-10))
            if np.all(feasible(up, 0.0)):
                bad.append(f"mortar {m}: l_S = {lS} is not the largest admissible factor")
    if n_limited == 0:
        bad.append("no mortar is limited: the case does not exercise R9")
    if r["stats"]["viol_rho"] or r["stats"]["viol_p"] or r["stats"]["nonpositive"]:
        bad.append("bound violations after the stage")
    return bad


def _wave_errors(n, N, inside):
    """L2 and maximum error of the high-order density residual of the density
    wave against its exact time derivative, on the n^3 octree over [-1, 1]^3
    with the middle third refined (inside) or everything else refined."""
    m = W.box_refined_mesh3(n, n, n, (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0), (-1 / 3, -1 / 3, -1 / 3, 1 / 3, 1 / 3, 1 / 3),
                            inside=inside)
    o = o3d.Oracle3D(m, N)
    u = W.density_wave3_state(m, N)
    X, Y, Z = W.node_coords3(m, N)
    vel = (0.1, 0.2, -0.1)
    rho_t = -sum(vel) * 0.98 * np.cos(np.pi * (X + Y + Z)) * np.pi
    r = o.rhs(u, dt=0.0).reshape(5, -1)[0]
    e = r - rho_t.ravel()
    return np.sqrt((o.masses() * e ** 2).sum() / 8.0), np.abs(e).max(), o.M


def check_consistency(N=3):
    bad = []
    for inside in (True, False):
        (a2, ai, Ma), (b2, bi, Mb) = _wave_errors(6, N, inside), _wave_errors(12, N, inside)
        if Ma == 0 or Mb == 0:
            bad.append("no mortar in the convergence meshes")
        r2, ri = np.log2(a2 / b2), np.log2(ai / bi)
        if not (r2 > N + 0.2 and ri > N - 0.5):
            bad.append(f"orders {r2:.2f} (L2), {ri:.2f} (max) with inside={inside}")
    return bad


# ----------------------------------------------------------------------------
# the pins
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["small_inside", "large_inside"])
def test_mortar_table(which):
    assert check_table({"small_inside": small_inside, "large_inside": large_inside}[which]()) == []


def test_mortar_directions():
    """The extruded meshes hold x- and y-normal mortars, the octrees all three
    directions with the large element on either side."""
    m3, _ = W.extruded_mesh3(W.box_refined_mesh(4, 4, (0.0, 0.0, 1.0, 1.0), (0.3, 0.3, 0.7, 0.7)))
    assert {k[0] for k in geometric_mortars(m3)} == {0, 1}
    for m in (small_inside(), large_inside()):
        assert {(k[0], k[2]) for k in geometric_mortars(m)} == {(d, s) for d in range(3) for s in (0, 1)}


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_reduces_to_2d_on_extruded_octree(N):
    assert check_reduction_2d(N, seed=N) == []


def test_reduces_to_2d_with_levels_one_and_two():
    m2 = W.box_refined_mesh(4, 4, (0.0, 0.0, 1.0, 1.0), (0.3, 0.3, 0.7, 0.7), base_level=1)
    assert check_reduction_2d(3, m2, seed=4) == []


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("which", ["small_inside", "large_inside"])
def test_axis_permutation_on_octree(N, which):
    m = {"small_inside": small_inside, "large_inside": large_inside}[which]()
    mp = permute_mesh3(m)
    u = W.random3_state(m, N, seed=7).reshape(5, -1)
    up = permute_state3(u, m.n_elems, N)
    o, op = o3d.Oracle3D(m, N), o3d.Oracle3D(mp, N)
    for lim in (0, 1, 2):
        dt = 0.0 if lim == 0 else 0.5 * o.dt(u, cfl=1.0)
        r = o.rhs(u, dt=dt, limiting=lim).reshape(5, -1)
        rp = op.rhs(up, dt=dt, limiting=lim).reshape(5, -1)
        rr = permute_state3(r, m.n_elems, N)
        scale = np.abs(r).max(axis=1)[[0, 3, 1, 2, 4]]
        assert (np.abs(rp - rr).max(axis=1) / scale).max() <= 1e-12, lim
    assert abs(o.dt(u) - op.dt(up)) <= 1e-14 * o.dt(u)


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("which", ["small_inside", "large_inside"])
def test_free_stream_and_conservation_on_octree(N, which):
    m = {"small_inside": small_inside, "large_inside": large_inside}[which]()
    if which == "large_inside":
        m.bc = (W.BC_PERIODIC,) * 6
    assert check_free_stream_conservation(m, N) == []


def test_free_stream_with_walls_and_outflow():
    assert check_free_stream_conservation(large_inside(), 3) == []


@pytest.mark.parametrize("case", range(7))
def test_fct_assembly_with_mortars(case):
    m, N, u = cases()[case]
    assert check_fct(m, N, u) == []


@pytest.mark.parametrize("case", range(7))
def test_mortar_factor_maximal(case):
    m, N, u = cases()[case]
    assert check_mortar_factor(m, N, u) == []


def test_r16_case_meets_inadmissible_interpolations():
    m, N, u = cases()[6]
    o = o3d.Oracle3D(m, N)
    flags = [interpolation_inadmissible(u, m.n_elems, N, t) for t in o.mortars()]
    assert 0 < sum(flags)


def test_high_order_consistency_on_octrees():
    assert check_consistency() == []


# ----------------------------------------------------------------------------
# each pin catches its planted mistakes
# ----------------------------------------------------------------------------

MUTATIONS = {
    # R9: no high-order mortar flux at all
    "mortar_zero": ("        if (g_force3 >= 0.0) lS = g_force3;\n        if (g_mortar3)",
                    "        lS = 0.0;\n        if (g_force3 >= 0.0) lS = g_force3;\n        if (g_mortar3)"),
    # R9: the budget n_i ignored
    "mortar_n1": ("double mi = mass3(c, i), ni = (double)c->mcount[i], tolr",
                  "double mi = mass3(c, i), ni = 1.0, tolr"),
    # R9: only the large side's nodes limit the factor
    "mortar_large_only": ("            if (th < lS) lS = th;\n",
                          "            if (th < lS && q < NR) lS = th;\n"),
    # FCT assembly: the large side's antidiffusive flux with the wrong sign
    "mortar_h_sign": ("                H[t][v] = -(FL2 - Flo[t][v]);",
                      "                H[t][v] = (FL2 - Flo[t][v]);"),
    # R5: small-face offsets swapped in the interpolation
    "interp_swap": ("double wgt = c->Ii[(p & 1) * np + l1][k1] * c->Ii[(p >> 1) * np + l2][k2];",
                    "double wgt = c->Ii[(p >> 1) * np + l1][k1] * c->Ii[(p & 1) * np + l2][k2];"),
    # R5: small-face offsets swapped in the projection
    "proj_swap": ("acc += c->P[k1][(p & 1) * np + l1] * c->P[k2][(p >> 1) * np + l2] * fs[p][l1 + np * l2][v];",
                  "acc += c->P[k1][(p >> 1) * np + l1] * c->P[k2][(p & 1) * np + l2] * fs[p][l1 + np * l2][v];"),
    # R32: the product weights of the mortar's low-order fluxes with the offsets swapped
    "weight_swap": ("double wgt = c->wt[k1][p1 * np + l1] * c->wt[k2][p2 * np + l2] * qa;",
                    "double wgt = c->wt[k1][p2 * np + l1] * c->wt[k2][p1 * np + l2] * qa;"),
    # R32: the graph's small-side weights with the offsets swapped
    "graph_weight_swap": ("double wgt = c->wt[k1][p1 * np + t1] * c->wt[k2][p2 * np + t2];",
                          "double wgt = c->wt[k1][p2 * np + t1] * c->wt[k2][p1 * np + t2];"),
    # the small faces' area taken as the large face's
    "small_area": ("double qaL = qarea(c, L, d), qaS = qaL / 4.0;",
                   "double qaL = qarea(c, L, d), qaS = qaL;"),
}

CHECKS = {
    "mortar_zero": "factor", "mortar_n1": "factor", "mortar_large_only": "factor", "mortar_h_sign": "fct",
    "interp_swap": "reduction", "proj_swap": "reduction", "weight_swap": "fct", "graph_weight_swap": "reduction",
    "small_area": "consistency",
}


@pytest.fixture(scope="module")
def mutants(tmp_path_factory):
    src = open(SRC).read()
    out = {}
    for k, (old, new) in MUTATIONS.items():
        assert src.count(old) == 1, f"mutation {k}: pattern not unique"
        d = tmp_path_factory.mktemp(f"mut3_{k}")
        out[k] = o3d.compile_source(src.replace(old, new), str(d / f"lib_{k}.so"))
    return out


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(mutants, name):
    check = CHECKS[name]
    with o3d.using(mutants[name]):
        if check == "factor":
            failures = sum((check_mortar_factor(m, N, u) for m, N, u in cases()), [])
        elif check == "fct":
            failures = sum((check_fct(m, N, u) for m, N, u in cases()), [])
        elif check == "reduction":
            failures = sum((check_reduction_2d(N, seed=N) for N in (2, 3)), [])
        else:
            failures = check_consistency()
    assert failures, f"mutation {name} passed the {check} pins"
