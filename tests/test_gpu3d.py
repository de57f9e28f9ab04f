"""GPU parity of the 3D path (include/idp_dgsem3d.h) against the 3D oracle
(oracle/o3d.py) on the same seeded inputs, through the C ABI.

Tolerances: right-hand sides (unlimited and limited) 1e-12 relative to the
residual scale max|u_v| / dt_idp, as in 2D; the time step 1e-13; SSP-RK3
steps 1e-10 relative to max|u_v| after 20 steps. The FP32 form against the
FP64 oracle: mass-weighted L1 of the density within 1e-5 and of the other
fields within 3e-5 after 20 steps, right-hand sides within 1e-5.
"""
import numpy as np
import pytest

from oracle import o3d
from paper_2607_06045_b300 import build, idp
from paper_2607_06045_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = 1.4


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    yield


def dev(u):
    import torch
    return torch.from_numpy(np.ascontiguousarray(u)).cuda()


def grid(kind, n=(3, 2, 4)):
    if kind == "periodic":
        return W.Grid3(*n, box=(0.0, 0.0, 0.0, 0.9, 0.6, 1.2))
    if kind == "walls":
        return W.Grid3(*n, box=(0.0, 0.0, 0.0, 0.9, 0.6, 1.2),
                       bc=(o3d.BC_WALL, o3d.BC_WALL, o3d.BC_OUTFLOW, o3d.BC_OUTFLOW, o3d.BC_PERIODIC, o3d.BC_PERIODIC))
    bcp = np.zeros((6, 5))
    bcp[:] = [1.2, 0.3, -0.2, 0.1, 1.5]
    return W.Grid3(*n, box=(0.0, 0.0, 0.0, 0.9, 0.6, 1.2),
                   bc=(o3d.BC_DIRICHLET, o3d.BC_OUTFLOW, o3d.BC_WALL, o3d.BC_DIRICHLET, o3d.BC_OUTFLOW, o3d.BC_WALL),
                   bc_prim=bcp)


def gpu_rhs(ctx, u, dt):
    import torch
    ud = dev(u)
    out = torch.empty_like(ud)
    ctx.idp3d_rhs(ud, dt, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def scale(u, dt_idp):
    return np.abs(u).reshape(5, -1).max(axis=1) / dt_idp


def rel(a, b, sc):
    return float((np.abs(np.asarray(a) - np.asarray(b)).reshape(5, -1).max(axis=1) / sc).max())


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["periodic", "walls", "dirichlet"])
def test_rhs(N, kind):
    g = grid(kind)
    u = W.random3_state(g, N, seed=10 * N + len(kind), rho_range=(0.3, 3.0), p_range=(0.3, 3.0), vmax=1.0)
    o = o3d.Oracle3D(g, N)
    dt_idp = o.dt(u, cfl=1.0)
    sc = scale(u, dt_idp)
    for lim in (0, 1, 2, 3):
        ctx = idp.Context3D(g, N, limiting=lim)
        dt = 0.0 if lim == 0 else 0.5 * dt_idp
        r_o = o.rhs(u, dt=dt, limiting=lim)
        r_g = gpu_rhs(ctx, u, dt)
        e = rel(r_g, r_o, sc)
        assert e <= 1e-12, (lim, e)
        ctx.close()


@pytest.mark.parametrize("N", [1, 3])
def test_dt(N):
    g = grid("dirichlet")
    u = W.random3_state(g, N, seed=3)
    o = o3d.Oracle3D(g, N)
    ctx = idp.Context3D(g, N, cfl=0.7)
    d_g = ctx.idp3d_dt(dev(u))
    d_o = o.dt(u, cfl=0.7)
    assert abs(d_g - d_o) <= 1e-13 * d_o
    ctx.close()


@pytest.mark.parametrize("N,lim", [(2, 2), (3, 1), (3, 2), (4, 2)])
def test_steps(N, lim):
    import torch
    g = grid("walls", n=(3, 3, 2))
    u = W.random3_state(g, N, seed=N, rho_range=(0.5, 2.0), p_range=(0.5, 2.0), vmax=0.5)
    o = o3d.Oracle3D(g, N)
    u_o, t_o, _, st_o = o.step(u, 20, cfl=0.5, limiting=lim)
    ctx = idp.Context3D(g, N, limiting=lim, cfl=0.5)
    ud = dev(u)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 20, t)
    assert rc == idp.IDP_OK
    torch.cuda.synchronize()
    sc = np.abs(u_o).reshape(5, -1).max(axis=1)
    err = (np.abs(ud.cpu().numpy() - u_o).reshape(5, -1).max(axis=1) / sc).max()
    assert err <= 1e-10, err
    assert abs(t[0] - t_o) <= 1e-12 * t_o
    rc, st = ctx.idp3d_limiter_stats()
    assert rc == idp.IDP_OK
    assert st["n_viol_density"] == 0 and st["n_viol_pressure"] == 0 and st["n_nonpositive"] == 0
    assert st["n_stages"] == 60
    ctx.close()


def test_conservation_and_blast_positivity():
    import torch
    N = 3
    g = W.Grid3(6, 6, 6)
    u = W.blast3_state(g, N, rho_bg=1e-5, p_bg=1e-6, rho_in=1.0, p_in=1e2)
    ctx = idp.Context3D(g, N, limiting=1, cfl=0.9)
    ud = dev(u)
    I0 = ctx.idp3d_integrals(ud)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 40, t)
    assert rc == idp.IDP_OK
    I1 = ctx.idp3d_integrals(ud)
    assert np.abs(I1 - I0).max() <= 1e-12 * np.abs(I0).max()
    q = ud.cpu().numpy().reshape(5, -1)
    p = (G - 1.0) * (q[4] - 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0])
    assert q[0].min() > 0.0 and p.min() > 0.0
    rc, st = ctx.idp3d_limiter_stats()
    assert st["n_nonpositive"] == 0 and st["n_viol_pressure"] == 0 and st["n_active"] > 0
    torch.cuda.synchronize()
    ctx.close()


def test_larger_grid_one_step():
    """16 x 16 x 8 elements at N = 3 (131k nodes, several element blocks per
    SM): one SSP-RK3 step against the oracle."""
    import torch
    N = 3
    g = W.Grid3(16, 16, 8, box=(0.0, 0.0, 0.0, 2.0, 2.0, 1.0))
    u = W.random3_state(g, N, seed=21, rho_range=(0.5, 2.0), p_range=(0.5, 2.0), vmax=0.5)
    o = o3d.Oracle3D(g, N)
    u_o, t_o, _, _ = o.step(u, 1, cfl=0.5, limiting=2)
    ctx = idp.Context3D(g, N, limiting=2, cfl=0.5)
    ud = dev(u)
    t = np.zeros(1)
    ctx.idp3d_step(ud, 1, t)
    torch.cuda.synchronize()
    sc = np.abs(u_o).reshape(5, -1).max(axis=1)
    err = (np.abs(ud.cpu().numpy() - u_o).reshape(5, -1).max(axis=1) / sc).max()
    assert err <= 1e-12, err
    ctx.close()


def test_bad_arguments():
    g = W.Grid3(2, 2, 2)
    with pytest.raises(idp.IdpError):
        idp.Context3D(g, 5)
    bad = W.Grid3(2, 2, 2, bc=(o3d.BC_PERIODIC, o3d.BC_WALL) + (o3d.BC_PERIODIC,) * 4)
    with pytest.raises(idp.IdpError):
        idp.Context3D(bad, 2)


# ----------------------------------------------------------------------------
# 2:1 octrees with mortars
# ----------------------------------------------------------------------------

UNIT = (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
MID = (0.34, 0.34, 0.34, 0.66, 0.66, 0.66)


def octree(kind):
    """small: the centre of a 3^3 periodic grid refined (six mortars, small
    elements inside); large: everything but the centre refined (the centre
    is the large element of six mortars), walls in x, Dirichlet and outflow
    in y, periodic in z; extruded: a 2:1 quadtree extruded in z (levels 1
    and 2, mortars normal to x and y)."""
    if kind == "small":
        return W.box_refined_mesh3(3, 3, 3, UNIT, MID)
    if kind == "large":
        bcp = np.zeros((6, 5))
        bcp[:] = [1.2, 0.3, -0.2, 0.1, 1.5]
        m = W.box_refined_mesh3(3, 3, 3, UNIT, MID, inside=False,
                                bc=(o3d.BC_WALL, o3d.BC_WALL, o3d.BC_DIRICHLET, o3d.BC_OUTFLOW, o3d.BC_PERIODIC,
                                    o3d.BC_PERIODIC))
        m.bc_prim = bcp
        return m
    m2 = W.box_refined_mesh(3, 2, (0.0, 0.0, 0.9, 0.6), (0.25, 0.2, 0.6, 0.45), base_level=1)
    return W.extruded_mesh3(m2, 0.0, 0.4)[0]


def sphere3(m, N, centre=(1 / 3, 0.4, 0.45), r0=0.15):
    X, Y, Z = W.node_coords3(m, N)
    inside = ((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2) < r0 ** 2
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * Z) + 2.0 * inside
    one = np.ones_like(X)
    return W.conserved3(rho, 0.3 * one, -0.2 * one, 0.25 * one, 1.0 + 4.0 * inside, G)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["small", "large", "extruded"])
def test_octree_rhs(N, kind):
    m = octree(kind)
    o = o3d.Oracle3D(m, N)
    for state in ("random", "sphere"):
        if state == "random":
            u = W.random3_state(m, N, seed=10 * N + len(kind), rho_range=(0.3, 3.0), p_range=(0.3, 3.0), vmax=1.0)
        else:
            u = sphere3(m, N)
        dt_idp = o.dt(u, cfl=1.0)
        sc = scale(u, dt_idp)
        for lim in (0, 1, 2, 3):
            ctx = idp.Context3D(m, N, limiting=lim)
            assert ctx.n_mortars == o.M > 0
            dt = 0.0 if lim == 0 else 0.5 * dt_idp
            e = rel(gpu_rhs(ctx, u, dt), o.rhs(u, dt=dt, limiting=lim), sc)
            assert e <= 1e-12, (state, lim, e)
            ctx.close()


def test_octree_rhs_with_inadmissible_interpolation():
    """A rough state whose large-side interpolation leaves the admissible set
    on some mortars: those keep their low-order flux (R16)."""
    m, N = octree("large"), 2
    u = W.random3_state(m, N, seed=6, rho_range=(0.1, 10.0), p_range=(0.1, 10.0), vmax=2.0)
    o = o3d.Oracle3D(m, N)
    dt_idp = o.dt(u, cfl=1.0)
    sc = scale(u, dt_idp)
    for lim, dt in ((0, 0.0), (2, 0.5 * dt_idp)):
        ctx = idp.Context3D(m, N, limiting=lim)
        e = rel(gpu_rhs(ctx, u, dt), o.rhs(u, dt=dt, limiting=lim), sc)
        assert e <= 1e-12, (lim, e)
        ctx.close()


@pytest.mark.parametrize("N", [1, 3, 4])
@pytest.mark.parametrize("kind", ["small", "large"])
def test_octree_dt(N, kind):
    m = octree(kind)
    u = W.random3_state(m, N, seed=3)
    o = o3d.Oracle3D(m, N)
    ctx = idp.Context3D(m, N, cfl=0.7)
    d_g, d_o = ctx.idp3d_dt(dev(u)), o.dt(u, cfl=0.7)
    assert abs(d_g - d_o) <= 1e-13 * d_o
    ctx.close()


@pytest.mark.parametrize("N,lim,kind", [(2, 2, "small"), (3, 1, "large"), (3, 2, "large"), (4, 2, "small"),
                                        (3, 2, "extruded"), (3, 3, "small"), (2, 3, "large")])
def test_octree_steps(N, lim, kind):
    import torch
    m = octree(kind)
    u = sphere3(m, N) if kind != "extruded" else W.random3_state(m, N, seed=N)
    o = o3d.Oracle3D(m, N)
    u_o, t_o, _, st_o = o.step(u, 20, cfl=0.5, limiting=lim)
    ctx = idp.Context3D(m, N, limiting=lim, cfl=0.5)
    ud = dev(u)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 20, t)
    assert rc == idp.IDP_OK
    torch.cuda.synchronize()
    sc = np.abs(u_o).reshape(5, -1).max(axis=1)
    err = (np.abs(ud.cpu().numpy() - u_o).reshape(5, -1).max(axis=1) / sc).max()
    assert err <= 1e-10, err
    assert abs(t[0] - t_o) <= 1e-12 * t_o
    rc, st = ctx.idp3d_limiter_stats()
    assert rc == idp.IDP_OK
    assert st["n_viol_density"] == 0 and st["n_viol_pressure"] == 0 and st["n_nonpositive"] == 0
    assert st["n_stages"] == 60
    assert (st["n_mortar_active"] > 0) == (st_o["n_mort_active"] > 0)
    ctx.close()


def test_octree_blast_conservation_and_positivity():
    import torch
    N = 3
    m = W.box_refined_mesh3(4, 4, 4, UNIT, (0.3, 0.3, 0.3, 0.7, 0.7, 0.7))
    u = W.blast3_state(m, N, rho_bg=1e-5, p_bg=1e-6, rho_in=1.0, p_in=1e2, centre=(0.45, 0.5, 0.55), r0=0.2)
    ctx = idp.Context3D(m, N, limiting=1, cfl=0.9)
    assert ctx.n_mortars > 0
    ud = dev(u)
    I0 = ctx.idp3d_integrals(ud)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 40, t)
    assert rc == idp.IDP_OK
    I1 = ctx.idp3d_integrals(ud)
    assert np.abs(I1 - I0).max() <= 1e-12 * np.abs(I0).max()
    q = ud.cpu().numpy().reshape(5, -1)
    p = (G - 1.0) * (q[4] - 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0])
    assert q[0].min() > 0.0 and p.min() > 0.0
    rc, st = ctx.idp3d_limiter_stats()
    assert st["n_nonpositive"] == 0 and st["n_viol_pressure"] == 0 and st["n_mortar_active"] > 0
    torch.cuda.synchronize()
    ctx.close()


def test_octree_bad_meshes():
    m = octree("small")
    # a level jump of two across a face: one small child refined again
    k = int(np.flatnonzero(m.level == 1)[0])
    lev, ix, iy, iz = (list(a) for a in (m.level, m.ix, m.iy, m.iz))
    a, b, c = ix.pop(k), iy.pop(k), iz.pop(k)
    lev.pop(k)
    for q in range(8):
        lev.append(2); ix.append(2 * a + (q & 1)); iy.append(2 * b + ((q >> 1) & 1)); iz.append(2 * c + (q >> 2))
    bad = W.Mesh3(3, 3, 3, UNIT, np.array(lev, np.int8), np.array(ix, np.int32), np.array(iy, np.int32),
                  np.array(iz, np.int32))
    with pytest.raises(idp.IdpError):
        idp.Context3D(bad, 2)
    # a gap: one leaf left out
    gap = W.Mesh3(3, 3, 3, UNIT, m.level[1:], m.ix[1:], m.iy[1:], m.iz[1:])
    with pytest.raises(idp.IdpError):
        idp.Context3D(gap, 2)


# ----------------------------------------------------------------------------
# the FP32 form (precision 1): fluxes in FP32, limiter and sums in FP64
# ----------------------------------------------------------------------------

def l1_fields3(u, ref, m):
    """Mass-weighted L1 difference per conserved field relative to the
    reference (momenta against sum m (|ref| + sqrt(rho E)))."""
    u, ref = np.asarray(u).reshape(5, -1), np.asarray(ref).reshape(5, -1)
    ps = np.sqrt(np.abs(ref[0] * ref[4]))
    out = []
    for v in range(5):
        den = (m * np.abs(ref[v])).sum() + ((m * ps).sum() if v in (1, 2, 3) else 0.0)
        out.append(float((m * np.abs(u[v] - ref[v])).sum() / den))
    return out


@pytest.mark.parametrize("N,kind,lim", [(2, "grid", 2), (3, "grid", 2), (4, "grid", 1), (3, "small", 2),
                                        (3, "large", 2), (2, "extruded", 2), (3, "small", 3)])
def test_fp32_form_steps(N, kind, lim):
    """20 SSP-RK3 steps of the FP32 form against the FP64 oracle: density L1
    within 1e-5 and the other fields within 3e-5 (as the 2D FP32 form), no
    bound violation, the time within 2e-5 (its time step is FP32, scaled
    down by 8e-6)."""
    import torch
    if kind == "grid":
        m = grid("walls", n=(3, 3, 2))
        u = W.random3_state(m, N, seed=N, rho_range=(0.5, 2.0), p_range=(0.5, 2.0), vmax=0.5)
    else:
        m = octree(kind)
        u = sphere3(m, N) if kind != "extruded" else W.random3_state(m, N, seed=N)
    o = o3d.Oracle3D(m, N)
    u_o, t_o, _, _ = o.step(u, 20, cfl=0.5, limiting=lim)
    ctx = idp.Context3D(m, N, limiting=lim, cfl=0.5, precision=1)
    ud = dev(u)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 20, t)
    assert rc == idp.IDP_OK
    torch.cuda.synchronize()
    e = l1_fields3(ud.cpu().numpy(), u_o, o.masses())
    assert e[0] <= 1e-5 and max(e[1:]) <= 3e-5, e
    assert abs(t[0] - t_o) <= 2e-5 * t_o
    rc, st = ctx.idp3d_limiter_stats()
    assert st["n_viol_density"] == 0 and st["n_viol_pressure"] == 0 and st["n_nonpositive"] == 0
    ctx.close()


@pytest.mark.parametrize("N", [1, 3, 4])
@pytest.mark.parametrize("kind", ["grid", "small", "large"])
def test_fp32_form_dt_is_safe_and_tight(N, kind):
    """The FP32 form's time step never exceeds the FP64 oracle's and is
    within 2e-5 of it, on random and sphere states."""
    m = grid("dirichlet") if kind == "grid" else octree(kind)
    o = o3d.Oracle3D(m, N)
    ctx = idp.Context3D(m, N, cfl=0.7, precision=1)
    for u in (W.random3_state(m, N, seed=3, rho_range=(0.1, 10.0), p_range=(0.1, 10.0), vmax=2.0),
              sphere3(m, N) if kind != "grid" else W.random3_state(m, N, seed=4)):
        d32, d64 = ctx.idp3d_dt(dev(u)), o.dt(u, cfl=0.7)
        assert d32 <= d64 and d32 >= d64 * (1.0 - 2e-5), (d32, d64)
    ctx.close()


def test_fp32_form_rhs():
    """One limited right-hand side of the FP32 form within 1e-5 of the
    oracle's, relative to the residual scale."""
    m, N = octree("small"), 3
    u = sphere3(m, N)
    o = o3d.Oracle3D(m, N)
    dt_idp = o.dt(u, cfl=1.0)
    sc = scale(u, dt_idp)
    for lim in (0, 2):
        ctx = idp.Context3D(m, N, limiting=lim, precision=1)
        dt = 0.0 if lim == 0 else 0.5 * dt_idp
        e = rel(gpu_rhs(ctx, u, dt), o.rhs(u, dt=dt, limiting=lim), sc)
        assert e <= 1e-5, (lim, e)
        ctx.close()


def test_fp32_form_near_vacuum_blast():
    import torch
    N = 3
    m = W.box_refined_mesh3(4, 4, 4, UNIT, (0.3, 0.3, 0.3, 0.7, 0.7, 0.7))
    u = W.blast3_state(m, N, rho_bg=1e-5, p_bg=1e-6, rho_in=1.0, p_in=1e2, centre=(0.45, 0.5, 0.55), r0=0.2)
    ctx = idp.Context3D(m, N, limiting=1, cfl=0.9, precision=1)
    ud = dev(u)
    I0 = ctx.idp3d_integrals(ud)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 40, t)
    assert rc == idp.IDP_OK
    I1 = ctx.idp3d_integrals(ud)
    assert np.abs(I1 - I0).max() <= 1e-12 * np.abs(I0).max()
    q = ud.cpu().numpy().reshape(5, -1)
    p = (G - 1.0) * (q[4] - 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0])
    assert q[0].min() > 0.0 and p.min() > 0.0
    torch.cuda.synchronize()
    ctx.close()


@pytest.mark.parametrize("seed,N", [(1, 2), (3, 3), (5, 4)])
def test_random_octree_rhs_and_steps(seed, N):
    """Seeded random 2:1 octrees (levels 0..2, level jumps on every face
    orientation): right-hand sides at 1e-12 and 10 steps at 1e-10."""
    import torch
    bc = (o3d.BC_OUTFLOW, o3d.BC_OUTFLOW, o3d.BC_PERIODIC, o3d.BC_PERIODIC, o3d.BC_WALL, o3d.BC_WALL)
    m = W.random_octree3(2, 3, 2, seed=seed, n_refine=4, max_level=2, bc=bc if seed == 5 else (o3d.BC_PERIODIC,) * 6)
    u = W.random3_state(m, N, seed=seed, rho_range=(0.5, 2.0), p_range=(0.5, 2.0), vmax=0.5)
    o = o3d.Oracle3D(m, N)
    dt_idp = o.dt(u, cfl=1.0)
    sc = scale(u, dt_idp)
    for lim in (0, 2):
        ctx = idp.Context3D(m, N, limiting=lim)
        dt = 0.0 if lim == 0 else 0.5 * dt_idp
        e = rel(gpu_rhs(ctx, u, dt), o.rhs(u, dt=dt, limiting=lim), sc)
        assert e <= 1e-12, (lim, e)
        ctx.close()
    u_o, t_o, _, _ = o.step(u, 10, cfl=0.5, limiting=2)
    ctx = idp.Context3D(m, N, limiting=2, cfl=0.5)
    ud = dev(u)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 10, t)
    assert rc == idp.IDP_OK
    torch.cuda.synchronize()
    sc2 = np.abs(u_o).reshape(5, -1).max(axis=1)
    assert (np.abs(ud.cpu().numpy() - u_o).reshape(5, -1).max(axis=1) / sc2).max() <= 1e-10
    ctx.close()


def test_combined_indicator_values():
    """The element kernel's shock indicators (limiting 3) on a sphere state
    take values strictly between 0 and 1 somewhere, and the combined steps
    keep the positivity bounds on an octree near-vacuum blast."""
    import torch
    N = 3
    m = W.box_refined_mesh3(4, 4, 4, UNIT, (0.3, 0.3, 0.3, 0.7, 0.7, 0.7))
    u = W.blast3_state(m, N, rho_bg=1e-5, p_bg=1e-6, rho_in=1.0, p_in=1e2, centre=(0.45, 0.5, 0.55), r0=0.2)
    o = o3d.Oracle3D(m, N)
    u_o, t_o, _, _ = o.step(u, 10, cfl=0.9, limiting=3)
    ctx = idp.Context3D(m, N, limiting=3, cfl=0.9)
    ud = dev(u)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 10, t)
    assert rc == idp.IDP_OK
    torch.cuda.synchronize()
    sc = np.abs(u_o).reshape(5, -1).max(axis=1)
    assert (np.abs(ud.cpu().numpy() - u_o).reshape(5, -1).max(axis=1) / sc).max() <= 1e-10
    rc, st = ctx.idp3d_limiter_stats()
    assert st["n_nonpositive"] == 0 and st["n_viol_pressure"] == 0 and st["n_viol_density"] == 0
    ctx.close()


@pytest.mark.parametrize("kind", ["small", "large"])
def test_stage_factors_read_back(kind):
    """The element kernel's shock indicators (limiting 3) equal the oracle's
    per element, and the mortar factors l_S of one limited stage (limiting
    2 and 3) equal the oracle's."""
    m, N = octree(kind), 2
    u = sphere3(m, N)
    o = o3d.Oracle3D(m, N)
    dt = 0.5 * o.dt(u, cfl=1.0)
    npe = (N + 1) ** 3
    U = u.reshape(5, m.n_elems, npe)
    p = (G - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])
    al = np.array([o3d.indicator3(N, p[e]) for e in range(m.n_elems)])
    for lim in (2, 3):
        ctx = idp.Context3D(m, N, limiting=lim)
        gpu_rhs(ctx, u, dt)
        a_g, ell_g = ctx.idp3d_stage_factors()
        ell_o = o.stage_debug(u, dt, limiting=lim)["mortar_ell"]
        assert np.abs(ell_g - ell_o).max() <= 1e-12, (lim, ell_g, ell_o)
        if lim == 3:
            assert np.abs(a_g - al).max() <= 1e-12
            assert 0.0 < al.mean() < 1.0
        ctx.close()
