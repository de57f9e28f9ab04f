"""3D GPU tests at the benchmark's full sizes, in the configuration bench.py
times (limiting 2, CFL 0.5, N = 3):

- the 40^3 blast: sampled elements of one limited and one unlimited
  right-hand side of the whole grid against the oracle, which evaluates each
  sampled element inside the 3 x 3 x 3 block of its neighbours (an element's
  residual depends only on its face neighbours and the stage's dt, which is
  passed in); FP64 path at 1e-12, FP32 form at 1e-5 of the residual scale;
- the 40^3 blast and the 32^3-base octree blast (1,536 mortars) over 30
  SSP-RK3 steps in both forms: no bound violation, positive density and
  pressure at every node, the totals conserved to 1e-12 while the blast is
  inside the box.
"""
import numpy as np
import pytest

from oracle import o3d
from paper_2607_06045_b300 import build, idp
from paper_2607_06045_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = 1.4
N = 3


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


def blast40():
    g = W.Grid3(40, 40, 40, bc=(W.BC_OUTFLOW,) * 6)
    return g, W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0)


def sub_block(g, u, e):
    """The block of element e and its face neighbours (clipped at the box),
    its state and e's index in it."""
    n = (g.nx, g.ny, g.nz)
    c = (e % g.nx, (e // g.nx) % g.ny, e // (g.nx * g.ny))
    lo = [max(0, c[d] - 1) for d in range(3)]
    hi = [min(n[d] - 1, c[d] + 1) for d in range(3)]
    m = [hi[d] - lo[d] + 1 for d in range(3)]
    x0, y0, z0, x1, y1, z1 = g.box
    h = ((x1 - x0) / g.nx, (y1 - y0) / g.ny, (z1 - z0) / g.nz)
    org = (x0, y0, z0)
    box = tuple(org[d] + lo[d] * h[d] for d in range(3)) + tuple(org[d] + (hi[d] + 1) * h[d] for d in range(3))
    sg = W.Grid3(m[0], m[1], m[2], box=box, bc=g.bc)
    U = np.asarray(u).reshape(5, g.nz, g.ny, g.nx, -1)
    sub = U[:, lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1].reshape(5, -1)
    le = ((c[2] - lo[2]) * m[1] + (c[1] - lo[1])) * m[0] + (c[0] - lo[0])
    return sg, np.ascontiguousarray(sub), le


@pytest.mark.parametrize("prec", [0, 1])
def test_blast40_sampled_rhs(prec):
    import torch
    g, u = blast40()
    ud = dev(u)
    ctx = idp.Context3D(g, N, limiting=2, cfl=0.5, precision=prec)
    dt_idp = ctx.idp3d_dt(ud) / 0.5
    rng = np.random.default_rng(7)
    # sampled elements: random ones, the blast's edge, and the box's corners
    X, Y, Z = W.node_coords3(g, N)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2).reshape(g.n_elems, -1)
    edge = np.flatnonzero((r.min(axis=1) < 0.15) & (r.max(axis=1) > 0.15))
    sample = np.unique(np.concatenate([rng.choice(g.n_elems, 8, replace=False), rng.choice(edge, 8, replace=False),
                                       [0, g.n_elems - 1]]))
    npe = (N + 1) ** 3
    tol = 1e-12 if prec == 0 else 1e-5
    for lim, dt in ((0, 0.0), (2, 0.5 * dt_idp)):
        c2 = idp.Context3D(g, N, limiting=lim, cfl=0.5, precision=prec)
        out = torch.empty_like(ud)
        c2.idp3d_rhs(ud, dt, out)
        torch.cuda.synchronize()
        r_g = out.cpu().numpy().reshape(5, g.n_elems, npe)
        c2.close()
        # per field max |u_v| / dt_idp; the momenta (zero at rest) on the scale sqrt(rho E)
        q = np.abs(u).reshape(5, -1)
        scale = np.maximum(q.max(axis=1), np.sqrt(q[0] * q[4]).max()) / dt_idp
        for e in sample:
            sg, su, le = sub_block(g, u, int(e))
            r_o = o3d.Oracle3D(sg, N).rhs(su, dt=dt, limiting=lim).reshape(5, sg.n_elems, npe)[:, le]
            err = (np.abs(r_g[:, e] - r_o).max(axis=1) / scale).max()
            assert err <= tol, (lim, int(e), err)
    ctx.close()


def invariants(ctx, ud):
    rc, st = ctx.idp3d_limiter_stats()
    assert rc == idp.IDP_OK
    assert st["n_viol_density"] == 0 and st["n_viol_pressure"] == 0 and st["n_nonpositive"] == 0, st
    q = ud.cpu().numpy().reshape(5, -1)
    p = (G - 1.0) * (q[4] - 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0])
    assert np.all(np.isfinite(q)) and q[0].min() > 0.0 and p.min() > 0.0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("mesh", ["grid40", "octree32"])
def test_bench_meshes_30_steps(mesh, prec):
    if mesh == "grid40":
        g, u = blast40()
    else:
        g = W.box_refined_mesh3(32, 32, 32, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), (0.25, 0.25, 0.25, 0.75, 0.75, 0.75),
                                bc=(W.BC_OUTFLOW,) * 6)
        u = W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0)
    ctx = idp.Context3D(g, N, limiting=2, cfl=0.5, precision=prec)
    if mesh == "octree32":
        assert ctx.n_mortars == 1536
    ud = dev(u)
    I0 = ctx.idp3d_integrals(ud)
    t = np.zeros(1)
    rc, _ = ctx.idp3d_step(ud, 30, t)
    assert rc == idp.IDP_OK
    invariants(ctx, ud)
    I1 = ctx.idp3d_integrals(ud)
    # the blast stays inside the box: mass and energy conserved, momentum
    # (zero at the start) on the scale sqrt(2 M E)
    M, E = I0[0], I0[4]
    sc = np.array([M, np.sqrt(2 * M * E), np.sqrt(2 * M * E), np.sqrt(2 * M * E), E])
    assert (np.abs(I1 - I0) / sc).max() <= 1e-12
    ctx.close()


@pytest.mark.parametrize("mesh", ["grid40", "octree32"])
def test_bench_meshes_dt(mesh):
    """The FP64 time step (an FP32 pass that picks the elements, then the
    FP64 quotients in them) equals the oracle's to 1e-13 on the benchmark's
    meshes, on the blast and on a uniform state, where every element ties."""
    if mesh == "grid40":
        g, u = blast40()
    else:
        g = W.box_refined_mesh3(32, 32, 32, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), (0.25, 0.25, 0.25, 0.75, 0.75, 0.75),
                                bc=(W.BC_OUTFLOW,) * 6)
        u = W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0)
    flat = W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=0.1)
    ctx = idp.Context3D(g, N, limiting=2, cfl=0.5)
    o = o3d.Oracle3D(g, N)
    for state in (u, flat):
        d_g, d_o = ctx.idp3d_dt(dev(state)), o.dt(state, cfl=0.5)
        assert abs(d_g - d_o) <= 1e-13 * d_o, (mesh, d_g, d_o)
    ctx.close()
