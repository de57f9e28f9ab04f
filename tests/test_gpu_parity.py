"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

Tolerances (FP64 path): per right-hand side 1e-12 relative to the residual
scale max|u_v| / dt_idp (the change of u over one IDP step, see
conftest.rhs_scale) and 1e-12 element by element relative to each element's
own residual scale (conftest.local_rhs_err); after 100 SSP-RK3 steps 1e-10
relative to max|u_v|.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import rel_err, rhs_scale, assert_l1_fields, local_rhs_err
from paper_2607_06045_b300 import build, idp
from paper_2607_06045_b300 import workloads as W

pytestmark = pytest.mark.gpu


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


def gpu_rhs(ctx, u, t, dt):
    import torch
    ud = dev(u)
    out = torch.empty_like(ud)
    ctx.idp_dgsem_rhs(ud, t, dt, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_rhs(mesh, N, u, limiting, t=0.0, cfl=0.5, gamma=1.4, tol=1e-12, precision=0, **kw):
    o = oracle.Oracle(mesh, N, gamma=gamma)
    ctx = idp.Context(mesh, N, gamma=gamma, limiting=limiting, precision=precision, **kw)
    dt_idp = o.dt(u, t, cfl=1.0)
    scale = rhs_scale(u, dt_idp)
    r_o = o.rhs(u, t=t, dt=0.0)
    r_g = gpu_rhs(ctx, u, t, 0.0)
    e0 = rel_err(r_g, r_o, scale)
    assert e0 <= tol, ("dg", e0)
    # element by element against each element's own residual scale
    l0 = local_rhs_err(r_g, r_o, u, mesh, N, gamma)
    assert l0 <= tol, ("dg, per element", l0)
    if limiting:
        dt = cfl * dt_idp
        r_o = o.rhs(u, t=t, dt=dt, limiting=limiting)
        r_g = gpu_rhs(ctx, u, t, dt)
        e1 = rel_err(r_g, r_o, scale)
        assert e1 <= tol, ("limited", e1)
        l1 = local_rhs_err(r_g, r_o, u, mesh, N, gamma)
        assert l1 <= tol, ("limited, per element", l1)
    ctx.close()


@pytest.mark.parametrize("limiting", [1, 2])
def test_square_rhs(limiting):
    m = W.square_mesh()
    check_rhs(m, 3, W.disc_wave_state(m, 3), limiting)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_degrees_rough_state(N):
    m = W.box_refined_mesh(5, 4, (0.0, 0.0, 1.25, 1.0), (0.3, 0.3, 0.8, 0.7))
    u = W.random_state(m, N, seed=N, rho_range=(0.2, 3.0), p_range=(0.2, 3.0), vmax=1.0)
    check_rhs(m, N, u, 2)


@pytest.mark.parametrize("N", [3, 4, 7])
def test_degrees_smooth_state_positivity(N):
    m = W.box_refined_mesh(6, 6, (0.0, 0.0, 1.0, 1.0), (0.2, 0.2, 0.6, 0.5))
    check_rhs(m, N, W.smooth_random_state(m, N, seed=10 + N), 1)


@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_DIRICHLET, W.BC_OUTFLOW])
def test_boundaries(bc):
    m = W.box_refined_mesh(5, 3, (0.0, 0.0, 2.0, 1.0), (0.5, 0.3, 1.5, 0.7), bc=(bc,) * 4)
    m.bc_prim = np.array([[1.2, 0.3, -0.1, 1.1], [0.9, 0.1, 0.2, 0.8], [1.0, -0.2, 0.3, 1.0], [1.1, 0.0, 0.0, 0.9]])
    u = W.random_state(m, 3, seed=7 + bc)
    check_rhs(m, 3, u, 2)


def test_dmr_boundaries():
    m = W.box_refined_mesh(16, 4, (0.0, 0.0, 4.0, 1.0), (0.0, 0.0, 1.0, 0.5), bc=(W.BC_DMR,) * 4)
    m.dmr_post = W.DMR_POST.copy()
    m.dmr_pre = W.DMR_PRE.copy()
    u = W.dmr_state(m, 3)
    for t in (0.0, 0.05):
        check_rhs(m, 3, u, 2, t=t)


def test_dt_parity():
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    o = oracle.Oracle(m, 3)
    for rule in (0, 1):
        ctx = idp.Context(m, 3, dt_rule=rule, cfl=0.7)
        d = ctx.idp_dgsem_dt(dev(u))[0]
        assert abs(d - o.dt(u, cfl=0.7, rule=rule)) <= 1e-13 * d
        ctx.close()


def test_fp32_form_dt_is_safe_and_tight():
    """The FP32 form's time step (FP32 wave speeds and quotient, scaled by
    1 - 4e-6) never exceeds the IDP restriction the oracle forms in FP64 and
    stays within 2e-5 of it, on states with mortars, walls, inflow and
    outflow boundaries and several simulations."""
    cases = []
    sq = W.square_mesh()
    cases.append(([sq], 3, [W.disc_wave_state(sq, 3)]))
    dm = W.dmr_sample_mesh()
    cases.append(([dm], 3, [W.dmr_state(dm, 3)]))
    cases.append(([sq], 5, [W.random_state(sq, 5, seed=3, rho_range=(0.1, 10.0), p_range=(0.1, 10.0), vmax=2.0)]))
    ms = W.batch_meshes(256, seed=0)
    small = np.argsort([mm.n_elems for mm in ms])[:3].tolist()
    rng = np.random.default_rng(1)
    us = [W.riemann4_state(mm, 3, rng) for mm in ms]
    cases.append(([ms[k] for k in small], 3, [us[k] for k in small]))
    for meshes, N, states in cases:
        ctx = idp.Context(meshes if len(meshes) > 1 else meshes[0], N, precision=1, cfl=0.5)
        d32 = ctx.idp_dgsem_dt(dev(W.concat_states(states)))
        ctx.close()
        for k, (m, u) in enumerate(zip(meshes, states)):
            d64 = oracle.Oracle(m, N).dt(u, cfl=0.5)
            assert d32[k] <= d64, (N, k, d32[k], d64)
            assert d32[k] >= d64 * (1.0 - 2e-5), (N, k, d32[k], d64)


def test_fp64_two_pass_dt_is_the_one_pass_dt():
    """The FP64 path's time step runs an FP32 pass that picks the elements
    whose quotients the FP64 pass forms. Its result equals, bit for bit, the
    one-pass FP64 time step of the extended kernel's context (which forms
    every node's FP64 quotient), and the oracle's to 1e-13: with mortars,
    walls, inflow and outflow, a uniform state (every element ties), several
    simulations and the full DMR mesh."""
    cases = []
    sq = W.square_mesh()
    cases.append(([sq], 3, [W.disc_wave_state(sq, 3)]))
    cases.append(([sq], 3, [W.random_state(sq, 3, seed=1, rho_range=(1.0, 1.0), p_range=(1.0, 1.0), vmax=0.0)]))
    dm = W.dmr_sample_mesh()
    cases.append(([dm], 3, [W.dmr_state(dm, 3)]))
    cases.append(([sq], 5, [W.random_state(sq, 5, seed=3, rho_range=(0.1, 10.0), p_range=(0.1, 10.0), vmax=2.0)]))
    ms = W.batch_meshes(256, seed=0)
    small = np.argsort([mm.n_elems for mm in ms])[:3].tolist()
    rng = np.random.default_rng(1)
    us = [W.riemann4_state(mm, 3, rng) for mm in ms]
    cases.append(([ms[k] for k in small], 3, [us[k] for k in small]))
    full = W.dmr_mesh()
    cases.append(([full], 3, [W.dmr_state(full, 3)]))
    for meshes, N, states in cases:
        mesh = meshes if len(meshes) > 1 else meshes[0]
        ud = dev(W.concat_states(states))
        two = idp.Context(mesh, N, cfl=0.5, limiting=2)
        one = idp.Context(mesh, N, cfl=0.5, limiting=2, entropy_bound=1)   # no face buffer: one FP64 pass
        d2, d1 = two.idp_dgsem_dt(ud), one.idp_dgsem_dt(ud)
        assert np.array_equal(d2, d1), (N, len(meshes), d2, d1)
        two.close()
        one.close()
        for k, (m, u) in enumerate(zip(meshes, states)):
            d64 = oracle.Oracle(m, N).dt(u, cfl=0.5)
            assert abs(d2[k] - d64) <= 1e-13 * d64, (N, k, d2[k], d64)


@pytest.mark.parametrize("limiting", [1, 2])
def test_square_100_steps(limiting):
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    o = oracle.Oracle(m, 3)
    u_o, t_o, dts, st = o.step(u, 100, cfl=0.5, limiting=limiting)
    ctx = idp.Context(m, 3, limiting=limiting, cfl=0.5)
    ud = dev(u)
    t = np.zeros(1)
    ctx.idp_dgsem_step(ud, 100, t)
    u_g = ud.cpu().numpy()
    scale = np.abs(u_o).reshape(4, -1).max(axis=1)
    err = (np.abs(u_g - u_o).reshape(4, -1).max(axis=1) / scale).max()
    assert err <= 1e-10, err
    assert abs(t[0] - t_o) <= 1e-12 * t_o
    rc, s = ctx.idp_dgsem_limiter_stats()
    assert rc == idp.IDP_OK
    assert s["n_viol_density"] == 0 and s["n_viol_pressure"] == 0 and s["n_nonpositive"] == 0
    assert s["n_stages"] == 300
    ctx.close()


def test_epb_invariance():
    import torch
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    dt = oracle.Oracle(m, 3).dt(u, cfl=0.5)
    outs = []
    for epb in (1, 2, 4, 8, 16):
        ctx = idp.Context(m, 3, elems_per_block=epb)
        outs.append(gpu_rhs(ctx, u, 0.0, dt))
        ctx.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_batched_matches_individual():
    ms = [W.square_mesh(), W.box_refined_mesh(6, 4, (0.0, 0.0, 1.5, 1.0), (0.2, 0.2, 0.9, 0.6)),
          W.uniform_mesh(5, 5, bc=(W.BC_OUTFLOW,) * 4)]
    us = [W.disc_wave_state(ms[0], 3), W.smooth_random_state(ms[1], 3, seed=3), W.random_state(ms[2], 3, seed=4)]
    ctx = idp.Context(ms, 3, cfl=0.5)
    ub = W.concat_states(us)
    ud = dev(ub)
    t = np.zeros(3)
    ctx.idp_dgsem_step(ud, 5, t)
    u_g = ud.cpu().numpy()
    off = ctx.sim_offsets
    for s in range(3):
        o = oracle.Oracle(ms[s], 3)
        u_o, t_o, _, _ = o.step(us[s], 5, cfl=0.5)
        part = u_g[:, off[s]:off[s + 1]]
        scale = np.abs(u_o).reshape(4, -1).max(axis=1)
        err = (np.abs(part - u_o).reshape(4, -1).max(axis=1) / scale).max()
        assert err <= 1e-11, (s, err)
        assert abs(t[s] - t_o) <= 1e-12 * t_o
    ctx.close()


def test_conservation_and_free_stream():
    import torch
    m = W.square_mesh()
    sh = (m.n_elems, 4, 4)
    uf = W.conserved(1.3 * np.ones(sh), 0.4 * np.ones(sh), -0.7 * np.ones(sh), 2.0 * np.ones(sh), 1.4)
    ctx = idp.Context(m, 3)
    r = gpu_rhs(ctx, uf, 0.0, 0.0)
    mm = oracle.Oracle(m, 3).masses()
    assert np.abs(r).max() < 1e-12 * 3.0 / mm.min()
    u = W.disc_wave_state(m, 3)
    ud = dev(u)
    I0 = ctx.idp_dgsem_integrals(ud)[0]
    t = np.zeros(1)
    ctx.idp_dgsem_step(ud, 50, t)
    I1 = ctx.idp_dgsem_integrals(ud)[0]
    scale = (mm[None] * np.abs(u)).reshape(4, -1).sum(axis=1)
    assert (np.abs(I1 - I0) / scale).max() <= 1e-13
    ctx.close()


def test_invalid_state_reported():
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    u[0, 5, 1, 1] = -1.0
    ctx = idp.Context(m, 3)
    ud = dev(u)
    t = np.zeros(1)
    rc, _ = ctx.idp_dgsem_step(ud, 1, t, check=False)
    assert rc == idp.IDP_E_STATE
    ctx.close()


def test_step_host_equals_device():
    import torch
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    ctx = idp.Context(m, 3)
    ud = dev(u)
    t1 = np.zeros(1)
    ctx.idp_dgsem_step(ud, 3, t1)
    uh = torch.from_numpy(u.copy()).pin_memory()
    t2 = np.zeros(1)
    ctx.idp_dgsem_step_host(uh, 3, t2)
    assert np.array_equal(uh.numpy(), ud.cpu().numpy())
    assert t1[0] == t2[0]
    ctx.close()


def test_dmr_full_size_rhs():
    """Full-size DMR workload (about 60k elements) in the benchmark's launch
    configuration: the limited right-hand side on every node."""
    m = W.dmr_mesh()
    u = W.dmr_state(m, 3)
    check_rhs(m, 3, u, 2)


def test_fp32_form_error_high_degree():
    """FP32 form (flux arithmetic in FP32, limiter and sums in FP64) against the
    FP64 oracle: density L1 error and zero positivity violations."""
    m = W.square_mesh()
    for N in (4, 7):
        u = W.disc_wave_state(m, N)
        o = oracle.Oracle(m, N)
        nst = 20
        u_o, t_o, _, _ = o.step(u, nst, cfl=0.5)
        ctx = idp.Context(m, N, precision=1, cfl=0.5)
        ud = dev(u)
        t = np.zeros(1)
        ctx.idp_dgsem_step(ud, nst, t)
        u_g = ud.cpu().numpy()
        mm = o.masses()
        assert_l1_fields(u_g, u_o, mm, what=N)
        rc, s = ctx.idp_dgsem_limiter_stats()
        assert s["n_nonpositive"] == 0 and s["n_viol_pressure"] == 0
        ctx.close()


def test_ragged_tails_every_launch_shape():
    """An element count that no block size divides (a 7 x 5 base with a refined
    box): every elements-per-block choice, one block per batch and persistent
    grids give the same bits, and the FP64 path matches the oracle."""
    m = W.box_refined_mesh(7, 5, (0.0, 0.0, 1.4, 1.0), (0.3, 0.2, 0.9, 0.7))
    assert m.n_elems % 2 == 1
    u = W.smooth_random_state(m, 3, seed=11)
    o = oracle.Oracle(m, 3)
    dt = o.dt(u, cfl=0.5)
    r_o = o.rhs(u, t=0.0, dt=dt, limiting=2)
    scale = rhs_scale(u, o.dt(u, cfl=1.0))
    for prec in (0, 1):
        outs = []
        for epb in (1, 2, 4, 8, 16):
            for gm in (1, 2):
                ctx = idp.Context(m, 3, precision=prec, elems_per_block=epb, grid_mode=gm)
                outs.append(gpu_rhs(ctx, u, 0.0, dt))
                e, p, g = ctx.idp_dgsem_launch_config()
                nb = -(-m.n_elems // epb)
                assert (e, p) == (epb, 1 if gm == 2 else 0)
                assert g == nb if gm == 1 else 1 <= g <= nb
                ctx.close()
        for r in outs[1:]:
            assert np.array_equal(r, outs[0])
        if prec == 0:
            assert rel_err(outs[0], r_o, scale) <= 1e-12


def test_autotuned_step_launch_config():
    """An autotuned context reports no launch before its first call and one
    of the candidates after it; its steps equal, bit for bit, those of a
    context with another fixed launch."""
    import torch
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    ctx = idp.Context(m, 3, limiting=2, cfl=0.5)
    assert ctx.idp_dgsem_launch_config() == (0, 0, 0)
    ua, ta = dev(u), np.zeros(1)
    ctx.idp_dgsem_step(ua, 3, ta)
    e, p, g = ctx.idp_dgsem_launch_config()
    assert e in (1, 2, 4, 8, 16) and p in (0, 1) and g >= 1
    other = 16 if e != 16 else 8
    fixed = idp.Context(m, 3, limiting=2, cfl=0.5, elems_per_block=other, grid_mode=1)
    ub, tb = dev(u), np.zeros(1)
    fixed.idp_dgsem_step(ub, 3, tb)
    torch.cuda.synchronize()
    assert fixed.idp_dgsem_launch_config() == (other, 0, -(-m.n_elems // other))
    assert ta[0] == tb[0]
    assert np.array_equal(ua.cpu().numpy(), ub.cpu().numpy())
    ctx.close()
    fixed.close()


def test_single_element_periodic():
    """One element whose four faces are its own neighbours (periodic 1 x 1)."""
    m = W.uniform_mesh(1, 1)
    u = W.smooth_random_state(m, 4, seed=5)
    check_rhs(m, 4, u, 2)
    o = oracle.Oracle(m, 4)
    u_o, t_o, _, _ = o.step(u, 10, cfl=0.5)
    ctx = idp.Context(m, 4, cfl=0.5)
    ud = dev(u)
    t = np.zeros(1)
    ctx.idp_dgsem_step(ud, 10, t)
    sc = np.abs(u_o).reshape(4, -1).max(axis=1)
    assert (np.abs(ud.cpu().numpy() - u_o).reshape(4, -1).max(axis=1) / sc).max() <= 1e-10
    ctx.close()


@pytest.mark.parametrize("N", [1, 3, 5])
def test_combined_limiting_rhs(N):
    """Combined positivity/local limiting (Sec. 3.5): the limited right-hand
    side on the refined-square data, whose jump makes the shock indicator vary."""
    m = W.square_mesh()
    check_rhs(m, N, W.disc_wave_state(m, N), 3)


def test_combined_limiting_dmr_full_size():
    m = W.dmr_mesh()
    check_rhs(m, 3, W.dmr_state(m, 3), 3)


def test_combined_limiting_steps():
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    o = oracle.Oracle(m, 3)
    u_o, t_o, _, st_o = o.step(u, 100, cfl=0.5, limiting=3)
    ctx = idp.Context(m, 3, limiting=3, cfl=0.5)
    ud = dev(u)
    t = np.zeros(1)
    ctx.idp_dgsem_step(ud, 100, t)
    sc = np.abs(u_o).reshape(4, -1).max(axis=1)
    assert (np.abs(ud.cpu().numpy() - u_o).reshape(4, -1).max(axis=1) / sc).max() <= 1e-10
    rc, st = ctx.idp_dgsem_limiter_stats()
    assert st["n_nonpositive"] == 0 and st["n_viol_density"] == 0 and st["n_viol_pressure"] == 0
    ctx.close()
    # FP32 form of the same run
    c32 = idp.Context(m, 3, limiting=3, cfl=0.5, precision=1)
    ud = dev(u)
    t = np.zeros(1)
    c32.idp_dgsem_step(ud, 20, t)
    u20, _, _, _ = o.step(u, 20, cfl=0.5, limiting=3)
    mm = o.masses()
    assert_l1_fields(ud.cpu().numpy(), u20, mm)
    c32.close()


def test_combined_limiting_reduces_to_positivity_on_smooth_data():
    m = W.density_wave_mesh(2)
    u = W.density_wave_state(m, 3)
    dt = 0.5 * oracle.Oracle(m, 3).dt(u, cfl=1.0)
    outs = []
    for lim in (1, 3):
        ctx = idp.Context(m, 3, limiting=lim)
        outs.append(gpu_rhs(ctx, u, 0.0, dt))
        ctx.close()
    assert np.array_equal(outs[0], outs[1])
