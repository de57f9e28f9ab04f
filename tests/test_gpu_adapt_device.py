"""The AMR step on the device (Sec. 2.4) against the host builder, through
the C ABI: one `idp_dgsem_adapt` call in a context must give the leaves,
the transferred state, and every mesh table (faces, mortars, mortar nodes,
mortar limiting blocks) that the host plan (`idp_amr_plan`), the host-side
transfer (`idp_amr_transfer`) and a context created for the new leaves
give, element for element, and the steps that follow must be the same bits.

The plan on the host is the reference here: it is a plain serial restatement
of the marking, family and 2:1 balance rules, pinned on the CPU by
tests/test_amr_plan.py and against the oracle's plan in
tests/test_oracle_amr.py.
"""
import numpy as np
import pytest

from oracle import amr
from paper_2607_06045_b300 import build, idp
from paper_2607_06045_b300 import workloads as W

pytestmark = pytest.mark.gpu

TABLES = ("fnbr", "ftype", "m_large", "m_small", "m_info", "mn_node", "mn_slot", "mb_node_off", "mb_for_off",
          "mb_foreign")


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


def noisy_state(mesh, N, seed, gamma=1.4):
    """Density noise whose amplitude is drawn per family of four siblings
    (zero for about a third of them), so that the indicator refines some
    families, coarsens others whole and leaves the rest."""
    rng = np.random.default_rng(seed)
    fam = {}
    amp = np.empty(mesh.n_elems)
    for e, (l, x, y) in enumerate(zip(mesh.level.tolist(), mesh.ix.tolist(), mesh.iy.tolist())):
        k = (l, x >> 1, y >> 1)
        if k not in fam:
            a = rng.uniform(0.0, 0.4)
            fam[k] = 0.0 if a < 0.13 else a
        amp[e] = fam[k]
    sh = (mesh.n_elems, N + 1, N + 1)
    rho = 1.0 + amp[:, None, None] * rng.uniform(-1.0, 1.0, sh)
    return W.conserved(rho, 0.1 * np.ones(sh), -0.05 * np.ones(sh), np.ones(sh), gamma)


def assert_same_mesh(cd, ch, what):
    td, th = cd.mesh_tables(True), ch.mesh_tables(True)
    assert td["sizes"] == th["sizes"], (what, td["sizes"], th["sizes"])
    for k in TABLES:
        assert np.array_equal(td[k], th[k]), (what, k)
    for a, b in zip(cd.leaves(), ch.leaves()):
        assert np.array_equal(a, b), what


def check_cycle(cd, ud, ch, uh, p, steps, what):
    """One adaptation on both paths, then `steps` steps of each: returns the
    two contexts and states for the next cycle."""
    import torch
    ch2, uh2, _, sch = ch.adapt(uh, p)
    ch.close()
    cd.idp_dgsem_limiter_stats()   # read (and reset) the statistics of the old mesh
    ud2, scd = cd.idp_dgsem_adapt(ud, p)
    torch.cuda.synchronize()
    assert cd.K == ch2.K and cd.M == ch2.M, what
    assert scd == sch, what
    assert torch.equal(ud2, uh2), what
    assert_same_mesh(cd, ch2, what)
    ud2 = ud2.clone()
    td, th = np.zeros(1), np.zeros(1)
    if steps:
        cd.idp_dgsem_step(ud2, steps, td)
        ch2.idp_dgsem_step(uh2, steps, th)
        torch.cuda.synchronize()
        assert td[0] == th[0], what
        assert torch.equal(ud2, uh2), what
        # the statistics' normalisers: the device sums the areas and mortar
        # lengths in another order than the host builder
        (_, sd), (_, sh) = cd.idp_dgsem_limiter_stats(), ch2.idp_dgsem_limiter_stats()
        for k in ("alpha_volume_mean", "alpha_mortar_mean"):
            assert sd[k] == pytest.approx(sh[k], rel=1e-12, abs=1e-300), (what, k)
        for k in ("n_stages", "n_volume_active", "n_mortar_active", "n_viol_density", "n_viol_pressure"):
            assert sd[k] == sh[k], (what, k)
    return ch2, ud2, uh2


CASES = {
    # periodic refined square, the disc's jump: refinement around it
    "square_disc": (W.square_mesh, lambda m, N: W.disc_wave_state(m, N),
                    dict(indicator=amr.IND_MAX, refine_threshold=0.2, coarsen_threshold=0.02, max_level=2)),
    # three levels of a refined box, noise per family: refine, coarsen and
    # the balance sweeps that undo coarsening and force refinement
    "box_noise": (lambda: W.box_refined_mesh(8, 8, (0.0, 0.0, 1.0, 1.0), (0.25, 0.25, 0.75, 0.75), base_level=1),
                  lambda m, N: noisy_state(m, N, 3),
                  dict(indicator=amr.IND_HENNEMANN, refine_threshold=0.35, coarsen_threshold=0.25, min_level=0,
                       max_level=4)),
    # outflow / reflecting boundaries of the DMR sample mesh
    "dmr_sample": (W.dmr_sample_mesh, lambda m, N: W.dmr_state(m, N),
                   dict(indicator=amr.IND_MAX, refine_threshold=0.3, coarsen_threshold=0.01, max_level=4)),
}


@pytest.mark.parametrize("precision,limiting", [(0, 2), (1, 2), (0, 3)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_device_adapt_equals_host(case, precision, limiting):
    mk, st, pk = CASES[case]
    m = mk()
    N = 3
    u = st(m, N)
    p = idp.amr_params(**pk)
    cd = idp.Context(m, N, precision=precision, limiting=limiting, cfl=0.5)
    ch = idp.Context(m, N, precision=precision, limiting=limiting, cfl=0.5)
    ud, uh = dev(u), dev(u)
    ch, ud, uh = check_cycle(cd, ud, ch, uh, p, 3, case)
    cd.close()
    ch.close()


def test_cycles_grow_and_shrink():
    """Four cycles of (device adapt, 5 steps) against the host path on the
    noise case: the mesh grows past the context's buffers and shrinks back,
    and every cycle stays bit-identical."""
    mk, st, pk = CASES["box_noise"]
    m = mk()
    N = 3
    u = st(m, N)
    cd = idp.Context(m, N, limiting=2, cfl=0.5)
    ch = idp.Context(m, N, limiting=2, cfl=0.5)
    ud, uh = dev(u), dev(u)
    sizes = [cd.K]
    for cyc, kw in enumerate([dict(refine_threshold=0.2, coarsen_threshold=0.0, max_level=4),
                              dict(refine_threshold=0.2, coarsen_threshold=0.0, max_level=5),
                              dict(refine_threshold=2.0, coarsen_threshold=0.9, min_level=0),
                              dict(refine_threshold=0.1, coarsen_threshold=0.0, max_level=5)]):
        p = idp.amr_params(indicator=amr.IND_HENNEMANN, **kw)
        ch, ud, uh = check_cycle(cd, ud, ch, uh, p, 5, f"cycle {cyc}")
        sizes.append(cd.K)
    assert sizes[1] > sizes[0] and sizes[3] < sizes[2] and sizes[4] > sizes[3], sizes
    cd.close()
    ch.close()


def test_dmr_sized_plan():
    """The DMR workload mesh (about 60 000 leaves, levels 0..3 over a 256 x 64
    base grid) adapted once with the benchmark's parameters."""
    m = W.dmr_mesh()
    N = 3
    u = W.dmr_state(m, N)
    p = idp.amr_params(indicator=amr.IND_MAX, refine_threshold=0.3, coarsen_threshold=0.01, min_level=0,
                       max_level=4)
    cd = idp.Context(m, N, limiting=2, cfl=0.5)
    ch = idp.Context(m, N, limiting=2, cfl=0.5)
    ud, uh = dev(u), dev(u)
    ch, ud, uh = check_cycle(cd, ud, ch, uh, p, 2, "dmr")
    cd.close()
    ch.close()


def test_capacity_too_small_leaves_the_context():
    import torch
    m = W.square_mesh()
    N = 3
    u = W.disc_wave_state(m, N)
    p = idp.amr_params(indicator=amr.IND_MAX, refine_threshold=0.2, coarsen_threshold=0.0, max_level=2)
    cd = idp.Context(m, N, limiting=2, cfl=0.5)
    ch = idp.Context(m, N, limiting=2, cfl=0.5)
    ud = dev(u)
    before = cd.mesh_tables(True)
    with pytest.raises(ValueError):
        cd.idp_dgsem_adapt(ud, p, capacity=m.n_elems)
    assert cd.K == m.n_elems
    after = cd.mesh_tables(True)
    for k in TABLES:
        assert np.array_equal(before[k], after[k]), k
    uh = dev(u)
    td, th = np.zeros(1), np.zeros(1)
    cd.idp_dgsem_step(ud, 3, td)
    ch.idp_dgsem_step(uh, 3, th)
    torch.cuda.synchronize()
    assert torch.equal(ud, uh)
    cd.close()
    ch.close()


def test_batch_contexts_are_refused():
    ms = W.batch_meshes(2)
    ctx = idp.Context(ms, 3)
    u = dev(W.concat_states([W.disc_wave_state(mm, 3) for mm in ms]))
    with pytest.raises(idp.IdpError):
        ctx.idp_dgsem_adapt(u, idp.amr_params())
    ctx.close()
