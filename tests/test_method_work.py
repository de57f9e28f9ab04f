"""The method's work from the oracle's op-counting build (the roofline
numerator of the benchmark).

- The counted build runs the oracle's own arithmetic: one SSP-RK3 step gives
  the plain oracle's bits.
- Each distinct evaluation counts once, by node identity, not by value: on
  a uniform state (every node equal) node preparation still counts its seven
  divisions, one square root and two absolute values per node and stage
  (velocity 2, pressure 1, sound speed 1, rho/p 1, wave speeds along x and y
  1 each), and the volume flux row counts two log-mean branch decisions per
  unordered pair of nodes in a row or column, 2N per node.
- The stored work table (written by `python -m oracle.opcount`) is what the
  counting build gives now for the benchmark's degree.
- The benchmark's kernel split of the table keeps every row once.
"""
import json

import numpy as np
import pytest

import oracle
from oracle import opcount as OC
from paper_2607_06045_b300 import roofline as R
from paper_2607_06045_b300 import workloads as W

G = 1.4


@pytest.mark.parametrize("N", [1, 3])
def test_counted_step_is_the_oracle(N):
    m = W.square_mesh()
    u = W.disc_wave_state(m, N)
    _, u1 = OC.count_step(m, N, u)
    u2, *_ = oracle.Oracle(m, N).step(u, 1, cfl=0.5, limiting=2)
    assert np.array_equal(u1.reshape(u2.shape), u2)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_counts_by_identity_not_value(N):
    m = W.box_refined_mesh(6, 6, (0.0, 0.0, 1.0, 1.0), (0.3, 0.3, 0.7, 0.7))
    sh = (m.n_elems, N + 1, N + 1)
    u = W.conserved(1.3 * np.ones(sh), 0.4 * np.ones(sh), -0.2 * np.ones(sh), 2.0 * np.ones(sh), G)
    c, _ = OC.count_step(m, N, u)
    pn = OC.per_node_stage(c, m.n_elems * (N + 1) ** 2)
    assert pn["node_prep"]["div"] == pytest.approx(7.0, abs=1e-12)
    assert pn["node_prep"]["sqrt"] == pytest.approx(1.0, abs=1e-12)
    assert pn["node_prep"]["abs"] == pytest.approx(2.0, abs=1e-12)
    assert pn["volume_flux"]["cmp"] == pytest.approx(2.0 * N, abs=1e-12)


def test_stored_table_matches_the_counting_build():
    table = R.method_table()
    m = W.dmr_sample_mesh()
    assert table["elements"] == m.n_elems
    N = 3
    c, _ = OC.count_step(m, N, W.dmr_state(m, N))
    pn = OC.per_node_stage(c, m.n_elems * (N + 1) ** 2)
    stored = table["degrees"][str(N)]["rows"]
    for r in OC.ROWS:
        assert stored[r]["flops"] == pytest.approx(round(OC.flops(pn[r]), 3), abs=1e-3), r
    assert table["degrees"][str(N)]["method_flops_per_node_stage"] == pytest.approx(
        sum(stored[r]["flops"] for r in OC.METHOD_ROWS), abs=1e-2)


@pytest.mark.parametrize("precision", [0, 1])
def test_kernel_split_keeps_every_row_once(precision):
    N, K = 3, 1000
    rows = R.method_rows(N)
    work = R.method_kernel_work(N, precision, K)
    total = sum(a + b for a, b in work.values())
    expect = sum(rows[r] for r in OC.METHOD_ROWS) * K * (N + 1) ** 2
    assert total == pytest.approx(expect, rel=1e-12)
    f64, f32 = R.method_flops(N, OC.METHOD_ROWS, precision)
    if precision == 0:
        assert f32 == 0
    else:
        assert f32 == pytest.approx(sum(rows[r] for r in R.FP32_FORM_FP32_ROWS), rel=1e-12)


def test_counted_3d_step_is_the_oracle():
    from oracle import o3d
    g = W.Grid3(3, 3, 2, bc=(3,) * 6)
    N = 3
    u = W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0, centre=(0.4, 0.5, 0.5), r0=0.3)
    _, u1 = OC.count_step3(g, N, u)
    u2, *_ = o3d.Oracle3D(g, N).step(u, 1, cfl=0.5, limiting=2)
    assert np.array_equal(u1.reshape(u2.shape), u2)


def test_stored_3d_table_matches_the_counting_build():
    t3 = R.method_table()["3d"]
    n = round(t3["elements"] ** (1.0 / 3.0))
    assert n ** 3 == t3["elements"]
    g = W.Grid3(n, n, n, bc=(3,) * 6)
    N = 2
    c, _ = OC.count_step3(g, N, W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0))
    pn = OC.per_node_stage(c, g.n_elems * (N + 1) ** 3)
    stored = t3["degrees"][str(N)]["rows"]
    for r in OC.ROWS:
        assert stored[r]["flops"] == pytest.approx(round(OC.flops(pn[r]), 3), abs=1e-3), r


def test_counted_3d_octree_step_is_the_oracle():
    from oracle import o3d
    m = W.box_refined_mesh3(4, 4, 4, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), (0.25, 0.25, 0.25, 0.75, 0.75, 0.75),
                            bc=(3,) * 6)
    N = 2
    u = W.blast3_state(m, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0, centre=(0.4, 0.5, 0.5), r0=0.3)
    _, u1 = OC.count_step3(m, N, u)
    u2, *_ = o3d.Oracle3D(m, N).step(u, 1, cfl=0.5, limiting=2)
    assert np.array_equal(u1.reshape(u2.shape), u2)


def test_stored_3d_octree_table_matches_the_counting_build():
    t = R.method_table()["3d_octree"]
    fresh = OC.work_table3_octree(degrees=(1,))
    assert fresh["elements"] == t["elements"]
    a, b = t["degrees"]["1"], fresh["degrees"]["1"]
    for k in ("node_flops_per_node_stage", "mortar_flops_per_mortar_stage", "mortars", "nodes"):
        assert a[k] == pytest.approx(b[k], abs=1e-3), k


def test_mortar_rows_scale_with_the_mortar_count():
    # the table's mortar rows are per node of its own mesh: on that mesh
    # (its elements and mortars) the per-mortar form gives the same work, and
    # on another mesh it follows the mortar count, not the node count
    t = R.method_table()
    assert t["mortars"] == oracle.Oracle(W.dmr_sample_mesh(), 1).n_mortars
    N, Kt, Mt = 3, t["elements"], t["mortars"]
    a = R.method_kernel_work(N, 0, Kt)
    b = R.method_kernel_work(N, 0, Kt, M=Mt)
    for k in a:
        assert b[k] == pytest.approx(a[k], rel=1e-12), k
    c = R.method_kernel_work(N, 0, 10 * Kt, M=Mt)
    for k in R.MORTAR_KERNELS:
        assert c[k] == pytest.approx(a[k], rel=1e-12), k
    assert c["element"][0] == pytest.approx(10 * a["element"][0], rel=1e-12)
