"""Host logic of bench.py's multi-process path, on CPU with the gloo backend
(world size 2): barrier, max over ranks and the whole-job aggregation, plus the
parsing of the clock samples."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    barrier_sync, max_over_ranks = bench.dist_helpers(dist, "cpu")
    barrier_sync()
    t = max_over_ranks(times[rank])
    units = 962224 * 3 * 10
    out[rank] = (t, bench.aggregate_rate(units, world, t))
    barrier_sync()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    world, port = 2, _free_port()
    times = [0.5, 0.8]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == pytest.approx(0.8)
        assert v == pytest.approx(world * 962224 * 3 * 10 / 0.8)


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard_sims(256, rank, world)
    out[rank] = (mine, bench.sum_over_ranks(dist, "cpu", len(mine) * 10))
    dist.destroy_process_group()


def test_batched_shards_gloo():
    """The batched workload's simulations split across two ranks: disjoint,
    complete, balanced, and the node totals sum over the ranks."""
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    a, b = res[0][0], res[1][0]
    assert not set(a) & set(b) and sorted(a + b) == list(range(256)) and len(a) == len(b) == 128
    assert res[0][1] == res[1][1] == 2560
    assert bench.shard_sims(256, 0, 1) == list(range(256))


def test_single_process_helpers():
    barrier_sync, max_over_ranks = bench.dist_helpers(None, "cpu")
    barrier_sync()
    assert max_over_ranks(1.25) == 1.25
    assert bench.aggregate_rate(100, 1, 2.0) == 50.0


def test_clock_parse():
    lines = ["0, 2032, 2032, 700.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 2032, 2032, 900.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 1980, 2032, 1000.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "garbage"]
    ck = bench.Clocks.parse(lines)
    assert ck["samples"] == 3
    assert ck["sm_mhz"] == 2032.0 and ck["sm_max_mhz"] == 2032.0
    assert ck["reasons"] == ["sw_power_cap"]
    assert bench.Clocks.parse([])["samples"] == 0


def test_reference_arm_json_contract():
    """`bench.py --impl reference` (the oracle on the host, no GPU) prints one
    JSON line with the contract's keys, its own cpu_baseline and an e2e entry
    without host-device copies."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] >= 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "DOF-updates/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert "workload" in d["config"]
