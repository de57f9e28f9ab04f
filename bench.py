"""Benchmark: IDP-DGSEM DOF-updates/s per RK stage on B300.

One benchmark step is one SSP-RK3 step of the whole hot path (time step,
three limited stages, each with mortar fluxes, the element pass and mortar
limiting) over the workload's state, which is resident in HBM. The default
workload is the double-Mach-reflection mesh (256 x 64 base, up to three
extra levels along the shock, about 60k elements, N = 3, FP64, local
limiting). The same JSON line also carries the FP32 form on that workload and
the batched workload (256 simulations, FP32 form).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the reference arm of this build) on a
1/16-size instance of the same DMR workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IDP-DGSEM DOF-updates/s per RK stage (FP64 vs FP32 form, batched); % roofline"
UNIT = "DOF-updates/s"
L2_BYTES = 126 * 2 ** 20


def rank_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def build_workload(name):
    from paper_2607_06045_b300 import workloads as W
    if name == "dmr":
        m = W.cfg2_mesh()
        return [m], W.cfg2_state(m, 3)
    if name == "batched":
        ms = W.cfg4_meshes(256, seed=0)
        rng = np.random.default_rng(1)
        return ms, W.concat_states([W.cfg4_state(m, 3, rng) for m in ms])
    raise ValueError(name)


def time_steps(ctx, u_dev, steps, warmup, flush, stream, sync_fn, clocks=None):
    """Per-step CUDA-event timing on the launching stream, L2 flushed between
    steps. Pass 1 (the headline): CUDA-graph steps bracketed by events. Pass 2:
    the same number of steps launched kernel by kernel with events around each
    element pass (the roofline's kernel duration)."""
    import torch
    t = np.zeros(ctx.n_sims)
    for _ in range(warmup):
        ctx.idp_dgsem_step(u_dev, 1, t, stream=stream.cuda_stream)
    out = []
    for mode in (1, 2):
        ctx.idp_dgsem_profile(mode)
        ctx.idp_dgsem_profile_read(reset=True)
        sync_fn()
        if clocks and mode == 1:
            clocks.start()
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()          # L2 flush, outside the timed span
            ctx.idp_dgsem_step(u_dev, 1, t, stream=stream.cuda_stream)
        sync_fn()
        if clocks and mode == 1:
            ck = clocks.stop()
        out.append(ctx.idp_dgsem_profile_read(reset=True))
    ctx.idp_dgsem_profile(0)
    (_, _, step_ms, nst), (el_ms, el_n, _, _) = out
    assert nst == steps
    return step_ms * 1e-3, el_ms, el_n, (ck if clocks else None)


def run_ours(args):
    import torch
    from paper_2607_06045_b300 import build, idp, roofline
    rank, local, world = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier_sync():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if dist is None:
            return x
        tt = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        return float(tt.item())

    probe = idp.idp_probe_pipes(stream.cuda_stream)
    fp64_tflops, fp32_tflops, w_div, w_sqrt, w_log = probe

    meshes, u0 = build_workload("dmr")
    nodes = u0.shape[1] * u0.shape[2] * u0.shape[3]
    results = {}
    for prec in (0, 1):
        ctx = idp.Context(meshes[0], 3, precision=prec, limiting=2, cfl=0.5)
        u_dev = torch.from_numpy(u0).cuda()
        clocks = Clocks(local) if prec == 0 else None
        barrier_sync()
        tot, el_ms, el_n, ck = time_steps(ctx, u_dev, args.steps, args.warmup, flush, stream, barrier_sync, clocks)
        tot = max_over_ranks(tot)
        rc, st = ctx.idp_dgsem_limiter_stats()
        results[prec] = dict(time=tot, el_ms=el_ms, el_n=el_n, clocks=ck, stats=st, ctx=ctx,
                             launches=ctx.launches_per_step() * args.steps, epb=None)
        if prec == 0:
            # end to end through the host-buffer entry point (pinned host state)
            uh = torch.from_numpy(u0.copy()).pin_memory()
            th = np.zeros(1)
            for _ in range(2):
                ctx.idp_dgsem_step_host(uh, 1, th, stream=stream.cuda_stream)
            barrier_sync()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                ctx.idp_dgsem_step_host(uh, 1, th, stream=stream.cuda_stream)
            e2e_t = max_over_ranks(time.perf_counter() - t0)
            results["e2e"] = e2e_t
        del u_dev
    # batched workload, FP32 form
    bm, ub = build_workload("batched")
    bnodes = ub.shape[1] * ub.shape[2] * ub.shape[3]
    bctx = idp.Context(bm, 3, precision=1, limiting=2, cfl=0.5)
    ubd = torch.from_numpy(ub).cuda()
    del ub
    bsteps = max(3, args.steps // 2)
    barrier_sync()
    btot, bel_ms, bel_n, _ = time_steps(bctx, ubd, bsteps, max(3, args.warmup // 2), flush, stream, barrier_sync)
    btot = max_over_ranks(btot)
    brc, bst = bctx.idp_dgsem_limiter_stats()

    if rank != 0:
        if dist is not None:
            dist.barrier()
        return
    r64, r32 = results[0], results[1]
    value = world * nodes * 3 * args.steps / r64["time"]
    w = (w_div, w_sqrt, w_log)
    f64 = roofline.element_flops(3, 0, *w)
    el_avg = r64["el_ms"] * 1e-3 / max(r64["el_n"], 1)
    achieved = f64 * nodes / el_avg * 1e-12
    f32 = roofline.element_flops(3, 1, *w)
    el32 = r32["el_ms"] * 1e-3 / max(r32["el_n"], 1)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r64["time"] / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "double Mach reflection, [0,4]x[0,1], 256x64 base + 3 levels along the shock",
                   "elements": int(u0.shape[1]), "N": 3, "dofs": int(nodes), "limiting": "local + positivity",
                   "cfl": 0.5, "precision": "fp64", "step": "one SSP-RK3 step (3 stages + dt)",
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": "k_element (element pass)",
                     "achieved": achieved, "peak": fp64_tflops, "unit": "TFLOP/s",
                     "frac": achieved / fp64_tflops,
                     "peak_source": "FP64 DFMA rate measured in this run (idp_probe_pipes)",
                     "flops_per_node_stage": f64, "weights_dfma_eq": {"div": w_div, "sqrt": w_sqrt, "log": w_log},
                     "launch_ms": el_avg * 1e3, "traffic": None},
        "e2e": {"value": world * nodes * 3 * args.steps / results["e2e"], "unit": UNIT,
                "h2d_bytes_per_step": int(u0.nbytes), "d2h_bytes_per_step": int(u0.nbytes)},
        "gpu_launches": int(r64["launches"]),
        "clocks": r64["clocks"],
        "stats": {k: r64["stats"][k] for k in ("alpha_volume_mean", "alpha_mortar_mean", "n_viol_density",
                                               "n_viol_pressure", "n_nonpositive")},
        "forms": {
            "fp32_form": {"value": world * nodes * 3 * args.steps / r32["time"], "unit": UNIT,
                          "ms_per_step": r32["time"] / args.steps * 1e3,
                          "speedup_vs_fp64": r64["time"] / r32["time"],
                          "roofline": {"bound": "alu", "achieved": f32 * nodes / el32 * 1e-12, "peak": fp64_tflops,
                                       "frac": f32 * nodes / el32 * 1e-12 / fp64_tflops, "unit": "TFLOP/s",
                                       "launch_ms": el32 * 1e3},
                          "gpu_launches": int(r32["launches"])},
            "batched_fp32": {"value": world * bnodes * 3 * bsteps / btot, "unit": UNIT,
                             "workload": "256 simulations, 8..128 base, 0-2 levels on seeded patches, N=3, "
                                         "four-quadrant Riemann data, FP32 form",
                             "elements": int(bctx.K), "dofs": int(bnodes), "steps": bsteps,
                             "speedup_vs_fp64": (bnodes * 3 * bsteps / btot) / (nodes * 3 * args.steps / r64["time"]),
                             "gpu_launches": int(bctx.launches_per_step() * bsteps),
                             "n_nonpositive": bst["n_nonpositive"]},
        },
        "probe": {"fp64_tflops": fp64_tflops, "fp32_tflops": fp32_tflops},
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_full()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()


def cpu_baseline_full():
    """The oracle as it stands on the host (one thread): two SSP-RK3 steps of
    the full DMR workload."""
    import oracle
    from paper_2607_06045_b300 import workloads as W
    m = W.cfg2_mesh()
    u = W.cfg2_state(m, 3)
    o = oracle.Oracle(m, 3)
    t0 = time.perf_counter()
    nsteps = 2
    o.step(u, nsteps, cfl=0.5, limiting=2)
    dt = time.perf_counter() - t0
    nodes = u.shape[1] * u.shape[2] * u.shape[3]
    return {"value": nodes * 3 * nsteps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{nsteps} SSP-RK3 steps of the full DMR workload ({nodes} DOFs), single-threaded C, {dt:.1f} s"}


def run_reference(args):
    rank, _, world = rank_env()
    if rank != 0:
        return
    import oracle
    from paper_2607_06045_b300 import workloads as W
    m = W.cfg2_sample_mesh()
    u = W.cfg2_state(m, 3)
    o = oracle.Oracle(m, 3)
    nodes = u.shape[1] * u.shape[2] * u.shape[3]
    t = 0.0
    for _ in range(args.warmup):
        u, t, _, _ = o.step(u, 1, t=t, cfl=0.5, limiting=2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, t, _, _ = o.step(u, 1, t=t, cfl=0.5, limiting=2)
    dt = time.perf_counter() - t0
    value = nodes * 3 * args.steps / dt
    sample = f"1/16-size DMR instance (64x16 base, {m.n_elems} elements, {nodes} DOFs), one SSP-RK3 step per bench step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "double Mach reflection (1/16-size instance of the 256x64 + 3 levels mesh)",
                       "N": 3, "limiting": "local + positivity", "cfl": 0.5},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
