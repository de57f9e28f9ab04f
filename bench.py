"""Benchmark: IDP-DGSEM DOF-updates/s per RK stage on B300.

One benchmark step is one SSP-RK3 step of the whole hot path (time step,
three limited stages, each with mortar fluxes, the element pass and mortar
limiting) over the workload's state, which is resident in HBM. The default
workload is the double-Mach-reflection mesh (256 x 64 base, up to three
extra levels along the shock, 60,139 elements, N = 3, FP64, local
limiting). The same JSON line also carries the FP32 form on that workload and
the batched workload (256 simulations, FP32 form).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the reference arm of this build) on a
1/16-size instance of the same DMR workload. Under torchrun every rank runs
its own replica of the workload (no data-path collective); the reported value
aggregates all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
# element-pass launch of the timed DMR contexts, per precision. A sweep of
# (elements per block, grid) pairs on a B300: the FP64 path is fastest with 4
# elements per block on a persistent grid of resident blocks (2.591 ms per
# step against 2.616 with 8 per block, one block per batch), the FP32 form
# with 8 per block, one block per batch (0.958 ms against 0.959 with 4 per
# block and 0.978 on the persistent grid). It is fixed rather than left to
# the autotuner so that a profiler run, whose serialised launches make the
# tuner's timings meaningless, launches the same grid as the timed run.
DMR_LAUNCH = {0: dict(elems_per_block=4, grid_mode=2), 1: dict(elems_per_block=8, grid_mode=1)}
# B300: 148 SMs, each retiring 2 FP64 fused multiply-adds per clock (the
# nominal 1.25 TFLOP/s FP64 rate at the maximum SM clock).
SMS, DFMA_PER_CLK_SM = 148, 2
# and 128 FP32 fused multiply-adds per clock
FFMA_PER_CLK_SM = 128
DMR_CONFIG = {"workload": "double Mach reflection, [0,4]x[0,1], 256x64 base + 3 levels along the shock",
              "elements": 60139, "N": 3, "dofs": 962224, "limiting": "local + positivity", "cfl": 0.5,
              "step": "one SSP-RK3 step (3 stages + dt)"}


def rank_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def dist_helpers(dist, device, sync=None):
    """Barrier (with device synchronisation on both sides) and max over ranks;
    plain local operations without a process group."""
    def barrier_sync():
        if sync:
            sync()
        if dist is not None:
            dist.barrier()
        if sync:
            sync()

    def max_over_ranks(x):
        if dist is None:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return barrier_sync, max_over_ranks


def shard_sims(n_sims, rank, world):
    """Simulations of the batched workload that rank `rank` of `world` runs:
    every world-th one, so that the ranks' loads stay alike (weak in ranks,
    the batch of independent simulations split with no communication)."""
    return list(range(rank, n_sims, world))


def sum_over_ranks(dist, device, x):
    """Sum of a number over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_rate(units_per_rank, world, max_time):
    """Whole-job throughput: units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / max_time


class Clocks:
    """nvidia-smi sampling (SM clock, limit and throttle reasons) around the
    timed region; start() returns once the first sample has arrived."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

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
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    @classmethod
    def parse(cls, lines):
        sm, mx, reasons = [], [], set()
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(cls.NAMES):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as fh:
            out = self.parse(fh.readlines())
        os.unlink(self.path)
        return out


def build_workload(name, subset=None):
    from paper_2607_06045_b300 import workloads as W
    if name == "dmr":
        m = W.dmr_mesh()
        return [m], W.dmr_state(m, 3)
    if name == "batched":
        ms = W.batch_meshes(256, seed=0)
        rng = np.random.default_rng(1)
        us = [W.riemann4_state(m, 3, rng) for m in ms]
        keep = range(len(ms)) if subset is None else subset
        return [ms[i] for i in keep], W.concat_states([us[i] for i in keep])
    if name == "vacuum":
        m, c = W.blast_mesh()
        return [m], W.blast_state(m, 5, c)
    raise ValueError(name)


def recorded_traffic():
    """DRAM bytes per element-pass launch from the committed ncu record, if the
    element-pass sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic_k_element_dmr.json")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None
        return rec["dram_bytes_read"] + rec["dram_bytes_write"]
    except (OSError, KeyError, ValueError):
        return None


def node_masses(mesh, N):
    """m_i = (dx dy / 4) w_i w_j per node, [K][N+1][N+1] (LGL weights)."""
    from numpy.polynomial import legendre as Lg
    x = np.sort(np.concatenate(([-1.0, 1.0], np.real(Lg.legroots(Lg.legder([0] * N + [1]))))))
    w = 2.0 / (N * (N + 1) * Lg.legval(x, [0] * N + [1]) ** 2)
    x0, y0, x1, y1 = mesh.box
    dx = (x1 - x0) / mesh.nx0 / 2.0 ** mesh.level
    dy = (y1 - y0) / mesh.ny0 / 2.0 ** mesh.level
    return (dx * dy / 4.0)[:, None, None] * w[None, :, None] * w[None, None, :]


def l1_per_field(u, ref, m):
    """Mass-weighted L1 difference per conserved field: sum m |u - ref| over
    sum m |ref| for rho and E, over sum m (|ref| + sqrt(rho E)) for the
    momenta (the state's momentum scale; a fluid at rest has none of its
    own)."""
    ps = np.sqrt(np.abs(ref[0] * ref[3]))
    out = {}
    for v, f in enumerate(("rho", "rho_v1", "rho_v2", "E")):
        den = (m * np.abs(ref[v])).sum() + ((m * ps).sum() if v in (1, 2) else 0.0)
        out[f] = float((m * np.abs(u[v] - ref[v])).sum() / max(den, 1e-300))
    return out


def parity_samples():
    """The parity-sized samples on which each FP32-form result states its L1
    error against the FP64 oracle: the 1/16 DMR instance (N = 3), the three
    smallest simulations of the batch (N = 3, as one batched context) and the
    near-vacuum blast on a 16 x 16 base (N = 5); five SSP-RK3 steps each."""
    from paper_2607_06045_b300 import workloads as W
    out = {}
    m = W.dmr_sample_mesh()
    out["fp32_form"] = dict(meshes=[m], N=3, u=[W.dmr_state(m, 3)], gamma=1.4,
                            sample="1/16 DMR instance (64x16 base + 3 levels), N=3, 5 steps")
    ms = W.batch_meshes(256, seed=0)
    rng = np.random.default_rng(1)
    us = [W.riemann4_state(mm, 3, rng) for mm in ms]
    small = np.argsort([mm.n_elems for mm in ms])[:3].tolist()
    out["batched_fp32"] = dict(meshes=[ms[k] for k in small], N=3, u=[us[k] for k in small], gamma=1.4,
                               sample=f"simulations {small} of the 256 (the three smallest), one batched context, "
                                      f"N=3, 5 steps")
    mv, cv = W.blast_mesh(n0=16)
    out["near_vacuum_fp32"] = dict(meshes=[mv], N=5, u=[W.blast_state(mv, 5, cv)], gamma=1.4,
                                   sample="near-vacuum blast on a 16x16 base + 2 levels, N=5, 5 steps")
    return out


PARITY_STEPS = 5


def cpu_baseline_parity_refs(samples):
    """CPU-baseline leg: the oracle (all host threads) on each parity sample."""
    import oracle
    refs = {}
    with oracle.using(oracle.build_omp()) as L:
        L.orc_set_threads(os.cpu_count() or 1)
        for name, smp in samples.items():
            refs[name] = []
            for m, u in zip(smp["meshes"], smp["u"]):
                o = oracle.Oracle(m, smp["N"], gamma=smp["gamma"])
                uo, _, _, _ = o.step(u, PARITY_STEPS, cfl=0.5, limiting=2)
                refs[name].append(uo)
    return refs


def l1_vs_oracle(samples, refs):
    """The FP32 form on each parity sample on the GPU against the oracle's
    states: per-field L1 (l1_per_field), the worst over a sample's
    simulations."""
    import torch
    from paper_2607_06045_b300 import idp
    from paper_2607_06045_b300 import workloads as W
    out = {}
    for name, smp in samples.items():
        ms, N = smp["meshes"], smp["N"]
        ctx = idp.Context(ms if len(ms) > 1 else ms[0], N, precision=1, limiting=2, cfl=0.5)
        ud = torch.from_numpy(W.concat_states(smp["u"])).cuda()
        t = np.zeros(len(ms))
        ctx.idp_dgsem_step(ud, PARITY_STEPS, t)
        ug = ud.cpu().numpy()
        off = ctx.sim_offsets
        worst = {}
        for k, (m, uo) in enumerate(zip(ms, refs[name])):
            e = l1_per_field(ug[:, off[k]:off[k + 1]], uo, node_masses(m, N))
            worst = {f: max(worst.get(f, 0.0), v) for f, v in e.items()}
        ctx.close()
        out[name] = dict(worst, steps=PARITY_STEPS, sample=smp["sample"], reference="FP64 oracle")
    return out


def method_work(roofline, N, precision, K, M, n_mnodes, w):
    """Per kernel and launch: (FP64 flops, FP32 flops, HBM bytes), the flops
    from the method's work table (the oracle's counting build), the bytes
    from the kernels' algorithmic traffic."""
    fl = roofline.method_kernel_work(N, precision, K, M=M)
    by = {name: b for name, (_, b) in roofline.kernel_work(N, precision, K, M, n_mnodes, *w).items()}
    # one kernel limits the mortars and applies their corrections
    by["mortar_limit"] += by.pop("mortar_apply")
    return {name: fl.get(name, (0.0, 0.0)) + (b,) for name, b in by.items()}


def kernel_rooflines(work, kern, steps, step_time, peak_tflops, hbm_gbs, peak32_tflops=None):
    """Per kernel: measured ms per launch, share of the kernel time, roofline
    time max(FP64 flops / FP64 peak + FP32 flops / FP32 peak, bytes / HBM) and
    its fraction of the measured time; and the step's roofline fraction (sum
    of the kernels' roofline times over the measured step time)."""
    out, tot, roof_step = {}, sum(ms for ms, n in kern.values()), 0.0
    for name, (ms, n) in kern.items():
        if n == 0:
            continue
        t = ms * 1e-3 / n
        d = {"ms_per_launch": t * 1e3, "launches_per_step": n / steps, "share": ms / tot}
        if name in work:
            if len(work[name]) == 3:
                f64, f32, by = work[name]
            else:
                (f64, by), f32 = work[name], 0.0
            ta = f64 / (peak_tflops * 1e12) + (f32 / (peak32_tflops * 1e12) if f32 else 0.0)
            tb = by / (hbm_gbs * 1e9)
            d.update({"bound": "alu" if ta >= tb else "hbm", "roofline_ms": max(ta, tb) * 1e3,
                      "frac": max(ta, tb) / t})
            roof_step += max(ta, tb) * n / steps
        out[name] = d
    return out, {"roofline_ms": roof_step * 1e3, "measured_ms": step_time * 1e3, "frac": roof_step / step_time}


def form_roofline(roofline, N, precision, nodes, el_s, peak, peak32, w):
    """Element-pass roofline of one form: the method's flops per node and
    stage (the oracle's counting build), FP64 rows over the FP64 peak and, in
    the FP32 form, the flux rows over the FP32 peak; beside it the issued
    FP64 efficiency of the kernels' own FP64 instruction count."""
    f64, f32 = roofline.method_flops(N, roofline.ELEMENT_ROWS, precision)
    t_roof = nodes * (f64 / (peak * 1e12) + f32 / (peak32 * 1e12))
    ach = (f64 + f32) * nodes / el_s * 1e-12
    issued = roofline.element_flops(N, precision, *w)
    ach_i = issued * nodes / el_s * 1e-12
    return {"bound": "alu", "achieved": ach, "peak": (f64 + f32) * nodes / t_roof * 1e-12, "unit": "TFLOP/s",
            "frac": t_roof / el_s, "flops_per_node_stage": f64 + f32, "fp64_flops_per_node_stage": f64,
            "fp32_flops_per_node_stage": f32, "flops_source": "oracle op-counting build (method_work.json), "
                                                             "one flop per operation",
            "peak_fp64": peak, "peak_fp32": peak32, "launch_ms": el_s * 1e3,
            "issued_fp64": {"flops_per_node_stage": issued, "achieved": ach_i, "peak": peak, "frac": ach_i / peak,
                            "weights_dfma_eq": {"div": w[0], "sqrt": w[1], "log": w[2]}}}


def vacuum_entry(vac, vnodes, world, roofline, w, peak, hbm, unit, peak32):
    """JSON entry of the near-vacuum blast (FP32 form, N = 5): rate, element-pass
    roofline, per-kernel rooflines, invariants."""
    steps = vac["steps"]
    el = vac["el_ms"] * 1e-3 / max(vac["el_n"], 1)
    kr, st = kernel_rooflines(method_work(roofline, 5, 1, vac["K"], vac["M"], 18 * vac["M"], w), vac["kern"],
                              steps, vac["time"] / steps, peak, hbm, peak32)
    return {"value": aggregate_rate(vnodes * 3 * steps, world, vac["time"]), "unit": unit,
            "workload": "near-vacuum blast: 512x512 base + 2 levels within r < 0.1, N=5, rho 1e-6 / p 1e-9 "
                        "background, disc rho 1 / p 1e3, outflow, FP32 form",
            "elements": int(vac["K"]), "dofs": int(vnodes), "steps": steps,
            "ms_per_step": vac["time"] / steps * 1e3, "ms_per_step_median": vac["median_ms"],
            "roofline": form_roofline(roofline, 5, 1, vnodes, el, peak, peak32, w),
            "kernels": kr, "step_roofline": st, "gpu_launches": int(vac["launches"]),
            "stats": {k: vac["stats"][k] for k in ("alpha_volume_mean", "alpha_mortar_mean", "n_viol_density",
                                                    "n_viol_pressure", "n_nonpositive")}}


def time_steps(ctx, u_dev, steps, warmup, flush, stream, sync_fn):
    """Per-step CUDA-event timing on the launching stream, L2 flushed between
    steps. Pass 1 (the headline): CUDA-graph steps bracketed by events. Pass 2:
    the same number of steps launched kernel by kernel with events around each
    element pass (the roofline's kernel duration)."""
    import torch
    t = np.zeros(ctx.n_sims)
    for _ in range(warmup):
        ctx.idp_dgsem_step(u_dev, 1, t, stream=stream.cuda_stream)
    out, per_step = [], []
    for mode in (1, 2):
        ctx.idp_dgsem_profile(mode)
        ctx.idp_dgsem_profile_read(reset=True)
        sync_fn()
        acc = [0.0, 0.0, 0.0, 0]
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()          # L2 flush, outside the timed span
            ctx.idp_dgsem_step(u_dev, 1, t, stream=stream.cuda_stream)
            if mode == 1:
                # each step's own event span (the step synchronises in profiling modes)
                _, _, ms, n = ctx.idp_dgsem_profile_read(reset=True)
                per_step.append(ms)
                acc[2] += ms
                acc[3] += n
        sync_fn()
        kern = ctx.idp_dgsem_profile_kernels(reset=False)
        if mode == 1:
            out.append(tuple(acc))
        else:
            out.append(ctx.idp_dgsem_profile_read(reset=True) + (kern,))
    ctx.idp_dgsem_profile(0)
    (_, _, step_ms, nst), (el_ms, el_n, _, _, kern) = out
    assert nst == steps
    time_steps.median_ms = float(np.median(per_step))
    return step_ms * 1e-3, el_ms, el_n, kern


def bench_3d(idp, flush, stream, args, n=40, N=3, octree=False, precision=0):
    """The 3D blast on an n^3 grid, or (octree) on an n^3 base grid with the
    leaves in [1/4, 3/4]^3 refined once: 2:1 mortars around the block;
    precision 1: the FP32 form."""
    import torch
    from paper_2607_06045_b300 import workloads as W
    if octree:
        g = W.box_refined_mesh3(n, n, n, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), (0.25, 0.25, 0.25, 0.75, 0.75, 0.75),
                                bc=(3,) * 6)
    else:
        g = W.Grid3(n, n, n, bc=(3,) * 6)
    u = W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0)
    ctx = idp.Context3D(g, N, limiting=2, cfl=0.5, precision=precision)
    ud = torch.from_numpy(u).cuda()
    del u
    t = np.zeros(1)
    steps = max(5, args.steps // 2)
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            ctx.idp3d_step(ud, 1, t, stream=stream.cuda_stream)
        times = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.idp3d_step(ud, 1, t, stream=stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    rc, st = ctx.idp3d_limiter_stats()
    dofs = g.n_elems * (N + 1) ** 3
    ms = float(np.mean(times))
    mesh_text = (f"{n}^3 base hexahedra with [1/4, 3/4]^3 refined once ({g.n_elems} leaves, {ctx.n_mortars} "
                 f"mortars)" if octree else f"{n}^3 hexahedra")
    # per step: the time step (FP64 path: a reset and its FP32 and FP64 passes), three element
    # launches, the advance; on octrees mortar flux, factor and apply per stage
    launches = (5 if precision else 7) + (9 if octree else 0)
    out = dict(value=dofs * 3 / (ms * 1e-3), unit=UNIT, ms_per_step=ms, ms_per_step_median=float(np.median(times)),
               steps=steps, elements=g.n_elems, dofs=dofs, gpu_launches=launches * steps,
               workload=f"3D blast: [0,1]^3, {mesh_text}, N={N}, sphere r < 0.15 at p = 10 in a gas at "
                        "rho = 1, p = 0.1, outflow, local limiting (d = 3, Gamma = 6), "
                        + ("FP32 form" if precision else "FP64"),
               stats={k: st[k] for k in ("alpha_mean", "n_viol_density", "n_viol_pressure", "n_nonpositive",
                                         "alpha_mortar", "n_mortar_active", "n_mortar_fallback")})
    if octree:
        out["mortars"] = ctx.n_mortars
        out["mortar_nodes"] = ctx.n_mortar_nodes
    ctx.close()
    return out


def run_ours(args):
    import torch
    from paper_2607_06045_b300 import build, idp, roofline
    rank, local, world = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    barrier_sync, max_over_ranks = dist_helpers(dist, "cuda", torch.cuda.synchronize)

    probe = idp.idp_probe_pipes(stream.cuda_stream)
    fp64_probe, fp32_probe, w_div, w_sqrt, w_log = probe

    meshes, u0 = build_workload("dmr")
    nodes = u0.shape[1] * u0.shape[2] * u0.shape[3]
    results = {}
    clocks = Clocks(local)
    for prec in (0, 1):
        ctx = idp.Context(meshes[0], 3, precision=prec, limiting=2, cfl=0.5, **DMR_LAUNCH[prec])
        u_dev = torch.from_numpy(u0).cuda()
        barrier_sync()
        if prec == 0:
            clocks.start()
        tot, el_ms, el_n, kern = time_steps(ctx, u_dev, args.steps, args.warmup, flush, stream, barrier_sync)
        if prec == 0:
            ck = clocks.stop()
        tot = max_over_ranks(tot)
        rc, st = ctx.idp_dgsem_limiter_stats()
        results[prec] = dict(time=tot, el_ms=el_ms, el_n=el_n, stats=st, ctx=ctx, kern=kern,
                             launches=ctx.launches_per_step() * args.steps, u_end=u_dev.cpu().numpy(),
                             median_ms=time_steps.median_ms,
                             launch=dict(zip(("elems_per_block", "persistent", "grid"),
                                             ctx.idp_dgsem_launch_config())))
        if prec == 0:
            results["clocks"] = ck
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
    # limiter variants (FP64 path, same workload): combined positivity/local
    # limiting (Sec. 3.5), the entropy bound and the low-order-solution
    # bounds of local limiting (Sec. 2.3, Eqs. Bounds_Barstates,
    # Bounds_LowOrder), and the low-order CFL estimate against the IDP step
    variants = {}
    vsteps = max(3, args.steps // 4)
    for name, kw in (("combined", dict(limiting=3)), ("entropy_bound", dict(limiting=2, entropy_bound=1)),
                     ("low_order_bounds", dict(limiting=2, bounds=1)),
                     ("low_order_bounds_entropy", dict(limiting=2, bounds=1, entropy_bound=1)),
                     ("all_to_all_mortar", dict(limiting=2, mortar_low=1))):
        vctx = idp.Context(meshes[0], 3, precision=0, cfl=0.5, **kw)
        u_dev = torch.from_numpy(u0).cuda()
        barrier_sync()
        vt, _, _, vk = time_steps(vctx, u_dev, vsteps, args.warmup, flush, stream, barrier_sync)
        vt = max_over_ranks(vt)
        _, vst = vctx.idp_dgsem_limiter_stats()
        variants[name] = dict(value=aggregate_rate(nodes * 3 * vsteps, world, vt), unit=UNIT,
                              ms_per_step=vt / vsteps * 1e3, steps=vsteps, options=kw,
                              gpu_launches=int(vctx.launches_per_step() * vsteps),
                              kernels={k: {"ms_per_launch": ms / n, "launches_per_step": n / vsteps}
                                       for k, (ms, n) in vk.items() if n},
                              stats={k: vst[k] for k in ("alpha_volume_mean", "alpha_mortar_mean", "n_viol_density",
                                                         "n_viol_pressure", "n_viol_entropy", "n_nonpositive")})
        vctx.close()
        del u_dev
    from paper_2607_06045_b300 import workloads as W
    # the refined periodic square (16 x 16 base, central 4 x 4 refined, N = 3,
    # FP64): too small to fill the GPU, timed for its latency per step
    sq = W.square_mesh()
    usq = W.disc_wave_state(sq, 3)
    lctx = idp.Context(sq, 3, limiting=2, cfl=0.5)
    lud = torch.from_numpy(usq).cuda()
    barrier_sync()
    lt, _, _, _ = time_steps(lctx, lud, args.steps, args.warmup, flush, stream, barrier_sync)
    variants["square_latency"] = dict(
        ms_per_step=lt / args.steps * 1e3, ms_per_step_median=time_steps.median_ms, steps=args.steps,
        elements=int(lctx.K), dofs=int(usq[0].size), value=usq[0].size * 3 * args.steps / lt, unit=UNIT,
        workload="periodic unit square, 16x16 base with the central 4x4 refined once, N=3, disc on a smooth "
                 "wave, local + positivity limiting, FP64",
        gpu_launches=int(lctx.launches_per_step() * args.steps))
    lctx.close()
    del lud
    # the DMR mesh at N = 4 and N = 7, the FP64 path and the FP32 form
    for NN_ in (4, 7):
        uN = W.dmr_state(meshes[0], NN_)
        nN = uN[0].size
        ent = {}
        for prec in (0, 1):
            nctx = idp.Context(meshes[0], NN_, precision=prec, limiting=2, cfl=0.5)
            nud = torch.from_numpy(uN).cuda()
            barrier_sync()
            nt, nel_ms, nel_n, nk = time_steps(nctx, nud, vsteps, args.warmup, flush, stream, barrier_sync)
            nt = max_over_ranks(nt)
            _, nst_ = nctx.idp_dgsem_limiter_stats()
            ent["fp32" if prec else "fp64"] = dict(
                value=aggregate_rate(nN * 3 * vsteps, world, nt), unit=UNIT, ms_per_step=nt / vsteps * 1e3,
                steps=vsteps, _el_s=nel_ms * 1e-3 / max(nel_n, 1), gpu_launches=int(nctx.launches_per_step() * vsteps),
                launch=dict(zip(("elems_per_block", "persistent", "grid"), nctx.idp_dgsem_launch_config())),
                stats={k: nst_[k] for k in ("alpha_volume_mean", "alpha_mortar_mean", "n_viol_density",
                                            "n_viol_pressure", "n_nonpositive")})
            nctx.close()
            del nud
        ent["speedup_fp32_vs_fp64"] = ent["fp64"]["ms_per_step"] / ent["fp32"]["ms_per_step"]
        variants[f"dmr_N{NN_}"] = dict(ent, elements=int(meshes[0].n_elems), dofs=int(nN), N=NN_,
                                       workload=f"the DMR mesh and initial data at N={NN_}")
    # high-Mach jet (gamma = 5/3, Mach ~2000 inflow), Chandrashekar's volume
    # flux with combined limiting as in the paper's astrophysical jet, on a
    # static 53,632-element mesh, both precisions
    jm = W.jet_mesh()
    ju = W.jet_state(jm, 3, W.JET_GAMMA)
    jnodes = ju.shape[1] * ju.shape[2] * ju.shape[3]
    for prec in (0, 1):
        jctx = idp.Context(jm, 3, gamma=W.JET_GAMMA, precision=prec, limiting=3, volume_flux=1, cfl=0.5)
        jud = torch.from_numpy(ju).cuda()
        barrier_sync()
        jt, _, _, jk = time_steps(jctx, jud, vsteps, args.warmup, flush, stream, barrier_sync)
        jt = max_over_ranks(jt)
        _, jst = jctx.idp_dgsem_limiter_stats()
        variants[f"jet_chandrashekar_{'fp32' if prec else 'fp64'}"] = dict(
            value=aggregate_rate(jnodes * 3 * vsteps, world, jt), unit=UNIT, ms_per_step=jt / vsteps * 1e3,
            steps=vsteps, elements=int(jctx.K), dofs=int(jnodes),
            workload="jet: [-0.5,0.5]^2, 64x64 base + 3 levels in |y| < 0.1, N=3, gamma 5/3, rho 5 / v1 800 "
                     "inflow band, combined limiting, Chandrashekar volume flux",
            gpu_launches=int(jctx.launches_per_step() * vsteps),
            kernels={k: {"ms_per_launch": ms / n, "launches_per_step": n / vsteps} for k, (ms, n) in jk.items() if n},
            stats={k: jst[k] for k in ("alpha_volume_mean", "alpha_mortar_mean", "n_viol_density",
                                       "n_viol_pressure", "n_nonpositive")})
        jctx.close()
        del jud
    # adaptive DMR (Sec. 2.4): every 10 steps an AMR step, levels 0..4 over
    # the DMR base grid. Device path: one call re-meshes in the context
    # (indicator, plan, transfer, face / mortar / node / block tables); host
    # path: indicator on the device, plan on the host, transfer on the
    # device and a new context for the new mesh. Wall time of each phase.
    import dataclasses
    ap = idp.amr_params(indicator=2, refine_threshold=0.3, coarsen_threshold=0.01, min_level=0, max_level=4)
    acycles, asteps = 3, 10

    def adaptive(device):
        actx = idp.Context(meshes[0], 3, limiting=2, cfl=0.5)
        aud = torch.from_numpy(u0).cuda()
        at = np.zeros(1)
        actx.idp_dgsem_step(aud.clone(), 1, np.zeros(1))   # first tuning, outside the cycles
        phase = ({"adapt": 0.0, "steps": 0.0} if device else
                 {"indicator": 0.0, "plan": 0.0, "transfer": 0.0, "create": 0.0, "steps": 0.0})
        node_stages, sizes, scaled_total, first_step = 0, [], 0, []
        # the caller's two state buffers (ping-pong), each for four times the
        # elements of the mesh it adapts from
        bufs = [torch.empty(4 * 4 * actx.K * 16, dtype=torch.float64, device="cuda") for _ in range(2)]
        barrier_sync()
        for cyc in range(acycles):
            if device and bufs[cyc % 2].numel() < 4 * 4 * actx.K * 16:
                bufs[cyc % 2] = torch.empty(4 * 4 * actx.K * 16, dtype=torch.float64, device="cuda")
            t0 = time.perf_counter()
            if device:
                aud, sc = actx.idp_dgsem_adapt(aud, ap, out=bufs[cyc % 2])
                torch.cuda.synchronize()
                marks = [time.perf_counter()]
            else:
                ind = actx.idp_dgsem_amr_indicator(aud, ap)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                pl = idp.idp_amr_plan(actx.meshes[0], ind.cpu().numpy(), ap)
                t2 = time.perf_counter()
                aun, sc = idp.idp_amr_transfer(3, 1.4, aud, pl[3], pl[4], ap.zs_threshold)
                t3 = time.perf_counter()
                mesh2 = dataclasses.replace(actx.meshes[0], level=pl[0], ix=pl[1], iy=pl[2])
                actx2 = idp.Context(mesh2, 3, opts=actx.opts)
                torch.cuda.synchronize()
                marks = [t1, t2, t3, time.perf_counter()]
                actx.close()
                actx, aud = actx2, aun
            ts = time.perf_counter()
            actx.idp_dgsem_step(aud, 1, at)
            torch.cuda.synchronize()
            first_step.append(time.perf_counter() - ts)
            actx.idp_dgsem_step(aud, asteps - 1, at)
            torch.cuda.synchronize()
            marks.append(time.perf_counter())
            prev = t0
            for k, tm in zip(phase, marks):
                phase[k] += tm - prev
                prev = tm
            node_stages += actx.K * 16 * 3 * asteps
            sizes.append(int(actx.K))
            scaled_total += sc
        _, ast = actx.idp_dgsem_limiter_stats()
        tot_wall = max_over_ranks(sum(phase.values()))
        amr_s = sum(v for k, v in phase.items() if k != "steps")
        res = dict(
            value=aggregate_rate(node_stages, world, tot_wall), unit=UNIT,
            elements_per_cycle=sizes, scaled_families=int(scaled_total),
            ms_per_cycle={k: v / acycles * 1e3 for k, v in phase.items()},
            amr_over_steps=amr_s / phase["steps"],
            first_step_ms=[v * 1e3 for v in first_step],
            stats={k: ast[k] for k in ("n_viol_density", "n_viol_pressure", "n_nonpositive")})
        actx.close()
        return res

    variants["adaptive_dmr"] = adaptive(True)
    variants["adaptive_dmr"]["note"] = (
        "wall clock over 3 cycles of (AMR step, 10 SSP-RK3 steps), the AMR step one idp_dgsem_adapt call that "
        "re-meshes on the device in the context, into the caller's preallocated state buffers (two, used in "
        "turn); the steps include the graph capture of each new mesh; "
        "amr_over_steps = AMR time / time of the 10 steps that follow")
    variants["adaptive_dmr_host_plan"] = adaptive(False)
    variants["adaptive_dmr_host_plan"]["note"] = (
        "the same cycles with the plan on the host and a new context per mesh (its first step tunes the launch)")
    dts = []
    for rule in (0, 1):
        dctx = idp.Context(meshes[0], 3, cfl=1.0, dt_rule=rule)
        dts.append(float(dctx.idp_dgsem_dt(torch.from_numpy(u0).cuda())[0]))
        dctx.close()
    # 3D (d = 3, Gamma = 6): a blast in a 40^3 grid of hexahedra, N = 3
    # (4.1M DOFs), local limiting, FP64; per-step CUDA events on the
    # launching stream, L2 flushed between steps
    variants["blast3d"] = bench_3d(idp, flush, stream, args)
    # the same blast on a 2:1 octree: 32^3 base, [1/4, 3/4]^3 refined once
    # (61,440 leaves, 1,536 mortars, 3.9M DOFs)
    variants["blast3d_octree"] = bench_3d(idp, flush, stream, args, n=32, octree=True)
    # the FP32 form of the 3D path on both meshes
    variants["blast3d_fp32"] = bench_3d(idp, flush, stream, args, precision=1)
    variants["blast3d_octree_fp32"] = bench_3d(idp, flush, stream, args, n=32, octree=True, precision=1)
    variants["dt_rules"] = {"idp": dts[0], "low_order_cfl": dts[1], "ratio": dts[1] / dts[0],
                            "note": "cfl = 1 on the initial state; steps to a fixed time scale with 1 / dt"}
    # near-vacuum blast (512 x 512 base + 2 levels, N = 5), FP32 form
    vm, vu = build_workload("vacuum")
    vnodes = vu.shape[1] * vu.shape[2] * vu.shape[3]
    vctx = idp.Context(vm[0], 5, precision=1, limiting=2, cfl=0.5)
    vud = torch.from_numpy(vu).cuda()
    del vu
    vsteps_v = max(3, args.steps // 10)
    barrier_sync()
    vtot, vel_ms, vel_n, vkern = time_steps(vctx, vud, vsteps_v, args.warmup, flush, stream, barrier_sync)
    vtot = max_over_ranks(vtot)
    _, vst5 = vctx.idp_dgsem_limiter_stats()
    vac = dict(time=vtot, el_ms=vel_ms, el_n=vel_n, kern=vkern, stats=vst5, K=vctx.K, M=vctx.M,
               launches=vctx.launches_per_step() * vsteps_v, steps=vsteps_v, median_ms=time_steps.median_ms)
    vctx.close()
    del vud
    # batched workload, FP32 form
    # the batch's independent simulations are split across the ranks
    bm, ub = build_workload("batched", shard_sims(256, rank, world) if world > 1 else None)
    bnodes = ub.shape[1] * ub.shape[2] * ub.shape[3]
    bnodes_all = sum_over_ranks(dist, "cuda", bnodes)
    bctx = idp.Context(bm, 3, precision=1, limiting=2, cfl=0.5)
    ubd = torch.from_numpy(ub).cuda()
    del ub
    bsteps = max(3, args.steps // 4)
    barrier_sync()
    btot, _, _, _ = time_steps(bctx, ubd, bsteps, max(3, args.warmup // 2), flush, stream, barrier_sync)
    btot = max_over_ranks(btot)
    brc, bst = bctx.idp_dgsem_limiter_stats()

    if rank != 0:
        barrier_sync()
        return
    r64, r32 = results[0], results[1]
    ck = results["clocks"]
    value = aggregate_rate(nodes * 3 * args.steps, world, r64["time"])
    sm_mhz = ck["sm_max_mhz"] or 2032.0
    peak = SMS * DFMA_PER_CLK_SM * 2 * sm_mhz * 1e6 * 1e-12
    peak32 = SMS * FFMA_PER_CLK_SM * 2 * sm_mhz * 1e6 * 1e-12
    w = (w_div, w_sqrt, w_log)
    el_avg = r64["el_ms"] * 1e-3 / max(r64["el_n"], 1)
    el32 = r32["el_ms"] * 1e-3 / max(r32["el_n"], 1)
    roof64 = form_roofline(roofline, 3, 0, nodes, el_avg, peak, peak32, w)
    roof32 = form_roofline(roofline, 3, 1, nodes, el32, peak, peak32, w)
    for NN_ in (4, 7):
        ent = variants[f"dmr_N{NN_}"]
        for key, prec in (("fp64", 0), ("fp32", 1)):
            e = ent[key]
            e["roofline"] = form_roofline(roofline, NN_, prec, ent["dofs"], e.pop("_el_s"), peak, peak32, w)
    # 3D: the whole step against the method's work of the 3D counting build
    b3 = variants["blast3d"]
    t3 = json.load(open(os.path.join(ROOT, "paper_2607_06045_b300", "method_work.json")))["3d"]["degrees"]["3"]
    f3 = t3["method_flops_per_node_stage"]
    ach3 = f3 * b3["dofs"] * 3 / (b3["ms_per_step"] * 1e-3) * 1e-12
    b3["step_roofline"] = dict(bound="alu", achieved=ach3, peak=peak, unit="TFLOP/s", frac=ach3 / peak,
                               flops_per_node_stage=f3,
                               flops_source="oracle op-counting build, 3D (method_work.json: 3d), one flop per "
                                            "operation; the whole step (time step, three stages, advance)")
    # 3D octree: the method's work per node (all rows but the mortars') and
    # per mortar, from the counting build on the same mesh at 1/64 size
    bo = variants["blast3d_octree"]
    to = json.load(open(os.path.join(ROOT, "paper_2607_06045_b300", "method_work.json")))["3d_octree"]["degrees"]["3"]
    fo = to["node_flops_per_node_stage"] * bo["dofs"] + to["mortar_flops_per_mortar_stage"] * bo["mortars"]
    acho = fo * 3 / (bo["ms_per_step"] * 1e-3) * 1e-12
    bo["step_roofline"] = dict(bound="alu", achieved=acho, peak=peak, unit="TFLOP/s", frac=acho / peak,
                               flops_per_stage=fo,
                               flops_source="oracle op-counting build, 3D octree (method_work.json: 3d_octree): "
                                            "per node and per mortar; the whole step")
    # 3D FP32 form: its FP32 rows over the FP32 peak plus the rest over the
    # FP64 peak give the roofline time of a step
    f32rows = ("node_prep", "volume_flux", "subcell_fv", "face_flux")
    for key, base in (("blast3d_fp32", t3), ("blast3d_octree_fp32", None)):
        bf = variants[key]
        rows3 = t3["rows"]
        f32 = sum(rows3[r]["flops"] for r in f32rows)
        if base is None:
            f64 = (to["node_flops_per_node_stage"] - f32) * bf["dofs"] + to["mortar_flops_per_mortar_stage"] * bf["mortars"]
        else:
            f64 = (f3 - f32) * bf["dofs"]
        t_roof = 3 * (f64 / (peak * 1e12) + f32 * bf["dofs"] / (peak32 * 1e12))
        bf["step_roofline"] = dict(bound="alu", roofline_ms=t_roof * 1e3, frac=t_roof / (bf["ms_per_step"] * 1e-3),
                                   flops_fp64_per_stage=f64, flops_fp32_per_stage=f32 * bf["dofs"],
                                   peak_fp64=peak, peak_fp32=peak32, unit="TFLOP/s",
                                   flops_source="3D counting build; rows node_prep, volume_flux, subcell_fv and "
                                                "face_flux in FP32, the rest in FP64")
        bf["speedup_vs_fp64"] = variants[key.replace("_fp32", "")]["ms_per_step"] / bf["ms_per_step"]
    bval = bnodes_all * 3 * bsteps / btot   # the whole batch over the slowest rank
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6400.0
    K, M = r64["ctx"].K, r64["ctx"].M
    kr64, st64 = kernel_rooflines(method_work(roofline, 3, 0, K, M, 12 * M, w), r64["kern"], args.steps,
                                  r64["time"] / args.steps, peak, hbm, peak32)
    kr32, st32 = kernel_rooflines(method_work(roofline, 3, 1, K, M, 12 * M, w), r32["kern"], args.steps,
                                  r32["time"] / args.steps, peak, hbm, peak32)
    # FP32 form against the FP64 path after the same number of steps from the
    # same state (the FP64 path matches the FP64 oracle to 1e-10 over 100 steps)
    l1 = l1_per_field(r32["u_end"], r64["u_end"], node_masses(meshes[0], 3))
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r64["time"] / args.steps * 1e3,
        "ms_per_step_median": r64["median_ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": dict(DMR_CONFIG, precision="fp64", l2="flushed between steps (256 MiB write)",
                       parallelism=f"replicas x{world}", element_launch=r64["launch"]),
        "roofline": dict(roof64, kernel="k_face + k_element (element pass, FP64 path)",
                         peak_source=f"derived: {SMS} SMs x {DFMA_PER_CLK_SM} FP64 FMA/clk x 2 flop x "
                                     f"{sm_mhz:.0f} MHz", peak_probe=fp64_probe, traffic=recorded_traffic()),
        "e2e": {"value": aggregate_rate(nodes * 3 * args.steps, world, results["e2e"]), "unit": UNIT,
                "h2d_bytes_per_step": int(u0.nbytes), "d2h_bytes_per_step": int(u0.nbytes)},
        "gpu_launches": int(r64["launches"]),
        "kernels": kr64,
        "step_roofline": dict(st64, peaks={"fp64_tflops": peak, "hbm_gbs": hbm}),
        "clocks": ck,
        "stats": {k: r64["stats"][k] for k in ("alpha_volume_mean", "alpha_mortar_mean", "n_viol_density",
                                               "n_viol_pressure", "n_nonpositive")},
        "forms": {
            "fp32_form": {"value": aggregate_rate(nodes * 3 * args.steps, world, r32["time"]), "unit": UNIT,
                          "ms_per_step": r32["time"] / args.steps * 1e3,
                          "speedup_vs_fp64": r64["time"] / r32["time"],
                          "element_launch": r32["launch"],
                          "roofline": roof32,
                          "gpu_launches": int(r32["launches"]),
                          "kernels": kr32,
                          "step_roofline": st32,
                          "l1_vs_fp64": dict(l1, steps=args.warmup + 2 * args.steps),
                          "stats": {k: r32["stats"][k] for k in ("alpha_volume_mean", "n_viol_density",
                                                                 "n_viol_pressure", "n_nonpositive")}},
            "near_vacuum_fp32": vacuum_entry(vac, vnodes, world, roofline, w, peak, hbm, UNIT, peak32),
            "batched_fp32": {"value": bval, "unit": UNIT,
                             "workload": "256 simulations, 8..128 base, 0-2 levels on seeded patches, N=3, "
                                         "four-quadrant Riemann data, FP32 form",
                             "elements_rank0": int(bctx.K), "dofs": int(bnodes_all), "steps": bsteps,
                             "scaling": "strong: the 256 simulations split across the ranks, no communication",
                             "speedup_vs_fp64": bval / value,
                             "gpu_launches": int(bctx.launches_per_step() * bsteps),
                             "stats": {k: bst[k] for k in ("alpha_volume_mean", "n_viol_density",
                                                           "n_viol_pressure", "n_nonpositive")}},
        },
        "probe": {"fp64_tflops": fp64_probe, "fp32_tflops": fp32_probe},
        "variants": dict(variants, ms_per_step_local=r64["time"] / args.steps * 1e3),
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_full()
        samples = parity_samples()
        l1o = l1_vs_oracle(samples, cpu_baseline_parity_refs(samples))
        for name, e in l1o.items():
            line["forms"][name]["l1_vs_oracle"] = e
    print(json.dumps(line), flush=True)
    barrier_sync()


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def time_oracle(m, u, nsteps, threads, warmup=0):
    """Seconds for nsteps SSP-RK3 steps of the oracle as it stands: the serial
    build (threads = 1) or its OpenMP build on `threads` host threads (the
    same bits); returns (seconds, threads used)."""
    import oracle
    path = oracle.build() if threads == 1 else oracle.build_omp()
    with oracle.using(path) as L:
        used = L.orc_set_threads(threads)
        o = oracle.Oracle(m, 3)
        t = 0.0
        for _ in range(warmup):
            u, t, _, _ = o.step(u, 1, t=t, cfl=0.5, limiting=2)
        t0 = time.perf_counter()
        for _ in range(nsteps):
            u, t, _, _ = o.step(u, 1, t=t, cfl=0.5, limiting=2)
        return time.perf_counter() - t0, used


def cpu_baseline_full():
    """The oracle as it stands on the host: two SSP-RK3 steps of the full DMR
    workload on all host threads (its OpenMP build), and the same on one
    thread."""
    from paper_2607_06045_b300 import workloads as W
    m = W.dmr_mesh()
    u = W.dmr_state(m, 3)
    nodes = u.shape[1] * u.shape[2] * u.shape[3]
    nsteps = 2
    dt_all, used = time_oracle(m, u, nsteps, os.cpu_count() or 1)
    dt_one, _ = time_oracle(m, u, nsteps, 1)
    return {"value": nodes * 3 * nsteps / dt_all, "unit": UNIT, "cores": used, "kind": "oracle", "cpu": cpu_model(),
            "host_threads": os.cpu_count(),
            "sample": f"{nsteps} SSP-RK3 steps of the full DMR workload ({nodes} DOFs), C oracle with OpenMP "
                      f"on {used} threads, {dt_all:.1f} s",
            "single_thread": {"value": nodes * 3 * nsteps / dt_one, "unit": UNIT, "cores": 1,
                              "sample": f"the same steps on one thread, {dt_one:.1f} s"}}


def run_reference(args):
    rank, _, world = rank_env()
    if rank != 0:
        return
    from paper_2607_06045_b300 import workloads as W
    m = W.dmr_sample_mesh()
    u = W.dmr_state(m, 3)
    nodes = u.shape[1] * u.shape[2] * u.shape[3]
    dt, used = time_oracle(m, u, args.steps, os.cpu_count() or 1, warmup=args.warmup)
    value = nodes * 3 * args.steps / dt
    sample = (f"1/16-size instance of the DMR workload (64x16 base, {m.n_elems} elements, {nodes} DOFs), "
              f"one SSP-RK3 step per bench step, C oracle with OpenMP on {used} threads")
    config = dict(DMR_CONFIG, workload="double Mach reflection, [0,4]x[0,1], 64x16 base + 3 levels along the "
                                       "shock (the 1/16-size instance of the GPU arm's mesh)",
                  elements=int(m.n_elems), dofs=int(nodes), same_config=False, precision="fp64",
                  parallelism=f"{used} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
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
