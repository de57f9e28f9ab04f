"""Small driver for profiler captures: builds one workload and runs a few
SSP-RK3 steps through the C ABI (no timing, no oracle).

  python -m paper_2607_06045_b300.profile_case --workload dmr --steps 3
"""
import argparse
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="dmr",
                    choices=["dmr", "square", "blast", "batched", "blast3d", "blast3d_octree"])
    ap.add_argument("--n3", type=int, default=40, help="3D: elements per direction")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--N", type=int, default=3)
    ap.add_argument("--epb", type=int, default=0, help="elements per block (0: autotune)")
    ap.add_argument("--grid-mode", type=int, default=0,
                    help="element-pass grid: 0 autotune (one block per batch with --epb), 1 one block per batch, "
                         "2 persistent")
    ap.add_argument("--limiting", type=int, default=2)
    ap.add_argument("--bounds", type=int, default=0, help="0 bar states, 1 low-order solution")
    ap.add_argument("--entropy", type=int, default=0, help="1: entropy bound")
    a = ap.parse_args(argv)
    import torch
    from paper_2607_06045_b300 import build, idp
    from paper_2607_06045_b300 import workloads as W
    build.build()
    if a.workload in ("blast3d", "blast3d_octree"):
        if a.workload == "blast3d":
            g = W.Grid3(a.n3, a.n3, a.n3, bc=(3,) * 6)
        else:   # the n3^3 base grid with [1/4, 3/4]^3 refined once
            g = W.box_refined_mesh3(a.n3, a.n3, a.n3, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0),
                                    (0.25, 0.25, 0.25, 0.75, 0.75, 0.75), bc=(3,) * 6)
        u = W.blast3_state(g, a.N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0)
        ctx = idp.Context3D(g, a.N, limiting=a.limiting, cfl=0.5, precision=a.precision)
        ud = torch.from_numpy(u).cuda()
        t = np.zeros(1)
        ctx.idp3d_step(ud, a.steps, t)
        torch.cuda.synchronize()
        print(f"ok: {a.workload} K={ctx.K} mortars={ctx.n_mortars} steps={a.steps} t={t[0]}")
        return
    if a.workload == "dmr":
        meshes = W.dmr_mesh(); u = W.dmr_state(meshes, a.N)
    elif a.workload == "square":
        meshes = W.square_mesh(); u = W.disc_wave_state(meshes, a.N)
    elif a.workload == "blast":
        meshes, c = W.blast_mesh(); u = W.blast_state(meshes, a.N, c)
    else:
        meshes = W.batch_meshes(256, seed=0)
        rng = np.random.default_rng(1)
        u = W.concat_states([W.riemann4_state(m, a.N, rng) for m in meshes])
    ctx = idp.Context(meshes, a.N, precision=a.precision, limiting=a.limiting, bounds=a.bounds,
                      entropy_bound=a.entropy, cfl=0.5, elems_per_block=a.epb, grid_mode=a.grid_mode)
    ud = torch.from_numpy(u).cuda()
    t = np.zeros(ctx.n_sims)
    stream = torch.cuda.Stream()
    ctx.idp_dgsem_step(ud, a.steps, t, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    print(f"ok: {a.workload} K={ctx.K} M={ctx.M} steps={a.steps} t={t[:3]}")


if __name__ == "__main__":
    main(sys.argv[1:])
