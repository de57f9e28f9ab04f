"""Op counts of the method from the oracle's counting build (opcount.cpp).

TEST AND MEASUREMENT INFRASTRUCTURE: the tests call it, and running it as a
script writes the work table that the benchmark's roofline reads
(``paper_2607_06045_b300/method_work.json``). The numbers are the oracle's
own arithmetic for one SSP-RK3 step, tallied per step of the hot path and
per operation class, normalised per node and stage.

  python -m oracle.opcount            # rewrite the work table
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "opcount.cpp")
_LIB = os.path.join(_HERE, "libopcount.so")
_lib = None

ROWS = ["other", "node_prep", "volume_flux", "subcell_fv", "face_flux", "mortar_flux", "low_update", "bounds",
        "volume_limit", "mortar_limit", "stage", "dt", "reform", "stats"]
CLASSES = ["add", "mul", "div", "sqrt", "log", "exp", "pow", "cmp", "abs"]
# rows that are the method's work (the re-formed quantities and the
# statistics are tallied apart)
METHOD_ROWS = ["node_prep", "volume_flux", "subcell_fv", "face_flux", "mortar_flux", "low_update", "bounds",
               "volume_limit", "mortar_limit", "stage", "dt"]
# flops per operation: every floating-point operation the oracle performs
# counts as one flop (add, multiply, divide, square root, logarithm,
# exponential, power, compare, absolute value), a fixed convention that no
# kernel's own routines enter; the per-class counts stay in the table
WEIGHTS = {k: 1 for k in CLASSES}


def build(force: bool = False) -> str:
    srcs = [_SRC, os.path.join(_HERE, "idp_oracle.c"), os.path.join(_HERE, "idp_oracle3d.c")]
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(p) for p in srcs):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fpermissive", "-w", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", _LIB, _SRC], cwd=_HERE)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
        L.opc_count_step.restype = C.c_int
        L.opc_count_step.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_int, C.POINTER(C.c_int8), ip, ip, ip, dp, dp, dp, dp,
                                     C.c_double, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_longlong)]
        L.opc_n_rows.restype = C.c_int
        L.opc_count_step3.restype = C.c_int
        L.opc_count_step3.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, dp, ip, dp, dp, C.c_double,
                                      C.c_int, C.POINTER(C.c_longlong)]
        _lib = L
    return _lib


def count_step(mesh, N, u, cfl=0.5, limiting=2, gamma=1.4, vflux=0, t0=0.0):
    """One counted SSP-RK3 step. Returns (counts[row][class] as a dict of
    dicts of ints, u after the step)."""
    L = lib()
    nrow = L.opc_n_rows()
    assert nrow == len(ROWS), (nrow, len(ROWS))
    lev = np.ascontiguousarray(mesh.level, dtype=np.int8)
    ix = np.ascontiguousarray(mesh.ix, dtype=np.int32)
    iy = np.ascontiguousarray(mesh.iy, dtype=np.int32)
    bc = np.ascontiguousarray(mesh.bc, dtype=np.int32)
    bcp = np.ascontiguousarray(mesh.bc_prim, dtype=np.float64).reshape(16)
    post = np.ascontiguousarray(mesh.dmr_post, dtype=np.float64)
    pre = np.ascontiguousarray(mesh.dmr_pre, dtype=np.float64)
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    out = np.zeros(nrow * len(CLASSES), dtype=np.int64)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    x0, y0, x1, y1 = mesh.box
    rc = L.opc_count_step(N, gamma, mesh.nx0, mesh.ny0, x0, y0, x1, y1, mesh.n_elems,
                          lev.ctypes.data_as(C.POINTER(C.c_int8)), ix.ctypes.data_as(ip), iy.ctypes.data_as(ip),
                          bc.ctypes.data_as(ip), bcp.ctypes.data_as(dp), post.ctypes.data_as(dp),
                          pre.ctypes.data_as(dp), uu.ctypes.data_as(dp), t0, cfl, limiting, vflux,
                          out.ctypes.data_as(C.POINTER(C.c_longlong)))
    if rc != 0:
        raise ValueError("counting build rejected the mesh")
    cnt = out.reshape(nrow, len(CLASSES))
    return {r: {k: int(cnt[i, j]) for j, k in enumerate(CLASSES)} for i, r in enumerate(ROWS)}, uu


def count_step3(grid, N, u, cfl=0.5, limiting=2, gamma=1.4):
    """One counted SSP-RK3 step of the 3D oracle on a grid (workloads.Grid3)
    or an octree (workloads.Mesh3). Returns (counts[row][class], u after the
    step)."""
    L = lib()
    nrow = L.opc_n_rows()
    box = np.ascontiguousarray(grid.box, dtype=np.float64)
    bc = np.ascontiguousarray(grid.bc, dtype=np.int32)
    bcp = np.ascontiguousarray(grid.bc_prim, dtype=np.float64).reshape(30)
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    out = np.zeros(nrow * len(CLASSES), dtype=np.int64)
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
    if hasattr(grid, "level"):
        lev = np.ascontiguousarray(grid.level, dtype=np.int8)
        ix, iy, iz = (np.ascontiguousarray(a, dtype=np.int32) for a in (grid.ix, grid.iy, grid.iz))
        rc = L.opc_count_step3_leaves(N, C.c_double(gamma), grid.nx0, grid.ny0, grid.nz0, box.ctypes.data_as(dp),
                                      int(lev.size), lev.ctypes.data_as(C.POINTER(C.c_int8)), ix.ctypes.data_as(ip),
                                      iy.ctypes.data_as(ip), iz.ctypes.data_as(ip), bc.ctypes.data_as(ip),
                                      bcp.ctypes.data_as(dp), uu.ctypes.data_as(dp), C.c_double(cfl), limiting,
                                      out.ctypes.data_as(C.POINTER(C.c_longlong)))
    else:
        rc = L.opc_count_step3(N, gamma, grid.nx, grid.ny, grid.nz, box.ctypes.data_as(dp), bc.ctypes.data_as(ip),
                               bcp.ctypes.data_as(dp), uu.ctypes.data_as(dp), cfl, limiting,
                               out.ctypes.data_as(C.POINTER(C.c_longlong)))
    if rc != 0:
        raise ValueError("counting build rejected the grid")
    cnt = out.reshape(nrow, len(CLASSES))
    return {r: {k: int(cnt[i, j]) for j, k in enumerate(CLASSES)} for i, r in enumerate(ROWS)}, uu


def per_node_stage(counts, n_nodes):
    """Counts per node and stage (a step has three stages)."""
    return {r: {k: v / (3.0 * n_nodes) for k, v in cl.items()} for r, cl in counts.items()}


def flops(classes: dict) -> float:
    return float(sum(WEIGHTS[k] * v for k, v in classes.items()))


def work_table(degrees=(1, 2, 3, 4, 5, 6, 7)):
    """Per-node-and-stage op counts by row and class, and the method's flops,
    on the 1/16-size double-Mach-reflection instance (its local limiting,
    shock and quiescent regions in the proportions of the full mesh)."""
    sys.path.insert(0, os.path.dirname(_HERE))
    from paper_2607_06045_b300 import workloads as W
    m = W.dmr_sample_mesh()
    from oracle import Oracle
    table = {"workload": "double Mach reflection, 64x16 base + 3 levels (dmr_sample_mesh), one SSP-RK3 step "
                         "from the initial state, local + positivity limiting, CFL 0.5",
             "elements": int(m.n_elems), "mortars": int(Oracle(m, 1).n_mortars),
             "weights": WEIGHTS, "method_rows": METHOD_ROWS, "degrees": {}}
    for N in degrees:
        u = W.dmr_state(m, N)
        c, _ = count_step(m, N, u)
        nodes = m.n_elems * (N + 1) ** 2
        pn = per_node_stage(c, nodes)
        rows = {r: {"ops": {k: round(v, 4) for k, v in pn[r].items() if v}, "flops": round(flops(pn[r]), 3)}
                for r in ROWS}
        total = sum(rows[r]["flops"] for r in METHOD_ROWS)
        table["degrees"][str(N)] = {"nodes": nodes, "rows": rows, "method_flops_per_node_stage": round(total, 3)}
    return table


def work_table3(degrees=(1, 2, 3, 4), n=10):
    """The same per-node-and-stage counts for the 3D scheme on the 3D blast
    workload at 1/64 of the benchmark's size (n^3 hexahedra, n = 10 against
    40; the same sphere and states)."""
    sys.path.insert(0, os.path.dirname(_HERE))
    from paper_2607_06045_b300 import workloads as W
    g = W.Grid3(n, n, n, bc=(3,) * 6)
    out = {"workload": f"3D blast, {n}^3 hexahedra over [0,1]^3 (sphere r < 0.15 at p = 10 in rho = 1, "
                       "p = 0.1, outflow), one SSP-RK3 step, local limiting, CFL 0.5",
           "elements": int(g.n_elems), "degrees": {}}
    for N in degrees:
        u = W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0)
        c, _ = count_step3(g, N, u)
        nodes = g.n_elems * (N + 1) ** 3
        pn = per_node_stage(c, nodes)
        rows = {r: {"ops": {k: round(v, 4) for k, v in pn[r].items() if v}, "flops": round(flops(pn[r]), 3)}
                for r in ROWS}
        total = sum(rows[r]["flops"] for r in METHOD_ROWS)
        out["degrees"][str(N)] = {"nodes": nodes, "rows": rows, "method_flops_per_node_stage": round(total, 3)}
    return out


MORTAR_ROWS = ["mortar_flux", "mortar_limit"]


def work_table3_octree(degrees=(1, 2, 3, 4), n=8):
    """The 3D scheme's work on a 2:1 octree, split into a part per node and a
    part per mortar: a counted step of the 3D blast on an n^3 base grid with
    [1/4, 3/4]^3 refined once (the octree benchmark's mesh at 1/64 of its
    size); per node and stage the method rows other than the mortar rows, per
    mortar and stage the mortar rows (mortar fluxes and their graph terms,
    mortar limiting)."""
    sys.path.insert(0, os.path.dirname(_HERE))
    from paper_2607_06045_b300 import workloads as W
    from oracle import o3d
    g = W.box_refined_mesh3(n, n, n, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), (0.25, 0.25, 0.25, 0.75, 0.75, 0.75),
                            bc=(3,) * 6)
    out = {"workload": f"3D blast, {n}^3 base hexahedra over [0,1]^3 with [1/4, 3/4]^3 refined once "
                       f"({g.n_elems} leaves), one SSP-RK3 step, local limiting, CFL 0.5",
           "elements": int(g.n_elems), "degrees": {}}
    for N in degrees:
        M = o3d.Oracle3D(g, N).M
        u = W.blast3_state(g, N, rho_bg=1.0, p_bg=0.1, rho_in=1.0, p_in=10.0)
        c, _ = count_step3(g, N, u)
        nodes = g.n_elems * (N + 1) ** 3
        pn = per_node_stage(c, nodes)
        pm = {r: {k: v / (3.0 * M) for k, v in c[r].items()} for r in MORTAR_ROWS}
        node_rows = [r for r in METHOD_ROWS if r not in MORTAR_ROWS]
        out["degrees"][str(N)] = {
            "nodes": nodes, "mortars": M,
            "node_flops_per_node_stage": round(sum(flops(pn[r]) for r in node_rows), 3),
            "mortar_flops_per_mortar_stage": round(sum(flops(pm[r]) for r in MORTAR_ROWS), 3),
            "mortar_rows": {r: round(flops(pm[r]), 3) for r in MORTAR_ROWS}}
    return out


TABLE = os.path.join(os.path.dirname(_HERE), "paper_2607_06045_b300", "method_work.json")

if __name__ == "__main__":
    t = work_table()
    t["3d"] = work_table3()
    t["3d_octree"] = work_table3_octree()
    with open(TABLE, "w") as f:
        json.dump(t, f, indent=1, sort_keys=True)
        f.write("\n")
    for N, d in t["degrees"].items():
        print(N, d["method_flops_per_node_stage"], {r: d["rows"][r]["flops"] for r in ROWS})
