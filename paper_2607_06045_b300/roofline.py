"""Work per node and stage of the hot path's kernels: the roofline numerators.

Two views are kept.

The method's work (``method_*``): the floating-point operations of the
method, counted on the oracle's own arithmetic by its op-counting build for
one SSP-RK3 step of the double-Mach-reflection instance, per step of the hot
path and normalised per node and stage (``method_work.json``, written by
``python -m oracle.opcount`` and checked by the tests). Every operation counts
as one flop. In the FP32 form the flux rows (node preparation, volume,
subcell, face and mortar fluxes) are FP32 work and the rest FP64, as the form
defines them; its roofline time is the FP64 work over the FP64 peak plus the
FP32 work over the FP32 peak.

The issued FP64 view (``element_ops_per_node`` and below) follows the
kernels' own FP64 instruction economy and is kept as the FP64-issue
efficiency beside the method's roofline:

B300 runs FP64 at 1/64 of the FP32 rate (measured 1.20 TFLOP/s with DFMA),
so the element pass is bound by the FP64 pipe; HBM traffic (about 100 bytes
per node and stage against 6.5 TB/s) is two orders of magnitude below it.
Work is counted in FP64 pipe instructions that the method's formulas need, for
an interior node of the limited scheme at N = 3 (counts scale with N as the
pair and interface counts below): an add, multiply, compare, min/max or fused
multiply-add is one instruction; a reciprocal ("div"), square root or
logarithm costs the number of DFMA-equivalents that idp_probe_pipes measures
for the routine the FP64 flux arithmetic uses (Newton-Raphson reciprocal,
Goldschmidt square root, Tang's logarithm). Each instruction counts as 2
DFMA-equivalent flops, the unit of the peak. In the FP32 form the flux
arithmetic runs in FP32 and only the FP64 instructions the form needs are
counted. Conforming face fluxes are counted once per face.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "method_work.json")
_work = None

# rows of the hot path computed in FP32 by the FP32 form
FP32_FORM_FP32_ROWS = ("node_prep", "volume_flux", "subcell_fv", "face_flux", "mortar_flux")
# the kernels that carry each row: the element pass (its face kernel takes
# the face row where it runs), the mortar flux kernel, the mortar limiting
# kernels (the factors and their application share the row) and the time step
ELEMENT_ROWS = ("node_prep", "volume_flux", "subcell_fv", "face_flux", "low_update", "bounds", "volume_limit",
                "stage")
KERNEL_ROWS = {"element": ELEMENT_ROWS, "face": ("face_flux",), "mortar_flux": ("mortar_flux",),
               "mortar_limit": ("mortar_limit",), "dt": ("dt",)}


def method_table() -> dict:
    """The work table of the oracle's counting build."""
    global _work
    if _work is None:
        with open(_TABLE) as f:
            _work = json.load(f)
    return _work


def method_rows(N: int) -> dict:
    """Flops per node and stage of each row of the hot path at degree N."""
    d = method_table()["degrees"][str(N)]
    return {r: v["flops"] for r, v in d["rows"].items()}


def method_flops(N: int, rows, precision: int = 0):
    """(FP64 flops, FP32 flops) per node and stage of the given rows: all FP64
    in the FP64 path; the flux rows in FP32 in the FP32 form."""
    r = method_rows(N)
    f64 = sum(r[k] for k in rows if precision == 0 or k not in FP32_FORM_FP32_ROWS)
    f32 = sum(r[k] for k in rows if precision == 1 and k in FP32_FORM_FP32_ROWS)
    return f64, f32


MORTAR_KERNELS = ("mortar_flux", "mortar_limit")


def method_kernel_work(N: int, precision: int, K: int, face_kernel=None, M=None) -> dict:
    """Per launch: (FP64 flops, FP32 flops) of each kernel's rows over the K
    elements of one launch. The table normalises the mortar rows per node of
    its own mesh; with M (the launch's mortars) they are taken per mortar of
    that mesh and scaled to M, else per node of the K elements. With the face
    kernel the face row is its work and the rest the element kernel's."""
    nodes = K * (N + 1) ** 2
    if face_kernel is None:
        face_kernel = precision == 0
    t = method_table()
    per_mortar = t["degrees"][str(N)]["nodes"] / t["mortars"]
    out = {}
    for name, rows in KERNEL_ROWS.items():
        if name == "face" and not face_kernel:
            continue
        if name == "element" and face_kernel:
            rows = tuple(r for r in rows if r != "face_flux")
        a, b = method_flops(N, rows, precision)
        scale = per_mortar * M if (M is not None and name in MORTAR_KERNELS) else nodes
        out[name] = (a * scale, b * scale)
    if face_kernel:
        # the two-pass time step: its FP32 pass forms the row's quotients at
        # every node, the FP64 pass only in the few elements it picks
        a, b = out.pop("dt")
        out["dt_filter"] = (0.0, a + b)
        out["dt"] = (0.0, 0.0)
    return out


@dataclass
class Ops:
    inst: float = 0.0   # FP64 add/mul/fma/compare/convert instructions
    div: float = 0.0
    sqrt: float = 0.0
    log: float = 0.0

    def __add__(self, o):
        return Ops(self.inst + o.inst, self.div + o.div, self.sqrt + o.sqrt, self.log + o.log)

    def __mul__(self, k):
        return Ops(self.inst * k, self.div * k, self.sqrt * k, self.log * k)

    __rmul__ = __mul__

    def dfma_eq(self, w_div, w_sqrt, w_log):
        """FP64 pipe instructions (DFMA-equivalents)."""
        return self.inst + w_div * self.div + w_sqrt * self.sqrt + w_log * self.log


def element_ops_per_node(N: int, precision: int = 0) -> dict:
    """FP64 work per node and stage of the limited element pass, by row."""
    NP = N + 1
    ifn = 2.0 * N / NP            # interior subcell interfaces per node
    ends = 2.0 * ifn              # interface end points per node
    facen = 2.0 / NP              # face-node flux evaluations per node (one per face)
    pairs = float(N)              # two-point fluxes per node (symmetric, once per pair)
    sbar = N * (N + 1) * (N + 2) / 6.0   # (pair, interface) contributions per row
    fp64 = precision == 0
    r = {}
    # a1 node preparation: 1/rho, v, p, c, beta, ln rho, ln p (the FP32 form
    # forms them in FP32)
    r["a1_node_prep"] = Ops(inst=10, div=2, sqrt=1, log=2) if fp64 else Ops()
    # a2 two-point fluxes: two log means sharing one reciprocal, Ranocha's flux
    r["a2_pair_fluxes"] = pairs * Ops(inst=40, div=1) if fp64 else Ops()
    # a2 Sbar contraction (one FMA per contribution and variable) and scaling
    r["a2_sbar_contraction"] = (Ops(inst=2 * sbar * 4 / NP) + ifn * Ops(inst=5)) if fp64 else Ops()
    # a3 low-order subcell flux, graph viscosity and 2d (flux type), bar state (FP64)
    r["a3_fv_subcell"] = ifn * (Ops(inst=35, div=1) if fp64 else Ops(inst=4))
    # a4 conforming/boundary LLF flux of the face node (flux type), bar state (FP64)
    r["a4_face_flux"] = facen * (Ops(inst=49, div=2, sqrt=1) if fp64 else Ops(inst=5))
    # a6/a7 low-order update (residual sums from the first term), bounds,
    # pressure-solve coefficients
    r["a6_a7_update_bounds"] = Ops(inst=27 + (1 if fp64 else 0))
    # a8 antidiffusive fluxes and exemption (FP64 path), Zalesak sums and factors
    r["a8_zalesak"] = (ifn * Ops(inst=4) if fp64 else Ops()) + ends * Ops(inst=1) + Ops(inst=4)
    # a8 pressure: the admissibility of the full correction at both end
    # points is certified in FP32 (the FP64 solve is rare)
    r["a8_pressure"] = Ops()
    # a10 blend, stage combination (2/3 of the stages), statistics thresholds
    r["a10_blend_stage"] = Ops(inst=ends * 4 + 4 + 8 * 2.0 / 3.0 + 2)
    total = Ops()
    for v in r.values():
        total = total + v
    r["total"] = total
    return r


def element_flops(N: int, precision: int, w_div: float, w_sqrt: float, w_log: float) -> float:
    """DFMA-equivalent FP64 flops (2 per pipe instruction) per node and stage."""
    return 2.0 * element_ops_per_node(N, precision)["total"].dfma_eq(w_div, w_sqrt, w_log)


# Algorithmic HBM bytes per node and stage: read u^(s) (32 B), read u^n in
# two of three stages (64/3 B), write u^(s+1) (32 B); face traces and mesh
# tables are re-reads of data already counted.
BYTES_PER_NODE_STAGE = 32.0 + 64.0 / 3.0 + 32.0


# ---------------------------------------------------------------------------
# The other kernels of a step: algorithmic FP64 work and HBM bytes per unit
# (node, mortar or mortar node), at degree N. Counts follow the kernels'
# formulas in the same units as above; the FP32 form counts only its FP64
# instructions (its FP32 work is far below the FP32 peak).
# ---------------------------------------------------------------------------

def _prim(precision: int) -> Ops:
    """Primitives and wave speed of one state (1/rho, v, p, c)."""
    return Ops(inst=7, div=1, sqrt=1) if precision == 0 else Ops()


def dt_ops_per_node(N: int, precision: int = 0, face: bool = False) -> Ops:
    """k_dt: own wave speeds, the outside wave speed of each face node (one
    per node on average at one face node per element side and node row), the
    2d sum and m / sum. With face = True (the FP64 path's face kernel runs on
    u^n first) the face's wave speed is read, not formed."""
    NP = N + 1
    facen = 4.0 * NP / (NP * NP)
    o = _prim(precision) + (0.0 if face else facen) * _prim(precision)
    if precision == 0:
        o = o + Ops(inst=8 + 2, div=1)
    return o


def mortar_flux_ops_per_mortar(N: int, precision: int = 0) -> Ops:
    """k_mortar_flux: trace primitives, interpolation (FP64), admissibility,
    LLF on the small faces, the sparse pair terms with bar states, the
    projection (FP64 sums) and the slot sums."""
    NP = N + 1
    npair = 3 * NP - 1
    o = Ops(inst=8 * NP * NP)                      # interpolation 2NP x 4 x NP
    o = o + Ops(inst=6 * 2 * NP)                   # admissibility of the interpolated states
    o = o + Ops(inst=8 * NP * NP + 12 * NP)        # projection and scaling
    o = o + Ops(inst=2 * NP * 4 * 3)               # small-face contributions
    o = o + Ops(inst=npair * (5 + 8))              # bar states and slot sums
    if precision == 0:
        o = o + 3 * NP * _prim(0) + 2 * NP * (_prim(0) + Ops(inst=24)) + npair * Ops(inst=22, div=1)
    return o


def mortar_limit_ops_per_slot(precision: int = 0) -> Ops:
    """k_mortar_limit: correction, density factor, pressure factor."""
    return Ops(inst=30, div=3)


def mortar_apply_ops_per_node(precision: int = 0) -> Ops:
    """k_mortar_apply: limited corrections, stage combination, checks."""
    return Ops(inst=35, div=2)


def kernel_work(N: int, precision: int, K: int, M: int, n_mnodes: int, w_div: float, w_sqrt: float,
                w_log: float, face_kernel=None) -> dict:
    """Per launch: (FP64 DFMA-equivalent flops, HBM bytes) of each kernel.
    With the conforming-face kernel (the FP64 path's default element kernel)
    the face fluxes (row a4) are its work and the rest the element kernel's;
    its bytes are the two face-node states it reads and the 52 bytes per face
    node it writes; the time-step kernel then reads the faces' wave speeds."""
    nodes = K * (N + 1) ** 2
    Q = 3 * (N + 1)
    w = (w_div, w_sqrt, w_log)
    if face_kernel is None:
        face_kernel = precision == 0
    rows = element_ops_per_node(N, precision)
    el_flops = element_flops(N, precision, *w) * nodes
    face = {}
    if face_kernel:
        fa = 2.0 * rows["a4_face_flux"].dfma_eq(*w) * nodes
        face = {"face": (fa, (64.0 + 52.0) * 2.0 / (N + 1) * nodes)}
        el_flops -= fa
    return {
        **face,
        "element": (el_flops, BYTES_PER_NODE_STAGE * nodes),
        # without the face kernel the time step reads the wave speeds that its
        # pre-pass wrote from the state (two values per node in the flux type)
        **({} if face_kernel else {"dt_speed": (0.0, (32.0 + 2.0 * (4 if precision else 8)) * nodes)}),
        # with the face kernel the time step's FP32 pass reads the state and
        # the faces' wave speeds and writes one minimum per element; its FP64
        # pass reads those minima (and the few picked elements' data)
        **({"dt_filter": (0.0, (32.0 + 8.0 * 4.0 / (N + 1)) * nodes + 4.0 * K),
            "dt": (0.0, 4.0 * K)} if face_kernel else
           {"dt": (2.0 * dt_ops_per_node(N, precision, face_kernel).dfma_eq(*w) * nodes,
                   2.0 * (4 if precision else 8) * nodes)}),
        "mortar_flux": (2.0 * mortar_flux_ops_per_mortar(N, precision).dfma_eq(*w) * M, (96.0 + 264.0) * (N + 1) * M),
        "mortar_limit": (2.0 * mortar_limit_ops_per_slot(precision).dfma_eq(*w) * Q * M, 112.0 * Q * M),
        "mortar_apply": (2.0 * mortar_apply_ops_per_node(precision).dfma_eq(*w) * n_mnodes, 136.0 * n_mnodes),
    }
