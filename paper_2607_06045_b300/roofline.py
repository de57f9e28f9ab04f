"""Algorithmic FP64 work per node and stage of the element pass (the roofline
numerator).

B300 runs FP64 at 1/64 of the FP32 rate (measured 1.20 TFLOP/s with DFMA),
so the element pass is bound by the FP64 pipe; HBM traffic (about 100 bytes
per node and stage against 6.5 TB/s) is two orders of magnitude below it.
Work is counted in FP64 pipe instructions that the method's formulas need, for
an interior node of the limited scheme at N = 3 (counts scale with N as the
pair and interface counts below): an add, multiply, compare, min/max or fused
multiply-add is one instruction; a division, square root or logarithm costs
the number of DFMA-equivalents that idp_probe_pipes measures for CUDA's FP64
routine. Each instruction counts as 2 DFMA-equivalent flops, the unit of the
measured peak. In the FP32 form the flux arithmetic runs in FP32 and only the
FP64 instructions (including the FP64<->FP32 conversions the form needs) are
counted. Conforming face fluxes are counted once per face.
"""
from __future__ import annotations

from dataclasses import dataclass


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
    facen = 2.0 / NP              # face-node flux evaluations per node (one per face)
    pairs = float(N)              # two-point fluxes per node (symmetric, once per pair)
    sbar = N * (N + 1) * (N + 2) / 6.0   # (pair, interface) contributions per row
    fp64 = precision == 0
    r = {}
    # a1 node preparation: 1/rho, v, p, c, beta, ln rho, ln p (FP32 form: the
    # four conversions of the state)
    r["a1_node_prep"] = Ops(inst=9, div=2, sqrt=1, log=2) if fp64 else Ops(inst=6)
    # a2 two-point fluxes: two log means sharing one division, Ranocha's flux
    r["a2_pair_fluxes"] = pairs * Ops(inst=40, div=1) if fp64 else Ops()
    # a2 Sbar contraction (one FMA per contribution and variable) and scaling
    r["a2_sbar_contraction"] = (Ops(inst=2 * sbar * 4 / NP) if fp64 else Ops()) + ifn * Ops(inst=5 if fp64 else 2)
    # a3 low-order subcell flux, graph viscosity, bar state, 2d
    r["a3_fv_subcell"] = ifn * (Ops(inst=36, div=1) if fp64 else Ops(inst=15))
    # a4 conforming/boundary LLF flux of the face node, its bar state and 2d
    r["a4_face_flux"] = facen * (Ops(inst=42, div=2, sqrt=1) if fp64 else Ops(inst=29))
    # a6/a7 low-order update, bar-state/positivity bounds, scaled pressure
    # solve coefficients, tolerance, dt check (+ FP32 copies in the FP32 form)
    r["a6_a7_update_bounds"] = Ops(inst=55 if fp64 else 63)
    # a8 antidiffusive fluxes and exemption (per interface), Zalesak factors
    r["a8_zalesak"] = ifn * Ops(inst=9 if fp64 else 13) + Ops(inst=26)
    # a8 pressure: per interface the admissibility of the full correction at
    # both end points, certified in FP32 (FP64 only when undecided)
    r["a8_pressure"] = ifn * Ops(inst=6)
    # a10 blend, stage combination, statistics
    r["a10_blend_stage"] = Ops(inst=45)
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
