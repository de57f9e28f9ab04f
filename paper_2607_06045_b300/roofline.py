"""Algorithmic work per node and stage of the element pass (roofline numerator).

The element pass is bound by the FP64 pipe (B300 runs FP64 at 1/64 of the
FP32 rate), so its roofline is FP64 arithmetic: work is counted in
DFMA-equivalent flops. An add, subtract, multiply, compare, min, max or
absolute value counts 1 flop, a fused multiply-add 2; division, square root
and logarithm count as the FP64 pipe time of CUDA's routines, measured by
idp_probe_pipes in DFMA-equivalents (2 flops each). The counts follow the
formulas of the element pass row by row (node preparation, pair fluxes and
their Sbar contraction, low-order subcell fluxes, face fluxes, low-order
update and bounds, Zalesak and pressure limiting, blend and stage update) for
an interior node in the limited mode. Conforming face fluxes are counted once
per face (the algorithm needs one evaluation per face). The FP32 form moves
the node primitives' logs, square roots and the pair, subcell and face flux
arithmetic to FP32; what stays FP64 is counted.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class Ops:
    flops: float = 0.0   # add/sub/mul/cmp-class FP64 operations (FMA = 2)
    div: float = 0.0
    sqrt: float = 0.0
    log: float = 0.0

    def __add__(self, o):
        return Ops(self.flops + o.flops, self.div + o.div, self.sqrt + o.sqrt, self.log + o.log)

    def __mul__(self, k):
        return Ops(self.flops * k, self.div * k, self.sqrt * k, self.log * k)

    __rmul__ = __mul__

    def dfma_flops(self, w_div, w_sqrt, w_log):
        """DFMA-equivalent flops given the routines' costs in DFMA-equivalents."""
        return self.flops + 2.0 * (w_div * self.div + w_sqrt * self.sqrt + w_log * self.log)


def element_ops_per_node(N: int, precision: int = 0, stage_comb: float = 2.0 / 3.0) -> dict:
    """FP64 operations per node and stage of the limited element pass, by row.

    stage_comb: average fraction of stages with the SSP combination (2 of 3).
    """
    NP = N + 1
    ifn = 2.0 * N / NP            # interior subcell interfaces per node
    facen = 2.0 / NP              # face-node flux evaluations per node (one per face)
    pairs = float(N)              # two-point fluxes per node (symmetric, once per pair)
    sbar_pairs = N * (N + 1) * (N + 2) / 6.0   # pairs summed per row over its interfaces
    fp64 = precision == 0
    rows = {}
    # a1 node preparation: 1/rho, v, p, c, beta, ln rho, ln beta
    prep = Ops(flops=8, div=4)
    if fp64:
        prep = prep + Ops(sqrt=1, log=2)
    rows["a1_node_prep"] = prep
    # a2 pair fluxes (two log means, averages, Ranocha's energy flux)
    rows["a2_pair_fluxes"] = pairs * Ops(flops=39, div=2) if fp64 else Ops()
    # a2 Sbar contraction into subcell fluxes (FMA per pair, variable), then
    # the weight * face-Jacobian scaling per interface
    sb = Ops(flops=2 * (2 * sbar_pairs * 4 * 2) / NP + 8 * ifn)
    rows["a2_sbar_contraction"] = sb if fp64 else Ops(flops=8 * ifn)
    # a3 low-order subcell fluxes, graph viscosity, bar state (FP64 part: the
    # bar state and the 2d sum; the flux in the FP32 form)
    rows["a3_fv_subcell"] = ifn * (Ops(flops=45, div=1) if fp64 else Ops(flops=9, div=1))
    # a4 conforming face LLF flux, its bar state and 2d
    rows["a4_face_flux"] = facen * (Ops(flops=64, div=7, sqrt=2) if fp64 else Ops(flops=12, div=5))
    # a6/a7 low-order update, density bounds, pmin, tolerance, dt check
    rows["a6_a7_update_bounds"] = Ops(flops=55, div=2)
    # a8 Zalesak density factors
    rows["a8_zalesak"] = Ops(flops=50, div=3)
    # a8 pressure: per interface two closed-form admissibility checks
    rows["a8_pressure"] = ifn * Ops(flops=84, div=1)
    # a10 blend, stage combination, stats and violation checks
    rows["a10_blend_stage"] = Ops(flops=51 + 12 * stage_comb, div=1)
    total = Ops()
    for v in rows.values():
        total = total + v
    rows["total"] = total
    return rows


def element_flops(N: int, precision: int, w_div: float, w_sqrt: float, w_log: float) -> float:
    """DFMA-equivalent FP64 flops per node and stage of the element pass."""
    return element_ops_per_node(N, precision)["total"].dfma_flops(w_div, w_sqrt, w_log)


# Algorithmic HBM bytes per node and stage: read u^(s) (32 B), read u^n in
# two of three stages (64/3 B), write u^(s+1) (32 B); face traces and mesh
# tables are re-reads of data already counted.
BYTES_PER_NODE_STAGE = 32.0 + 64.0 / 3.0 + 32.0
