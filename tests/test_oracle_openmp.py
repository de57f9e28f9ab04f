"""The OpenMP build of the oracle (the all-cores CPU baseline) gives the
serial build's bits: its parallel loops write disjoint outputs and every sum
across them stays serial."""
import os

import numpy as np
import pytest

import oracle
from paper_2607_06045_b300 import workloads as W


@pytest.mark.parametrize("limiting", [1, 2, 3])
def test_openmp_build_is_bit_identical(limiting):
    m = W.square_mesh()
    u = W.disc_wave_state(m, 3)
    outs = []
    for path in (oracle.build(), oracle.build_omp()):
        with oracle.using(path) as L:
            L.orc_set_threads(max(2, min(4, os.cpu_count() or 2)))
            o = oracle.Oracle(m, 3)
            dt = o.dt(u, cfl=0.5)
            r, ut = o.stage(u, 0.0, dt, limiting=limiting)
            un, t, dts, st = o.step(u, 3, cfl=0.5, limiting=limiting)
            outs.append((r, ut, un, dts, st))
    for a, b in zip(outs[0][:4], outs[1][:4]):
        assert np.array_equal(a, b)
    assert outs[0][4] == outs[1][4]
