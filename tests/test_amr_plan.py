"""The library's AMR plan (host C++, no GPU needed) against the oracle's
plan (oracle/amr.py): identical new leaves, kinds and sources on hand-made
and seeded cases, including balance propagation across periodic boundaries
and a DMR-sized mesh with the oracle's density indicators; argument errors.
"""
import numpy as np
import pytest

import oracle
from oracle import amr
from paper_2607_06045_b300 import idp
from paper_2607_06045_b300 import workloads as W


def _both(mesh, ind, **kw):
    po = amr.Params(**kw)
    pc = idp.amr_params(**kw)
    a = amr.plan(mesh, ind, po)
    b = idp.idp_amr_plan(mesh, ind, pc)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    return a


def _family_random(mesh, seed):
    rng = np.random.default_rng(seed)
    cell = rng.uniform(0, 1, (mesh.nx0, mesh.ny0))
    return np.array([cell[x >> l, y >> l] for l, x, y in zip(mesh.level.tolist(), mesh.ix.tolist(), mesh.iy.tolist())])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plan_matches_oracle_random(seed):
    m = W.square_mesh()
    ind = _family_random(m, seed)
    pl = _both(m, ind, refine_threshold=0.7, coarsen_threshold=0.4, min_level=0, max_level=3)
    assert (pl[3] == 1).any()
    mesh2 = W.Mesh(nx0=m.nx0, ny0=m.ny0, box=m.box, level=pl[0], ix=pl[1], iy=pl[2], bc=m.bc)
    assert W.check_balanced(mesh2)


@pytest.mark.parametrize("periodic", [False, True])
def test_plan_matches_oracle_balance(periodic):
    bc = (W.BC_PERIODIC,) * 4 if periodic else (W.BC_OUTFLOW,) * 4
    m = W.box_refined_mesh(4, 4, (0.0, 0.0, 1.0, 1.0), (0.0, 0.0, 0.25, 1.0), bc=bc)
    ind = np.full(m.n_elems, 0.2)
    ind[[k for k in range(m.n_elems) if m.level[k] == 1 and m.ix[k] == 0]] = 0.9
    _both(m, ind, refine_threshold=0.5, coarsen_threshold=0.1, max_level=3)
    # everything coarsens where it can
    _both(m, np.zeros(m.n_elems), refine_threshold=0.5, coarsen_threshold=0.1, max_level=3)


def test_plan_matches_oracle_dmr_indicators():
    m = W.dmr_mesh()
    u = W.dmr_state(m, 3)
    ind = amr.indicators(u, 3, amr.Params(indicator=amr.IND_MAX))
    pl = _both(m, ind, indicator=amr.IND_MAX, refine_threshold=0.3, coarsen_threshold=0.01, min_level=0,
               max_level=4)
    assert (pl[3] == 1).any() and (pl[3] == 2).any()


def test_plan_argument_errors():
    m = W.uniform_mesh(2, 2, level=1)
    ind = np.ones(m.n_elems)
    import ctypes as C
    d, keep = idp.mesh_desc(m)
    p = idp.amr_params(max_level=2)
    n = C.c_int32()
    cap = 4
    buf8, bufs = np.zeros(cap, np.int8), [np.zeros(cap * 4, np.int32) for _ in range(4)]
    ip = C.POINTER(C.c_int32)
    rc = idp.lib().idp_amr_plan(C.byref(d), ind.ctypes.data_as(C.POINTER(C.c_double)), C.byref(p), cap, C.byref(n),
                                buf8.ctypes.data_as(C.POINTER(C.c_int8)), *(b.ctypes.data_as(ip) for b in bufs))
    assert rc == idp.IDP_E_ARG and n.value == 4 * m.n_elems   # capacity too small; the size is reported
    bad = idp.amr_params(max_level=1, min_level=2)
    with pytest.raises(Exception):
        idp.idp_amr_plan(m, ind, bad)
    # an unbalanced input mesh
    mu = W.Mesh(nx0=2, ny0=1, box=(0.0, 0.0, 2.0, 1.0), level=np.array([0] + [2] * 16, np.int8),
                ix=np.array([0] + [4 + a for a in range(4) for b in range(4)], np.int32),
                iy=np.array([0] + [b for a in range(4) for b in range(4)], np.int32), bc=(W.BC_OUTFLOW,) * 4)
    with pytest.raises(Exception):
        idp.idp_amr_plan(mu, np.zeros(mu.n_elems))


def test_transfer_argument_errors_without_gpu():
    """idp_amr_transfer checks the plan before it touches the GPU."""
    import ctypes as C
    L = idp.lib()
    ip = C.POINTER(C.c_int32)
    dummy = C.c_void_p(16)   # never dereferenced: every case below fails its checks first

    def call(kind, src, n_old=4, N=3, gamma=1.4, eps=1e-10):
        kind = np.ascontiguousarray(kind, np.int32)
        src = np.ascontiguousarray(src, np.int32).reshape(-1, 4)
        return L.idp_amr_transfer(N, gamma, dummy, n_old, dummy, len(kind), kind.ctypes.data_as(ip),
                                  src.ctypes.data_as(ip), eps, None, None)
    assert call([0], [[7, -1, -1, -1]]) == idp.IDP_E_ARG                   # source out of range
    assert call([1, 1, 1], [[0, 0, -1, -1], [0, 1, -1, -1], [0, 2, -1, -1]]) == idp.IDP_E_ARG   # short family
    assert call([1, 1, 1, 1], [[0, 0, -1, -1], [0, 1, -1, -1], [0, 3, -1, -1], [0, 2, -1, -1]]) == idp.IDP_E_ARG
    assert call([2], [[0, 1, 2, 9]]) == idp.IDP_E_ARG                      # coarsened child out of range
    assert call([3], [[0, -1, -1, -1]]) == idp.IDP_E_ARG                   # unknown kind
    assert call([0], [[0, -1, -1, -1]], N=8) == idp.IDP_E_ARG              # degree beyond the library's
    assert call([0], [[0, -1, -1, -1]], gamma=1.0) == idp.IDP_E_ARG
    assert call([0], [[0, -1, -1, -1]], eps=-1.0) == idp.IDP_E_ARG
