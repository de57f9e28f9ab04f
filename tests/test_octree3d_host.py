"""The 3D octree connectivity of the CUDA library's host runtime
(idp3d_octree_tables, include/idp_dgsem3d.h), checked on the CPU without a
GPU: the mortar table equals the 3D oracle's and the one found from the leaf
boxes alone; the face-neighbour table is symmetric, marks boundaries only on
non-periodic sides of the box and points each mortar side at its own slots;
the mortar-node count equals the distinct nodes on mortar faces; unbalanced,
gapped, overlapping and out-of-range leaf sets are rejected.
"""
import numpy as np
import pytest

from oracle import o3d
from paper_2607_06045_b300 import idp
from paper_2607_06045_b300 import workloads as W
from test_oracle3d_mortar import face_nodes, geometric_mortars

UNIT = (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
MID = (0.34, 0.34, 0.34, 0.66, 0.66, 0.66)


def meshes():
    out = [W.box_refined_mesh3(3, 3, 3, UNIT, MID),
           W.box_refined_mesh3(3, 3, 3, UNIT, MID, inside=False,
                               bc=(W.BC_WALL, W.BC_WALL, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_PERIODIC, W.BC_PERIODIC)),
           W.extruded_mesh3(W.box_refined_mesh(3, 2, (0.0, 0.0, 0.9, 0.6), (0.25, 0.2, 0.6, 0.45), base_level=1))[0]]
    out += [W.random_octree3(3, 2, 2, seed=s, n_refine=5, max_level=2) for s in (1, 3)]
    out.append(W.random_octree3(2, 3, 2, seed=5, n_refine=4, max_level=2,
                                bc=(W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_WALL, W.BC_WALL)))
    return out


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2607_06045_b300 import build
    build.build()


@pytest.mark.parametrize("k", range(6))
def test_mortar_table_matches_oracle_and_geometry(k):
    m = meshes()[k]
    info, _, _ = idp.octree_tables3(m, 2)
    assert len(info) > 0
    assert np.array_equal(info, o3d.Oracle3D(m, 2).mortars())
    geo = geometric_mortars(m)
    assert {(int(t[0]), int(t[1]), int(t[2])): [int(x) for x in t[3:]] for t in info} == geo


@pytest.mark.parametrize("N", [1, 3])
@pytest.mark.parametrize("k", range(6))
def test_neighbour_table(k, N):
    m = meshes()[k]
    info, nbr, MN = idp.octree_tables3(m, N)
    NR = (N + 1) ** 2
    Q = 5 * NR
    K = m.n_elems
    Lm = int(m.level.max())
    n0 = (m.nx0, m.ny0, m.nz0)
    c = np.stack([m.ix, m.iy, m.iz], 1).astype(np.int64)
    for e in range(K):
        for s in range(6):
            v = int(nbr[e, s])
            d, hi = s // 2, s & 1
            if v >= 0:
                assert nbr[v, s ^ 1] == e
                assert m.level[v] == m.level[e]
            elif v == -1:
                # a boundary side lies on the box's boundary, which is not periodic
                edge = (n0[d] << int(m.level[e])) - 1 if hi else 0
                assert c[e, d] == edge and m.bc[s] != W.BC_PERIODIC
            else:
                slot = -2 - v
                mo, f = slot // Q, (slot % Q) // NR
                assert slot % NR == 0
                t = info[mo]
                if f == 0:
                    assert t[1] == e and t[0] == d and t[2] == hi
                else:
                    assert t[3 + f - 1] == e and t[0] == d and t[2] == 1 - hi
    # every mortar's five faces point at it
    for mo, t in enumerate(info):
        d, L, low = int(t[0]), int(t[1]), int(t[2])
        assert nbr[L, 2 * d + low] == -2 - mo * Q
        for p in range(4):
            assert nbr[t[3 + p], 2 * d + (1 - low)] == -2 - (mo * Q + (1 + p) * NR)
    # mortar nodes: the distinct nodes on mortar faces
    nodes = set()
    for t in info:
        d, L, low = int(t[0]), int(t[1]), int(t[2])
        nodes |= face_nodes(L, 2 * d + low, N)
        for p in range(4):
            nodes |= face_nodes(int(t[3 + p]), 2 * d + 1 - low, N)
    assert MN == len(nodes)
    assert Lm <= 2


def test_uniform_grid_has_no_mortars():
    g = W.Grid3(3, 2, 4, bc=(W.BC_WALL, W.BC_WALL) + (W.BC_PERIODIC,) * 4)
    lev = np.zeros(g.n_elems, np.int8)
    e = np.arange(g.n_elems)
    m = W.Mesh3(3, 2, 4, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), lev, (e % 3).astype(np.int32),
                ((e // 3) % 2).astype(np.int32), (e // 6).astype(np.int32), bc=g.bc)
    info, nbr, MN = idp.octree_tables3(m, 2)
    assert len(info) == 0 and MN == 0
    ex, ey, ez = e % 3, (e // 3) % 2, e // 6
    assert np.array_equal(nbr[:, 1], np.where(ex < 2, e + 1, -1))
    assert np.array_equal(nbr[:, 3], ez * 6 + ((ey + 1) % 2) * 3 + ex)
    assert np.array_equal(nbr[:, 5], ((ez + 1) % 4) * 6 + ey * 3 + ex)


def _with(m, level, ix, iy, iz):
    return W.Mesh3(m.nx0, m.ny0, m.nz0, m.box, np.array(level, np.int8), np.array(ix, np.int32),
                   np.array(iy, np.int32), np.array(iz, np.int32), bc=m.bc)


def test_rejects_bad_leaf_sets():
    m = W.box_refined_mesh3(3, 3, 3, UNIT, MID)
    lev, ix, iy, iz = (list(a) for a in (m.level, m.ix, m.iy, m.iz))
    # a level jump of two: one small child refined again
    k = lev.index(1)
    a, b, c = ix[k], iy[k], iz[k]
    j2 = ([x for i, x in enumerate(lev) if i != k] + [2] * 8,
          [x for i, x in enumerate(ix) if i != k] + [2 * a + (q & 1) for q in range(8)],
          [x for i, x in enumerate(iy) if i != k] + [2 * b + ((q >> 1) & 1) for q in range(8)],
          [x for i, x in enumerate(iz) if i != k] + [2 * c + (q >> 2) for q in range(8)])
    bad = [_with(m, *j2),
           _with(m, lev[1:], ix[1:], iy[1:], iz[1:]),                        # a gap
           _with(m, lev + [0], ix + [ix[0]], iy + [iy[0]], iz + [iz[0]]),    # a duplicate
           _with(m, lev + [1], ix + [2 * ix[0]], iy + [2 * iy[0]], iz + [2 * iz[0]]),   # an overlap
           _with(m, lev[:-1] + [0], ix[:-1] + [3], iy[:-1] + [0], iz[:-1] + [0])]       # out of range
    for b in bad:
        with pytest.raises(idp.IdpError):
            idp.octree_tables3(b, 2)
