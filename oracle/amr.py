"""Plain reference of one adaptive-mesh-refinement step (test infrastructure):
element indicators, the adaptation plan (one level of refinement or
coarsening per step with 2:1 face balance), and the solution transfer with
the Zhang-Shu positivity fix of Sec. 2.4 (readings R26-R28).

TEST INFRASTRUCTURE ONLY; see the package docstring. Per-element arithmetic
(indicators, interpolation, projection, scaling) is the C oracle's; this
module holds the bookkeeping written as plain loops over dictionaries.

The plan (R28): an element is marked for refinement when its indicator
exceeds refine_threshold and its level is below max_level, for coarsening
when it is below coarsen_threshold and its level above min_level.
Coarsening needs all four children of a parent to be leaves marked for it,
otherwise their marks are dropped. Then, while two face neighbours would end
two or more levels apart, the coarser one gives up its coarsening (with its
whole family) or, if it was not coarsening, is refined. New elements follow
the old order: a refined leaf becomes its four children (child c = cx + 2 cy)
in place, a coarsened family becomes its parent at its first member's place.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _d, lib

IND_HENNEMANN, IND_LOHNER, IND_MAX = 0, 1, 2
VAR_DENSITY, VAR_PRESSURE = 0, 1


@dataclass
class Params:
    indicator: int = IND_HENNEMANN
    variable: int = VAR_DENSITY
    refine_threshold: float = 0.5
    coarsen_threshold: float = 0.05
    min_level: int = 0
    max_level: int = 3
    lohner_filter: float = 0.2
    zs_threshold: float = 1e-10


def _setup():
    L = lib()
    if not getattr(L, "_amr_ready", False):
        dp = C.POINTER(C.c_double)
        L.orc_lohner.restype = C.c_double
        L.orc_lohner.argtypes = [C.c_int, C.c_double, dp]
        L.orc_refine.argtypes = [C.c_int, dp, dp]
        L.orc_coarsen.argtypes = [C.c_int, dp, dp]
        L.orc_zhang_shu.restype = C.c_double
        L.orc_zhang_shu.argtypes = [C.c_int, C.c_double, C.c_int, dp, dp, C.c_double]
        L._amr_ready = True
    return L


def element_values(u, e, variable, gamma):
    """Nodal density or pressure of element e, [np][np] (j, i)."""
    q = u[:, e]
    if variable == VAR_DENSITY:
        return np.ascontiguousarray(q[0])
    return np.ascontiguousarray((gamma - 1.0) * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / q[0]))


def indicators(u, N, params: Params, gamma=1.4):
    """Per-element indicator (Hennemann et al.'s modal energy indicator of
    R20, the Loehner-type indicator of R27, or the larger of the two)."""
    from . import indicator as hennemann
    L = _setup()
    K = u.shape[1]
    out = np.zeros(K)
    for e in range(K):
        v = element_values(u, e, params.variable, gamma)
        h = hennemann(N, v) if params.indicator in (IND_HENNEMANN, IND_MAX) else 0.0
        lo = L.orc_lohner(N, params.lohner_filter, _d(v)) if params.indicator in (IND_LOHNER, IND_MAX) else 0.0
        out[e] = max(h, lo)
    return out


def plan(mesh, ind, params: Params):
    """(level, ix, iy, kind, src) of the adapted mesh; kind 0 copy (src[0]
    the old element), 1 child (src[0] the old parent, src[1] the child
    position), 2 coarsened parent (src the four old children in child
    order)."""
    lev = [int(x) for x in mesh.level]
    ix = [int(x) for x in mesh.ix]
    iy = [int(x) for x in mesh.iy]
    K = len(lev)
    key = {(lev[e], ix[e], iy[e]): e for e in range(K)}
    mark = [0] * K
    for e in range(K):
        if ind[e] > params.refine_threshold and lev[e] < params.max_level:
            mark[e] = 1
        elif ind[e] < params.coarsen_threshold and lev[e] > params.min_level:
            mark[e] = -1

    def family(e):
        l, x, y = lev[e], ix[e], iy[e]
        px, py = x >> 1, y >> 1
        return [key.get((l, 2 * px + cx, 2 * py + cy), -1) for cy in (0, 1) for cx in (0, 1)]

    for e in range(K):
        if mark[e] == -1:
            f = family(e)
            if any(m < 0 or mark[m] != -1 for m in f):
                for m in f:
                    if m >= 0 and mark[m] == -1:
                        mark[m] = 0
    perx, pery = mesh.bc[0] == 0, mesh.bc[2] == 0

    def neighbours(e, s):
        """Leaves adjacent to leaf e across side s (same level, coarser, or
        the two finer ones)."""
        l, x, y = lev[e], ix[e], iy[e]
        nx, ny = mesh.nx0 << l, mesh.ny0 << l
        qx = x + (-1 if s == 0 else 1 if s == 1 else 0)
        qy = y + (-1 if s == 2 else 1 if s == 3 else 0)
        if qx < 0 or qx >= nx:
            if not perx:
                return []
            qx %= nx
        if qy < 0 or qy >= ny:
            if not pery:
                return []
            qy %= ny
        if (l, qx, qy) in key:
            return [key[(l, qx, qy)]]
        if l > 0 and (l - 1, qx >> 1, qy >> 1) in key:
            return [key[(l - 1, qx >> 1, qy >> 1)]]
        if s < 2:
            cx = 1 if s == 0 else 0
            return [key[(l + 1, 2 * qx + cx, 2 * qy + cy)] for cy in (0, 1)]
        cy = 1 if s == 2 else 0
        return [key[(l + 1, 2 * qx + cx, 2 * qy + cy)] for cx in (0, 1)]

    changed = True
    while changed:
        changed = False
        for e in range(K):
            fe = lev[e] + mark[e]
            for s in range(4):
                for f in neighbours(e, s):
                    if lev[f] + mark[f] - fe >= 2:
                        if mark[e] == -1:
                            for m in family(e):
                                if m >= 0:
                                    mark[m] = 0
                        else:
                            mark[e] = 1
                        fe = lev[e] + mark[e]
                        changed = True
    out_l, out_x, out_y, kind, src = [], [], [], [], []
    for e in range(K):
        l, x, y = lev[e], ix[e], iy[e]
        if mark[e] == 1:
            for c in range(4):
                out_l.append(l + 1); out_x.append(2 * x + (c & 1)); out_y.append(2 * y + (c >> 1))
                kind.append(1); src.append([e, c, -1, -1])
        elif mark[e] == -1:
            f = family(e)
            if min(f) == e:
                out_l.append(l - 1); out_x.append(x >> 1); out_y.append(y >> 1)
                kind.append(2); src.append(f)
        else:
            out_l.append(l); out_x.append(x); out_y.append(y)
            kind.append(0); src.append([e, -1, -1, -1])
    return (np.array(out_l, np.int8), np.array(out_x, np.int32), np.array(out_y, np.int32),
            np.array(kind, np.int32), np.array(src, np.int32).reshape(-1, 4))


def element_mean(q):
    """Mean of an element's nodal states q[4][np][np] under the LGL quadrature."""
    N = q.shape[1] - 1
    from . import lgl
    _, w = lgl(N)
    return np.einsum("vji,j,i->v", q, w, w) / 4.0


def transfer(u, N, pl, gamma=1.4, eps=1e-10):
    """State on the adapted mesh: copies, refined children (interpolation),
    coarsened parents (L2 projection), then the Zhang-Shu scaling of each
    refined family toward the old parent's mean and of each coarsened parent
    toward its own mean. Returns (u_new, number of scaled families)."""
    L = _setup()
    _, _, _, kind, src = pl
    np_ = N + 1
    Kn = len(kind)
    un = np.zeros((4, Kn, np_, np_))
    scaled = 0
    e = 0
    while e < Kn:
        k = kind[e]
        if k == 0:
            un[:, e] = u[:, src[e, 0]]
            e += 1
        elif k == 1:
            p = src[e, 0]
            parent = np.ascontiguousarray(u[:, p])
            ch = np.zeros((4, 4, np_, np_))
            L.orc_refine(N, _d(parent), _d(ch))
            fam = np.ascontiguousarray(ch)
            ref = np.ascontiguousarray(element_mean(parent))
            th = L.orc_zhang_shu(N, gamma, 4, _d(fam), _d(ref), eps)
            scaled += 0.0 <= th < 1.0
            for c in range(4):
                un[:, e + c] = fam[c]
            e += 4
        else:
            ch = np.ascontiguousarray(np.stack([u[:, m] for m in src[e]]))
            par = np.zeros((4, np_, np_))
            L.orc_coarsen(N, _d(ch), _d(par))
            ref = np.ascontiguousarray(element_mean(par))
            par = np.ascontiguousarray(par)
            th = L.orc_zhang_shu(N, gamma, 1, _d(par), _d(ref), eps)
            scaled += 0.0 <= th < 1.0
            un[:, e] = par
            e += 1
    return un, scaled
