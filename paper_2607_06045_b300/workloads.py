"""Seeded synthetic inputs: quadtree meshes and initial states.

This module generates the inputs that both the CUDA path and the CPU oracle
consume: the leaves of a 2:1 face-balanced Cartesian quadtree (Sec. 3.1: a
leaf at level n belongs to a grid of 2^n elements per base element and
direction; Sec. 2.2: neighbouring elements differ by at most one level) and
the conserved state u[4][K][N+1][N+1] sampled at the nodes of each element.

It holds none of the method's arithmetic. Node positions use numpy's own
Legendre routines (the roots of P_N' plus the two end points); the conserved
state is the ideal-gas map from primitive variables. Everything is seeded with
``numpy.random.default_rng(seed)``.

A mesh is kept as a *level map*: an integer array over the finest cells whose
entry is the level of the leaf covering that cell. Refining a leaf adds one to
all of its cells; leaves are recovered as the aligned blocks of equal level.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

# Boundary kinds, numbered as in the C header (idp_bc).
BC_PERIODIC, BC_WALL, BC_DIRICHLET, BC_OUTFLOW, BC_DMR, BC_JET = 0, 1, 2, 3, 4, 5


@dataclasses.dataclass
class Mesh:
    """Leaves of a quadtree over a box with an nx0 x ny0 level-0 grid."""

    nx0: int
    ny0: int
    box: tuple  # (x0, y0, x1, y1)
    level: np.ndarray  # int8 [K]
    ix: np.ndarray  # int32 [K], index at the leaf's own level
    iy: np.ndarray  # int32 [K]
    bc: tuple = (BC_PERIODIC,) * 4  # sides -x, +x, -y, +y
    bc_prim: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros((4, 4)))  # Dirichlet (rho, v1, v2, p)
    dmr_post: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(4))
    dmr_pre: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(4))

    @property
    def n_elems(self) -> int:
        return int(self.level.shape[0])

    def periodic(self):
        return (self.bc[0] == BC_PERIODIC, self.bc[2] == BC_PERIODIC)


# ----------------------------------------------------------------------------
# level-map quadtree helpers
# ----------------------------------------------------------------------------

def _leaves_from_map(lmap: np.ndarray, L: int):
    """Return (level, ix, iy) of all leaves of a level map with finest level L."""
    nxf, nyf = lmap.shape
    fx, fy = np.meshgrid(np.arange(nxf), np.arange(nyf), indexing="ij")
    shift = (L - lmap).astype(np.int64)
    anchor = ((fx & ((1 << shift) - 1)) == 0) & ((fy & ((1 << shift) - 1)) == 0)
    lev = lmap[anchor].astype(np.int8)
    sx = shift[anchor]
    ix = (fx[anchor] >> sx).astype(np.int32)
    iy = (fy[anchor] >> sx).astype(np.int32)
    # order: by level-0 base cell (row-major in y, then x), then Morton-free
    # simple order within the map scan (x outer, y inner) is kept.
    return lev, ix, iy


def _leaf_centres(lmap, L, nx0, ny0, box):
    """Centre coordinates of the leaf covering each finest cell."""
    x0, y0, x1, y1 = box
    nxf, nyf = lmap.shape
    fx, fy = np.meshgrid(np.arange(nxf), np.arange(nyf), indexing="ij")
    s = (L - lmap).astype(np.int64)
    bx = (fx >> s)
    by = (fy >> s)
    hx = (x1 - x0) / (nx0 * (1 << lmap.astype(np.int64)))
    hy = (y1 - y0) / (ny0 * (1 << lmap.astype(np.int64)))
    return x0 + (bx + 0.5) * hx, y0 + (by + 0.5) * hy, hx, hy


def _neighbour_max(lmap, periodic):
    """Per finest cell, the maximum level among its four face neighbours."""
    px, py = periodic
    out = np.full(lmap.shape, -1, dtype=np.int32)
    a = lmap.astype(np.int32)
    for axis, per in ((0, px), (1, py)):
        for sh in (1, -1):
            if per:
                nb = np.roll(a, sh, axis=axis)
            else:
                nb = np.full_like(a, -1)
                if axis == 0:
                    if sh == 1:
                        nb[1:, :] = a[:-1, :]
                    else:
                        nb[:-1, :] = a[1:, :]
                else:
                    if sh == 1:
                        nb[:, 1:] = a[:, :-1]
                    else:
                        nb[:, :-1] = a[:, 1:]
            out = np.maximum(out, nb)
    return out


def _leaf_reduce_max(lmap, L, cellval):
    """Max of a per-cell value over each leaf, broadcast back to its cells."""
    nxf, nyf = lmap.shape
    fx, fy = np.meshgrid(np.arange(nxf), np.arange(nyf), indexing="ij")
    s = (L - lmap).astype(np.int64)
    # unique leaf key: anchor cell index
    ax = (fx >> s) << s
    ay = (fy >> s) << s
    key = ax * nyf + ay
    best = np.full(nxf * nyf, np.iinfo(np.int64).min, dtype=np.int64)
    np.maximum.at(best, key.ravel(), cellval.astype(np.int64).ravel())
    return best[key]


def balance_2to1(lmap: np.ndarray, L: int, periodic) -> np.ndarray:
    """Refine leaves until face neighbours differ by at most one level."""
    lmap = lmap.copy()
    while True:
        nbm = _neighbour_max(lmap, periodic)
        need = (nbm >= lmap.astype(np.int32) + 2).astype(np.int64)
        flag = _leaf_reduce_max(lmap, L, need) > 0
        if not flag.any():
            return lmap
        lmap = lmap + flag.astype(lmap.dtype)


def refine_where(lmap, L, nx0, ny0, box, fn: Callable, max_level: int):
    """Refine every leaf (below max_level) whose centre (x, y, hx, hy) -> True."""
    cx, cy, hx, hy = _leaf_centres(lmap, L, nx0, ny0, box)
    flag = fn(cx, cy, hx, hy) & (lmap < max_level)
    return lmap + flag.astype(lmap.dtype)


def mesh_from_map(lmap, L, nx0, ny0, box, **kw) -> Mesh:
    lev, ix, iy = _leaves_from_map(lmap, L)
    return Mesh(nx0=nx0, ny0=ny0, box=tuple(float(b) for b in box),
                level=lev, ix=ix, iy=iy, **kw)


def check_balanced(mesh: Mesh) -> bool:
    """True when every face neighbour differs by at most one level."""
    L = int(mesh.level.max()) if mesh.n_elems else 0
    lmap = np.zeros((mesh.nx0 << L, mesh.ny0 << L), dtype=np.int16)
    for l, x, y in zip(mesh.level.tolist(), mesh.ix.tolist(), mesh.iy.tolist()):
        s = L - l
        lmap[x << s:(x + 1) << s, y << s:(y + 1) << s] = l
    nbm = _neighbour_max(lmap, mesh.periodic())
    return bool((nbm <= lmap.astype(np.int32) + 1).all())


# ----------------------------------------------------------------------------
# nodes and states
# ----------------------------------------------------------------------------

def lgl_points(N: int) -> np.ndarray:
    """LGL points from numpy's Legendre class: -1, roots of P_N', +1."""
    if N == 1:
        return np.array([-1.0, 1.0])
    r = np.polynomial.legendre.Legendre.basis(N).deriv().roots()
    r = np.sort(np.real(r))
    return np.concatenate([[-1.0], r, [1.0]])


def node_coords(mesh: Mesh, N: int):
    """x, y of every node, shape [K][N+1][N+1] indexed [e][j][i]."""
    x0, y0, x1, y1 = mesh.box
    lev = mesh.level.astype(np.int64)
    hx = (x1 - x0) / (mesh.nx0 * (1 << lev))
    hy = (y1 - y0) / (mesh.ny0 * (1 << lev))
    cx = x0 + (mesh.ix + 0.5) * hx
    cy = y0 + (mesh.iy + 0.5) * hy
    s = lgl_points(N)
    X = cx[:, None, None] + 0.5 * hx[:, None, None] * s[None, None, :]
    Y = cy[:, None, None] + 0.5 * hy[:, None, None] * s[None, :, None]
    X = np.broadcast_to(X, (mesh.n_elems, N + 1, N + 1)).copy()
    Y = np.broadcast_to(Y, (mesh.n_elems, N + 1, N + 1)).copy()
    return X, Y


def conserved(rho, v1, v2, p, gamma):
    """Ideal-gas conserved state (rho, rho v1, rho v2, E) stacked on axis 0."""
    rho = np.asarray(rho, dtype=np.float64)
    E = p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)
    return np.ascontiguousarray(
        np.stack([rho, rho * v1, rho * v2, E * np.ones_like(rho)], axis=0))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def uniform_mesh(nx0, ny0, box=(0.0, 0.0, 1.0, 1.0), level=0, bc=(BC_PERIODIC,) * 4):
    n = 1 << level
    ix, iy = np.meshgrid(np.arange(nx0 * n), np.arange(ny0 * n), indexing="ij")
    return Mesh(nx0=nx0, ny0=ny0, box=box,
                level=np.full(ix.size, level, dtype=np.int8),
                ix=ix.ravel().astype(np.int32), iy=iy.ravel().astype(np.int32), bc=bc)


def box_refined_mesh(nx0, ny0, box, rbox, base_level=0, bc=(BC_PERIODIC,) * 4):
    """A uniform mesh at base_level with elements whose centre lies in rbox
    refined once more: the statically refined box of Sec. 3.1."""
    L = base_level + 1
    lmap = np.full((nx0 << L, ny0 << L), base_level, dtype=np.int16)
    rx0, ry0, rx1, ry1 = rbox

    def inside(cx, cy, hx, hy):
        return (cx > rx0) & (cx < rx1) & (cy > ry0) & (cy < ry1)

    lmap = refine_where(lmap, L, nx0, ny0, box, inside, L)
    lmap = balance_2to1(lmap, L, (bc[0] == BC_PERIODIC, bc[2] == BC_PERIODIC))
    return mesh_from_map(lmap, L, nx0, ny0, box, bc=bc)


def square_mesh():
    """Periodic unit square, 16 x 16 base grid, the central 4 x 4 block refined
    once: 304 elements and 16 hanging faces."""
    return box_refined_mesh(16, 16, (0.0, 0.0, 1.0, 1.0), (0.375, 0.375, 0.625, 0.625))


def disc_wave_state(mesh: Mesh, N: int, gamma=1.4):
    """Smooth density 1 + 0.5 sin(2 pi x) sin(2 pi y) with a disc r < 0.15 about
    the domain centre at rho = 2, p = 5 (p = 1 elsewhere); u = v = 0.1."""
    X, Y = node_coords(mesh, N)
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    p = np.ones_like(X)
    disc = (X - 0.5) ** 2 + (Y - 0.5) ** 2 < 0.15 ** 2
    rho = np.where(disc, 2.0, rho)
    p = np.where(disc, 5.0, p)
    return conserved(rho, 0.1 * np.ones_like(X), 0.1 * np.ones_like(X), p, gamma)


DMR_POST = np.array([8.0, 8.25 * math.cos(math.pi / 6), -8.25 * math.sin(math.pi / 6), 116.5])
DMR_PRE = np.array([1.4, 0.0, 0.0, 1.0])


def dmr_mesh(seed=0, target=(54000, 66000), max_extra=3, nx0=256, ny0=64):
    """[0,4] x [0,1], 256 x 64 base grid, up to three extra levels where a
    density-jump indicator fires across the 60 degree Mach-10 shock, balanced
    2:1; the indicator threshold is bisected until K lies in ``target``.

    The indicator compares the density of a smoothed shock profile (width
    0.05) between each leaf and its face neighbours; a seeded jitter of 1e-3 in
    the threshold breaks ties between equal jumps."""
    box = (0.0, 0.0, 4.0, 1.0)
    rng = np.random.default_rng(seed)
    jitter = 1.0 + 1e-3 * rng.standard_normal()
    L = max_extra

    def rho_s(x, y):
        d = (x - (1.0 / 6.0 + y / math.sqrt(3.0))) * math.sqrt(3.0) / 2.0
        return DMR_PRE[0] + (DMR_POST[0] - DMR_PRE[0]) * 0.5 * (1.0 - np.tanh(d / 0.05))

    def build(tau):
        lmap = np.zeros((nx0 << L, ny0 << L), dtype=np.int16)
        for _ in range(max_extra):
            cx, cy, hx, hy = _leaf_centres(lmap, L, nx0, ny0, box)
            r = rho_s(cx, cy)
            jump = np.zeros_like(r)
            for axis in (0, 1):
                for sh in (1, -1):
                    nb = np.roll(r, sh, axis=axis)
                    jump = np.maximum(jump, np.abs(nb - r))
            flag = (_leaf_reduce_max(lmap, L, (jump > tau * jitter).astype(np.int64)) > 0)
            flag &= lmap < max_extra
            lmap = balance_2to1(lmap + flag.astype(lmap.dtype), L, (False, False))
        return lmap

    lo, hi = 1e-4, 6.6
    lmap = build(lo)
    for _ in range(40):
        mid = math.sqrt(lo * hi)
        lmap = build(mid)
        K = int((1.0 / (1 << (2 * (L - lmap.astype(np.int64))))).sum())
        if target[0] <= K <= target[1]:
            break
        if K > target[1]:
            lo = mid
        else:
            hi = mid
    m = mesh_from_map(lmap, L, nx0, ny0, box, bc=(BC_DMR,) * 4)
    m.dmr_post = DMR_POST.copy()
    m.dmr_pre = DMR_PRE.copy()
    return m


def dmr_sample_mesh(seed=0):
    """A 1/16-size instance of the same DMR workload (64 x 16 base grid, the
    same three-level shock refinement, K in [3400, 4100]) for CPU timing."""
    return dmr_mesh(seed=seed, target=(3400, 4100), nx0=64, ny0=16)


def dmr_state(mesh: Mesh, N: int, gamma=1.4):
    """Post-shock state left of x = 1/6 + y / sqrt(3), quiescent gas right of it."""
    X, Y = node_coords(mesh, N)
    left = X < 1.0 / 6.0 + Y / math.sqrt(3.0)
    pr = [np.where(left, DMR_POST[k], DMR_PRE[k]) for k in range(4)]
    return conserved(pr[0], pr[1], pr[2], pr[3], gamma)


def batch_meshes(n_sims=256, seed=0):
    """Batched workload: base side s = round(8 * 16**U) per simulation, then 0-2
    refinement levels on 1-4 random rectangular patches, balanced 2:1; outflow
    boundaries on the unit square."""
    rng = np.random.default_rng(seed)
    meshes = []
    for _ in range(n_sims):
        s = int(round(8 * 16 ** rng.uniform()))
        extra = int(rng.integers(0, 3))
        npatch = int(rng.integers(1, 5))
        L = max(extra, 0)
        lmap = np.zeros((s << L, s << L), dtype=np.int16)
        box = (0.0, 0.0, 1.0, 1.0)
        patches = []
        for _p in range(npatch):
            a = rng.uniform(0, 1, 2)
            b = rng.uniform(0, 1, 2)
            patches.append((min(a[0], b[0]), min(a[1], b[1]), max(a[0], b[0]), max(a[1], b[1])))
        for lev in range(extra):
            def inpatch(cx, cy, hx, hy):
                f = np.zeros(cx.shape, dtype=bool)
                for (px0, py0, px1, py1) in patches:
                    f |= (cx > px0) & (cx < px1) & (cy > py0) & (cy < py1)
                return f
            lmap = refine_where(lmap, L, s, s, box, inpatch, extra)
            lmap = balance_2to1(lmap, L, (False, False))
        meshes.append(mesh_from_map(lmap, L, s, s, box, bc=(BC_OUTFLOW,) * 4))
    return meshes


def riemann4_state(mesh: Mesh, N: int, rng: np.random.Generator, gamma=1.4):
    """Seeded four-quadrant Riemann problem split at (0.5, 0.5): rho, p
    log-uniform in [0.1, 10], u, v uniform in [-1, 1] per quadrant."""
    X, Y = node_coords(mesh, N)
    q = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
    rho_q = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 4))
    p_q = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 4))
    u_q = rng.uniform(-1, 1, 4)
    v_q = rng.uniform(-1, 1, 4)
    return conserved(rho_q[q], u_q[q], v_q[q], p_q[q], gamma)


def blast_mesh(seed=0, n0=512):
    """Near-vacuum blast: n0 x n0 base grid on the unit square, two extra levels
    for leaves within r < 0.1 of a seeded centre in [0.3, 0.7]^2, balanced 2:1,
    outflow boundaries. Returns (mesh, centre)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.3, 0.7, 2)
    L = 2
    box = (0.0, 0.0, 1.0, 1.0)
    lmap = np.zeros((n0 << L, n0 << L), dtype=np.int16)
    for _ in range(2):
        def near(cx, cy, hx, hy):
            return (cx - c[0]) ** 2 + (cy - c[1]) ** 2 < 0.1 ** 2
        lmap = refine_where(lmap, L, n0, n0, box, near, L)
        lmap = balance_2to1(lmap, L, (False, False))
    return mesh_from_map(lmap, L, n0, n0, box, bc=(BC_OUTFLOW,) * 4), c


def blast_state(mesh: Mesh, N: int, centre, gamma=1.4):
    """Background rho = 1e-6, p = 1e-9; disc r < 0.05 with rho = 1, p = 1e3."""
    X, Y = node_coords(mesh, N)
    disc = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 < 0.05 ** 2
    rho = np.where(disc, 1.0, 1e-6)
    p = np.where(disc, 1e3, 1e-9)
    z = np.zeros_like(X)
    return conserved(rho, z, z, p, gamma)


# --- high-Mach jet (gamma = 5/3) ---------------------------------------------

JET_IN = np.array([5.0, 800.0, 0.0, 0.4127])      # inflow band (rho, v1, v2, p)
JET_AMBIENT = np.array([0.5, 0.0, 0.0, 0.4127])   # gas at rest
JET_GAMMA = 5.0 / 3.0


def jet_mesh(n0=64, levels=3, half_width=0.1):
    """Astrophysical-jet geometry of Sec. 3 on a static mesh: [-0.5, 0.5]^2,
    n0 x n0 base grid, `levels` extra levels for leaves within |y| < half_width,
    balanced 2:1; jet boundary on the x sides (inflow band |y| <= 0.05 on -x,
    ambient state elsewhere), periodic in y."""
    box = (-0.5, -0.5, 0.5, 0.5)
    lmap = np.zeros((n0 << levels, n0 << levels), dtype=np.int16)
    for _ in range(levels):
        def band(cx, cy, hx, hy):
            return np.abs(cy) < half_width
        lmap = refine_where(lmap, levels, n0, n0, box, band, levels)
        lmap = balance_2to1(lmap, levels, (False, True))
    m = mesh_from_map(lmap, levels, n0, n0, box, bc=(BC_JET, BC_JET, BC_PERIODIC, BC_PERIODIC))
    m.dmr_post = JET_IN.copy()
    m.dmr_pre = JET_AMBIENT.copy()
    return m


def jet_state(mesh: Mesh, N: int, gamma=JET_GAMMA, seed=None):
    """The ambient gas at rest; with a seed, a small seeded perturbation of the
    density (1%) so that the volume fluxes do not vanish before the jet enters."""
    X, Y = node_coords(mesh, N)
    rho = np.full_like(X, JET_AMBIENT[0])
    if seed is not None:
        rng = np.random.default_rng(seed)
        k = rng.integers(1, 4, 2)
        ph = rng.uniform(0, 2 * math.pi, 2)
        rho = rho * (1.0 + 0.01 * np.sin(2 * math.pi * k[0] * X + ph[0]) * np.sin(2 * math.pi * k[1] * Y + ph[1]))
    z = np.zeros_like(X)
    return conserved(rho, z, z, np.full_like(X, JET_AMBIENT[3]), gamma)


# --- smooth test problems ----------------------------------------------------

def density_wave_mesh(base_level):
    """Periodic [-1,1]^2 at base_level with the box [-0.5,0] x [-0.5,0.5] refined
    once (Sec. 3.1)."""
    n = 1 << base_level
    return box_refined_mesh(n, n, (-1.0, -1.0, 1.0, 1.0), (-0.5, -0.5, 0.0, 0.5))


def density_wave_state(mesh, N, t=0.0, gamma=1.4):
    """rho = 2 + 0.98 sin(2 pi (x + y - 0.3 t)), v = (0.1, 0.2), p = 20 (Sec. 3.1),
    exact at time t."""
    X, Y = node_coords(mesh, N)
    rho = 2.0 + 0.98 * np.sin(2 * np.pi * ((X - 0.1 * t) + (Y - 0.2 * t)))
    return conserved(rho, 0.1 * np.ones_like(X), 0.2 * np.ones_like(X), 20.0 * np.ones_like(X), gamma)


def vortex_state(mesh, N, t=0.0, gamma=1.4, centre=(0.0, 0.0), vel=(1.0, 1.0),
                 strength=5.0, period=(10.0, 10.0)):
    """Isentropic vortex advected with ``vel``; exact solution at time t is the
    translated initial state (with periodic images on a period box)."""
    X, Y = node_coords(mesh, N)
    cx = centre[0] + vel[0] * t
    cy = centre[1] + vel[1] * t
    dx = (X - cx + 0.5 * period[0]) % period[0] - 0.5 * period[0]
    dy = (Y - cy + 0.5 * period[1]) % period[1] - 0.5 * period[1]
    r2 = dx * dx + dy * dy
    f = strength / (2 * np.pi) * np.exp(0.5 * (1 - r2))
    T = 1.0 - (gamma - 1) * strength ** 2 / (8 * gamma * np.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1.0 / (gamma - 1))
    p = rho * T
    return conserved(rho, vel[0] - f * dy, vel[1] + f * dx, p, gamma)


def random_state(mesh, N, seed=0, gamma=1.4, rho_range=(0.5, 2.0), p_range=(0.5, 2.0), vmax=0.5):
    """Seeded nodal noise: a rough but admissible state for parity tests."""
    rng = np.random.default_rng(seed)
    shape = (mesh.n_elems, N + 1, N + 1)
    rho = rng.uniform(*rho_range, shape)
    p = rng.uniform(*p_range, shape)
    v1 = rng.uniform(-vmax, vmax, shape)
    v2 = rng.uniform(-vmax, vmax, shape)
    return conserved(rho, v1, v2, p, gamma)


def smooth_random_state(mesh, N, seed=0, gamma=1.4, amp=0.2, modes=3):
    """Seeded smooth periodic fields (a few Fourier modes) around rho = p = 1."""
    rng = np.random.default_rng(seed)
    X, Y = node_coords(mesh, N)
    x0, y0, x1, y1 = mesh.box
    ux = 2 * np.pi * (X - x0) / (x1 - x0)
    uy = 2 * np.pi * (Y - y0) / (y1 - y0)

    def field():
        f = np.zeros_like(X)
        for _ in range(modes):
            kx, ky = rng.integers(0, 3, 2)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(-1, 1) * np.sin(kx * ux + ky * uy + ph)
        return f / modes

    rho = 1.0 + amp * field()
    p = 1.0 + amp * field()
    v1 = 0.3 * field()
    v2 = 0.3 * field()
    return conserved(rho, v1, v2, p, gamma)


def concat_states(states: Sequence[np.ndarray]) -> np.ndarray:
    """Concatenate per-simulation states [4][K_s][..] along the element axis."""
    return np.ascontiguousarray(np.concatenate(states, axis=1))


# ----------------------------------------------------------------------------
# 3D: conforming Cartesian grids of hexahedra
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Grid3:
    """A conforming nx x ny x nz grid of hexahedra over box (x0, y0, z0, x1,
    y1, z1), boundary kinds per side (-x, +x, -y, +y, -z, +z) and the
    Dirichlet primitive states (rho, v1, v2, v3, p) per side. Elements are
    ordered e = (ez ny + ey) nx + ex."""

    nx: int
    ny: int
    nz: int
    box: tuple = (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
    bc: tuple = (BC_PERIODIC,) * 6
    bc_prim: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((6, 5)))

    @property
    def n_elems(self) -> int:
        return self.nx * self.ny * self.nz


def node_coords3(grid, N: int):
    """x, y, z of every node of a Grid3 or a Mesh3, shape [K][N+1][N+1][N+1]
    indexed [e][k][j][i]."""
    if hasattr(grid, "level"):
        return node_coords_mesh3(grid, N)
    x0, y0, z0, x1, y1, z1 = grid.box
    hx, hy, hz = (x1 - x0) / grid.nx, (y1 - y0) / grid.ny, (z1 - z0) / grid.nz
    ez, ey, ex = np.meshgrid(np.arange(grid.nz), np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    cx = (x0 + (ex.ravel() + 0.5) * hx)[:, None, None, None]
    cy = (y0 + (ey.ravel() + 0.5) * hy)[:, None, None, None]
    cz = (z0 + (ez.ravel() + 0.5) * hz)[:, None, None, None]
    s = lgl_points(N)
    shape = (grid.n_elems, N + 1, N + 1, N + 1)
    X = np.broadcast_to(cx + 0.5 * hx * s[None, None, None, :], shape).copy()
    Y = np.broadcast_to(cy + 0.5 * hy * s[None, None, :, None], shape).copy()
    Z = np.broadcast_to(cz + 0.5 * hz * s[None, :, None, None], shape).copy()
    return X, Y, Z


def conserved3(rho, v1, v2, v3, p, gamma):
    """Ideal-gas conserved state (rho, rho v1, rho v2, rho v3, E) on axis 0."""
    rho = np.asarray(rho, dtype=np.float64)
    E = p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3)
    return np.ascontiguousarray(np.stack([rho, rho * v1, rho * v2, rho * v3, E * np.ones_like(rho)], axis=0))


def density_wave3_state(grid: Grid3, N: int, t=0.0, gamma=1.4, vel=(0.1, 0.2, -0.1)):
    """The density wave of Sec. 3.1 (Eq. entropywave2D) with a third direction:
    rho = 2 + 0.98 sin(2 pi (x + y + z - (v1 + v2 + v3) t) / L), constant
    velocity and p = 20 on a periodic box of side L in each direction (the
    exact solution is the advected initial state)."""
    X, Y, Z = node_coords3(grid, N)
    x0, y0, z0, x1, y1, z1 = grid.box
    L = x1 - x0
    ph = (X - vel[0] * t) + (Y - vel[1] * t) + (Z - vel[2] * t)
    rho = 2.0 + 0.98 * np.sin(2 * np.pi * ph / L)
    one = np.ones_like(X)
    return conserved3(rho, vel[0] * one, vel[1] * one, vel[2] * one, 20.0 * one, gamma)


def random3_state(grid: Grid3, N: int, seed=0, gamma=1.4, rho_range=(0.5, 2.0), p_range=(0.5, 2.0), vmax=0.5):
    """Seeded nodal noise: rho and p log-uniform in their ranges, velocities
    uniform in [-vmax, vmax]."""
    rng = np.random.default_rng(seed)
    shape = (grid.n_elems, N + 1, N + 1, N + 1)
    rho = np.exp(rng.uniform(np.log(rho_range[0]), np.log(rho_range[1]), shape))
    p = np.exp(rng.uniform(np.log(p_range[0]), np.log(p_range[1]), shape))
    v = [rng.uniform(-vmax, vmax, shape) for _ in range(3)]
    return conserved3(rho, v[0], v[1], v[2], p, gamma)


def blast3_state(grid: Grid3, N: int, centre=(0.5, 0.5, 0.5), r0=0.15, gamma=1.4, rho_bg=1e-3, p_bg=1e-3,
                 rho_in=1.0, p_in=10.0):
    """A sphere r < r0 about centre at (rho_in, p_in) in a gas at rest at
    (rho_bg, p_bg): a 3D blast with a near-vacuum background."""
    X, Y, Z = node_coords3(grid, N)
    r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
    inside = r2 < r0 * r0
    rho = np.where(inside, rho_in, rho_bg)
    p = np.where(inside, p_in, p_bg)
    zero = np.zeros_like(X)
    return conserved3(rho, zero, zero, zero, p, gamma)


def slab_from_2d(u2, mesh, N: int, nz: int):
    """A 3D state [5][nx ny nz][N+1]^3 that repeats the 2D state [4][K][N+1]^2
    of a uniform level-0 mesh in z (v3 = 0), on the grid Grid3(mesh.nx0,
    mesh.ny0, nz): the reduction of the 3D scheme to the 2D one. Also returns
    for each 3D element its 2D element."""
    nx, ny = mesh.nx0, mesh.ny0
    src = np.asarray(u2).reshape(4, mesh.n_elems, N + 1, N + 1)
    e2 = np.zeros(nx * ny * nz, dtype=np.int64)
    for e in range(mesh.n_elems):
        for ez in range(nz):
            e2[(ez * ny + int(mesh.iy[e])) * nx + int(mesh.ix[e])] = e
    out = np.zeros((5, nx * ny * nz, N + 1, N + 1, N + 1))
    for k in range(N + 1):
        out[0, :, k] = src[0][e2]
        out[1, :, k] = src[1][e2]
        out[2, :, k] = src[2][e2]
        out[4, :, k] = src[3][e2]
    return out, e2


@dataclasses.dataclass
class Mesh3:
    """Leaves of a 2:1 octree over a box with an nx0 x ny0 x nz0 level-0 grid:
    leaf e at level level[e], index (ix, iy, iz)[e] on its level's grid."""

    nx0: int
    ny0: int
    nz0: int
    box: tuple  # (x0, y0, z0, x1, y1, z1)
    level: np.ndarray  # int8 [K]
    ix: np.ndarray     # int32 [K]
    iy: np.ndarray
    iz: np.ndarray
    bc: tuple = (BC_PERIODIC,) * 6
    bc_prim: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((6, 5)))

    @property
    def n_elems(self) -> int:
        return int(self.level.shape[0])


def box_refined_mesh3(nx0, ny0, nz0, box, rbox, bc=(BC_PERIODIC,) * 6, base_level=0, inside=True):
    """A uniform octree at base_level with the leaves whose centre lies in
    rbox = (x0, y0, z0, x1, y1, z1) (outside it, with inside=False) refined
    once (one level jump: 2:1)."""
    lev, ix, iy, iz = [], [], [], []
    n = 1 << base_level
    x0, y0, z0, x1, y1, z1 = box
    hx, hy, hz = (x1 - x0) / (nx0 * n), (y1 - y0) / (ny0 * n), (z1 - z0) / (nz0 * n)
    for c in range(nz0 * n):
        for b in range(ny0 * n):
            for a in range(nx0 * n):
                cx, cy, cz = x0 + (a + 0.5) * hx, y0 + (b + 0.5) * hy, z0 + (c + 0.5) * hz
                hit = rbox[0] < cx < rbox[3] and rbox[1] < cy < rbox[4] and rbox[2] < cz < rbox[5]
                if hit == inside:
                    for q in range(8):
                        lev.append(base_level + 1)
                        ix.append(2 * a + (q & 1)); iy.append(2 * b + ((q >> 1) & 1)); iz.append(2 * c + (q >> 2))
                else:
                    lev.append(base_level); ix.append(a); iy.append(b); iz.append(c)
    return Mesh3(nx0, ny0, nz0, box, np.array(lev, np.int8), np.array(ix, np.int32), np.array(iy, np.int32),
                 np.array(iz, np.int32), bc=bc)


def extruded_mesh3(mesh2: Mesh, z0=0.0, z1=1.0, bcz=(BC_PERIODIC, BC_PERIODIC)):
    """The octree that extrudes a quadtree mesh in z over one level-0 cell:
    2D leaf (l, ix, iy) becomes the 2^l leaves (l, ix, iy, iz); with states
    that do not depend on z the 3D scheme reduces to the 2D one on it. Also
    returns, per 3D leaf, its 2D leaf."""
    lev, ix, iy, iz, e2 = [], [], [], [], []
    for e in range(mesh2.n_elems):
        l = int(mesh2.level[e])
        for c in range(1 << l):
            lev.append(l); ix.append(int(mesh2.ix[e])); iy.append(int(mesh2.iy[e])); iz.append(c); e2.append(e)
    x0, y0, x1, y1 = mesh2.box
    m3 = Mesh3(mesh2.nx0, mesh2.ny0, 1, (x0, y0, z0, x1, y1, z1), np.array(lev, np.int8), np.array(ix, np.int32),
               np.array(iy, np.int32), np.array(iz, np.int32), bc=tuple(mesh2.bc) + tuple(bcz))
    return m3, np.array(e2, np.int64)


def node_coords_mesh3(mesh: Mesh3, N: int):
    """x, y, z of every node of an octree, [K][N+1][N+1][N+1] indexed [e][k][j][i]."""
    x0, y0, z0, x1, y1, z1 = mesh.box
    lv = mesh.level.astype(np.int64)
    hx = (x1 - x0) / (mesh.nx0 * (1 << lv))
    hy = (y1 - y0) / (mesh.ny0 * (1 << lv))
    hz = (z1 - z0) / (mesh.nz0 * (1 << lv))
    s = lgl_points(N)
    cx = (x0 + (mesh.ix + 0.5) * hx)[:, None, None, None]
    cy = (y0 + (mesh.iy + 0.5) * hy)[:, None, None, None]
    cz = (z0 + (mesh.iz + 0.5) * hz)[:, None, None, None]
    shape = (mesh.n_elems, N + 1, N + 1, N + 1)
    X = np.broadcast_to(cx + 0.5 * hx[:, None, None, None] * s[None, None, None, :], shape).copy()
    Y = np.broadcast_to(cy + 0.5 * hy[:, None, None, None] * s[None, None, :, None], shape).copy()
    Z = np.broadcast_to(cz + 0.5 * hz[:, None, None, None] * s[None, :, None, None], shape).copy()
    return X, Y, Z


def extrude_state(u2, e2, N: int):
    """The 3D state on extruded_mesh3 that repeats the 2D state in z (v3 = 0)."""
    src = np.asarray(u2).reshape(4, -1, N + 1, N + 1)
    out = np.zeros((5, len(e2), N + 1, N + 1, N + 1))
    for k in range(N + 1):
        out[0, :, k] = src[0][e2]
        out[1, :, k] = src[1][e2]
        out[2, :, k] = src[2][e2]
        out[4, :, k] = src[3][e2]
    return out


def random_octree3(nx0, ny0, nz0, box=(0.0, 0.0, 0.0, 1.0, 1.0, 1.0), seed=0, n_refine=6, max_level=2,
                   bc=(BC_PERIODIC,) * 6):
    """A seeded 2:1-balanced octree: n_refine times a random leaf below
    max_level is refined, then leaves are refined until face neighbours
    (across periodic sides too) differ by at most one level. Kept as a level
    map over the finest cells, as the 2D meshes."""
    rng = np.random.default_rng(seed)
    L = max_level
    lmap = np.zeros((nx0 << L, ny0 << L, nz0 << L), dtype=np.int16)
    per = [bc[2 * d] == BC_PERIODIC for d in range(3)]

    def leaves():
        f = np.indices(lmap.shape).reshape(3, -1)
        lv = lmap.reshape(-1).astype(np.int64)
        sh = L - lv
        anchor = np.all((f & ((1 << sh) - 1)) == 0, axis=0)
        return lv[anchor], f[:, anchor] >> sh[anchor]

    def refine(l, c):
        s = L - l
        x, y, z = (int(v) << s for v in c)
        lmap[x:x + (1 << s), y:y + (1 << s), z:z + (1 << s)] += 1

    for _ in range(n_refine):
        lv, c = leaves()
        cand = np.flatnonzero(lv < max_level)
        if cand.size == 0:
            break
        k = int(rng.choice(cand))
        refine(int(lv[k]), c[:, k])
    while True:
        nbm = np.full(lmap.shape, -1, dtype=np.int32)
        a = lmap.astype(np.int32)
        for d in range(3):
            for sh in (1, -1):
                if per[d]:
                    nb = np.roll(a, sh, axis=d)
                else:
                    nb = np.full_like(a, -1)
                    src = [slice(None)] * 3
                    dst = [slice(None)] * 3
                    if sh == 1:
                        dst[d], src[d] = slice(1, None), slice(None, -1)
                    else:
                        dst[d], src[d] = slice(None, -1), slice(1, None)
                    nb[tuple(dst)] = a[tuple(src)]
                nbm = np.maximum(nbm, nb)
        need = nbm >= a + 2
        if not need.any():
            break
        lv, c = leaves()
        for k in range(lv.size):
            s = L - int(lv[k])
            x, y, z = (int(v) << s for v in c[:, k])
            if need[x:x + (1 << s), y:y + (1 << s), z:z + (1 << s)].any():
                refine(int(lv[k]), c[:, k])
    lv, c = leaves()
    return Mesh3(nx0, ny0, nz0, tuple(float(b) for b in box), lv.astype(np.int8), c[0].astype(np.int32),
                 c[1].astype(np.int32), c[2].astype(np.int32), bc=tuple(bc))
