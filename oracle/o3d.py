"""The 3D oracle (``idp_oracle3d.c``): IDP-limited LGL-DGSEM for the 3D Euler
equations on a conforming Cartesian grid of hexahedra.

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it. It shares no code with the
CUDA path. The library is built from ``idp_oracle3d.c`` together with
``idp_oracle.c`` (the LGL operators and the logarithmic mean).

State layout u[5][K][N+1][N+1][N+1] (rho, rho v1, rho v2, rho v3, rho e; x
index fastest), elements e = (ez ny + ey) nx + ex.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "idp_oracle3d.c")
_SRC2 = os.path.join(_HERE, "idp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle3d.so")
_lib = None

BC_PERIODIC, BC_WALL, BC_DIRICHLET, BC_OUTFLOW = 0, 1, 2, 3
ST_NAMES = ["alpha_vol_m", "mass", "n_vol_active", "viol_rho", "viol_p", "nonpositive", "dt_exceed",
            "min_rho", "min_p", "alpha_mort_a", "mort_area", "n_mort_active"]
_FLAGS = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                                                          os.path.getmtime(_SRC2)):
        subprocess.check_call(_FLAGS + ["-o", _LIB, _SRC, _SRC2, "-lm"])
    return _LIB


def compile_source(src: str, out: str) -> str:
    """Compile 3D oracle source text (with the unchanged idp_oracle.c) to the
    library ``out``: the tests that plant a mistake in a copy use it."""
    c_path = out[:-3] + ".c" if out.endswith(".so") else out + ".c"
    with open(c_path, "w") as f:
        f.write(src)
    subprocess.check_call(_FLAGS + ["-o", out, c_path, _SRC2, "-lm"])
    return out


def load(path: str):
    L = C.CDLL(path)
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
    L.o3_create.restype = C.c_void_p
    L.o3_create.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, dp, ip, dp, C.POINTER(C.c_int)]
    L.o3_create_leaves.restype = C.c_void_p
    L.o3_create_leaves.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, dp, C.c_int, C.POINTER(C.c_int8),
                                   ip, ip, ip, ip, dp, C.POINTER(C.c_int)]
    L.o3_n_mortars.restype = C.c_int
    L.o3_n_mortars.argtypes = [C.c_void_p]
    L.o3_set_mortar_out.argtypes = [dp, dp]
    L.o3_indicator.restype = C.c_double
    L.o3_indicator.argtypes = [C.c_int, dp, dp]
    L.o3_set_force_alpha.argtypes = [C.c_double]
    L.o3_mortar_table.argtypes = [C.c_void_p, ip]
    L.o3_destroy.argtypes = [C.c_void_p]
    L.o3_n_nodes.restype = C.c_int
    L.o3_n_nodes.argtypes = [C.c_void_p]
    L.o3_stage.argtypes = [C.c_void_p, dp, C.c_double, C.c_int, C.c_double, dp, dp, dp]
    L.o3_rhs.argtypes = [C.c_void_p, dp, C.c_double, C.c_int, C.c_double, dp, dp]
    L.o3_step.argtypes = [C.c_void_p, dp, C.c_int, dp, C.c_double, C.c_int, C.c_double, dp, dp]
    L.o3_dt.restype = C.c_double
    L.o3_dt.argtypes = [C.c_void_p, dp, C.c_double]
    L.o3_integrals.argtypes = [C.c_void_p, dp, dp]
    L.o3_masses.argtypes = [C.c_void_p, dp]
    L.o3_dg_residual.argtypes = [C.c_void_p, dp, dp]
    L.o3_fv_residual.argtypes = [C.c_void_p, dp, dp, dp]
    L.o3_stats_init.argtypes = [dp]
    L.o3_set_force_ell.argtypes = [C.c_double]
    L.o3_set_dbg_out.argtypes = [dp, dp]
    L.o3_ranocha.argtypes = [C.c_double, dp, dp, C.c_int, dp]
    L.o3_llf.argtypes = [C.c_double, dp, dp, C.c_int, dp]
    L.o3_theta.restype = C.c_double
    L.o3_theta.argtypes = [C.c_double, dp, dp, C.c_double, C.c_double]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


class using:
    """Route this module's calls through another build of the 3D oracle."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _lib
        _lib = load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Oracle3D:
    """The 3D oracle on a uniform grid (attributes nx, ny, nz, box, bc,
    bc_prim, n_elems: workloads.Grid3) or on a 2:1 octree (attributes nx0,
    ny0, nz0, box, level, ix, iy, iz, bc, bc_prim: workloads.Mesh3)."""

    def __init__(self, grid, N: int, gamma: float = 1.4):
        self.grid, self.N, self.np, self.gamma = grid, N, N + 1, gamma
        self._L = lib()
        err = C.c_int()
        box = np.ascontiguousarray(grid.box, dtype=np.float64)
        bc = np.ascontiguousarray(grid.bc, dtype=np.int32)
        bcp = np.ascontiguousarray(grid.bc_prim, dtype=np.float64).reshape(30)
        ip = C.POINTER(C.c_int32)
        if hasattr(grid, "level"):
            lev = np.ascontiguousarray(grid.level, dtype=np.int8)
            ix, iy, iz = (np.ascontiguousarray(a, dtype=np.int32) for a in (grid.ix, grid.iy, grid.iz))
            self._keep = (lev, ix, iy, iz)
            self._h = self._L.o3_create_leaves(N, gamma, grid.nx0, grid.ny0, grid.nz0, _d(box), int(lev.size),
                                               lev.ctypes.data_as(C.POINTER(C.c_int8)), ix.ctypes.data_as(ip),
                                               iy.ctypes.data_as(ip), iz.ctypes.data_as(ip), bc.ctypes.data_as(ip),
                                               _d(bcp), C.byref(err))
        else:
            self._h = self._L.o3_create(N, gamma, grid.nx, grid.ny, grid.nz, _d(box), bc.ctypes.data_as(ip), _d(bcp),
                                        C.byref(err))
        if not self._h:
            raise ValueError(f"o3_create failed ({err.value})")
        self.nn = self._L.o3_n_nodes(self._h)
        self.M = self._L.o3_n_mortars(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.o3_destroy(self._h)
            self._h = None

    def _u(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == 5 * self.nn, (u.shape, self.nn)
        return u

    def shape(self):
        return (5, self.grid.n_elems, self.np, self.np, self.np)

    def rhs(self, u, dt=0.0, limiting=2, beta=0.1, stats=None):
        """Residual per unit mass; dt = 0 gives the unlimited DG right-hand side."""
        u = self._u(u)
        out = np.zeros_like(u)
        st = np.zeros(16) if stats is None else stats
        if stats is None:
            self._L.o3_stats_init(_d(st))
        self._L.o3_rhs(self._h, _d(u), dt, limiting, beta, _d(out), _d(st))
        return out

    def stage(self, u, dt, limiting=2, beta=0.1, stats=None):
        """(mass-weighted limited residual, limited stage state)."""
        u = self._u(u)
        res, ut = np.zeros_like(u), np.zeros_like(u)
        st = np.zeros(16) if stats is None else stats
        if stats is None:
            self._L.o3_stats_init(_d(st))
        self._L.o3_stage(self._h, _d(u), dt, limiting, beta, _d(res), _d(ut), _d(st))
        return res, ut

    def stage_debug(self, u, dt, limiting=2, beta=0.1, force_ell=None):
        """One limited stage with the limiter's intermediate values (test
        use): dict with res, ut, stats, node [nn][10] (u_FV (5), rho_min,
        rho_max, p_min, R+, R-) and iface [nif][12] (left node, right node,
        exempt, Zalesak factor, theta_left, theta_right, factor, A (5))."""
        nif = self.grid.n_elems * 3 * self.np * self.np * self.N
        node, iface, mell = np.zeros((self.nn, 10)), np.zeros((nif, 12)), np.zeros(max(self.M, 1))
        mrec = np.zeros((max(self.M, 1), 5 * self.np * self.np, 20))
        st = np.zeros(16)
        self._L.o3_stats_init(_d(st))
        self._L.o3_set_dbg_out(_d(node), _d(iface))
        self._L.o3_set_mortar_out(_d(mell), _d(mrec))
        if force_ell is not None:
            self._L.o3_set_force_ell(float(force_ell))
        try:
            res, ut = self.stage(u, dt, limiting=limiting, beta=beta, stats=st)
        finally:
            self._L.o3_set_dbg_out(None, None)
            self._L.o3_set_mortar_out(None, None)
            self._L.o3_set_force_ell(-1.0)
        return {"res": res, "ut": ut, "stats": {k: float(st[i]) for i, k in enumerate(ST_NAMES)},
                "node": node, "iface": iface, "mortar_ell": mell[:self.M], "mortar": mrec[:self.M]}

    def mortars(self):
        """[M][7]: d, large element, large on the low side, small elements p = p1 + 2 p2."""
        t = np.zeros((max(self.M, 1), 7), np.int32)
        self._L.o3_mortar_table(self._h, t.ctypes.data_as(C.POINTER(C.c_int32)))
        return t[:self.M]

    def dt(self, u, cfl=0.5):
        return self._L.o3_dt(self._h, _d(self._u(u)), cfl)

    def step(self, u, nsteps, t=0.0, cfl=0.5, limiting=2, beta=0.1):
        """Returns (u_new, t_new, dt_history, stats dict)."""
        u = self._u(u).copy()
        tt = np.array([t])
        dts = np.zeros(max(nsteps, 1))
        st = np.zeros(16)
        self._L.o3_stats_init(_d(st))
        self._L.o3_step(self._h, _d(u), nsteps, _d(tt), cfl, limiting, beta, _d(dts), _d(st))
        return u, float(tt[0]), dts[:nsteps], {k: float(st[i]) for i, k in enumerate(ST_NAMES)}

    def masses(self):
        m = np.zeros(self.nn)
        self._L.o3_masses(self._h, _d(m))
        return m

    def integrals(self, u):
        out = np.zeros(5)
        self._L.o3_integrals(self._h, _d(self._u(u)), _d(out))
        return out

    def dg_residual(self, u):
        u = self._u(u)
        out = np.zeros_like(u)
        self._L.o3_dg_residual(self._h, _d(u), _d(out))
        return out

    def fv_residual(self, u):
        u = self._u(u)
        out, ds = np.zeros_like(u), np.zeros(self.nn)
        self._L.o3_fv_residual(self._h, _d(u), _d(out), _d(ds))
        return out, ds


def set_force_ell(v: float):
    """Every limiting factor replaced by v (v < 0: off); test hook."""
    lib().o3_set_force_ell(float(v))


def ranocha(gamma, uL, uR, d):
    f = np.zeros(5)
    lib().o3_ranocha(gamma, _d(np.ascontiguousarray(uL, dtype=np.float64)),
                     _d(np.ascontiguousarray(uR, dtype=np.float64)), d, _d(f))
    return f


def llf(gamma, uL, uR, d):
    f = np.zeros(5)
    lib().o3_llf(gamma, _d(np.ascontiguousarray(uL, dtype=np.float64)),
                 _d(np.ascontiguousarray(uR, dtype=np.float64)), d, _d(f))
    return f


def indicator3(N, p):
    """The 3D shock indicator alpha in [0, 1] of one element from its nodal
    pressures p[k][j][i] (the combined limiting's, reading R34)."""
    xi = np.asarray(oracle_lgl_nodes(N), dtype=np.float64)
    pp = np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
    return float(lib().o3_indicator(N, _d(xi), _d(pp)))


def oracle_lgl_nodes(N):
    """The LGL nodes of the 2D oracle's operators (shared by the 3D one)."""
    import oracle as _o
    return _o.lgl(N)[0]


def set_force_alpha(v):
    """Every element's shock indicator replaced by v (v < 0: off); test hook."""
    lib().o3_set_force_alpha(float(v))
