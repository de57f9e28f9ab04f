"""Plain FP64 CPU oracle of the IDP-limited LGL-DGSEM (test infrastructure).

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the CUDA path in ``paper_2607_06045_b300``.

The arithmetic lives in ``idp_oracle.c`` (plain C, compiled with
``-O2 -ffp-contract=off``); this module only marshals arrays through ctypes.
Parity status per function: every function is pinned by ``tests/test_oracle_*``
against the paper's printed values, closed forms or brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "idp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ST_NAMES = ["alpha_vol_m", "mass", "n_vol_active", "alpha_mort_len", "len", "n_mort_active",
            "viol_rho", "viol_p", "nonpositive", "dt_exceed", "min_rho", "min_p", "viol_eta"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no vectorising float contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
               "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build_omp(force: bool = False) -> str:
    """The same source with OpenMP over the loops whose iterations write
    disjoint outputs (the all-cores CPU baseline; same bits as the serial
    build)."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", _LIB_OMP, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB_OMP


def lib():
    """The loaded oracle library (built on first use)."""
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def compile_source(src: str, out: str) -> str:
    """Compile oracle C source text to the shared library ``out`` with the
    oracle's own flags (used by the tests that plant a mistake in a copy of
    the oracle to check that a pin catches it)."""
    c_path = out[:-3] + ".c" if out.endswith(".so") else out + ".c"
    with open(c_path, "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
                           "-shared", "-o", out, c_path, "-lm"])
    return out


class using:
    """Context manager: route every call of this module through the oracle
    library at ``path`` (another build of the oracle source), restoring the
    default library on exit. Oracle objects must be created inside it."""

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


def load(path: str):
    """Load an oracle library and declare its entry points."""
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                             C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int8), ip, ip, ip,
                             dp, dp, dp, C.c_int, C.POINTER(C.c_int)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_lgl.argtypes = [C.c_int, dp, dp]
    L.orc_operators.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp, dp, dp]
    L.orc_logmean.restype = C.c_double
    L.orc_logmean.argtypes = [C.c_double, C.c_double]
    L.orc_ranocha.argtypes = [C.c_double, dp, dp, C.c_int, dp]
    L.orc_llf.argtypes = [C.c_double, dp, dp, C.c_double, C.c_double, dp]
    L.orc_theta.restype = C.c_double
    L.orc_theta.argtypes = [C.c_double, dp, dp, C.c_double, C.c_double]
    L.orc_indicator.restype = C.c_double
    L.orc_indicator.argtypes = [C.c_int, dp, dp]
    L.orc_n_mortars.restype = C.c_int
    L.orc_n_mortars.argtypes = [C.c_void_p]
    L.orc_mortars.argtypes = [C.c_void_p, ip]
    L.orc_faces.argtypes = [C.c_void_p, ip, ip]
    L.orc_graph_size.restype = C.c_int
    L.orc_graph_size.argtypes = [C.c_void_p]
    L.orc_graph.argtypes = [C.c_void_p, ip, ip, dp, dp]
    L.orc_stage.argtypes = [C.c_void_p, dp, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int,
                            dp, dp, dp]
    L.orc_rhs.argtypes = [C.c_void_p, dp, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int, dp, dp]
    L.orc_step.argtypes = [C.c_void_p, dp, C.c_int, dp, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int,
                           C.c_int, dp, dp]
    L.orc_set_volume_flux.argtypes = [C.c_void_p, C.c_int]
    L.orc_mortar_weights.argtypes = [C.c_void_p, dp]
    L.orc_chandrashekar.argtypes = [C.c_double, dp, dp, C.c_int, dp]
    L.orc_theta_entropy.restype = C.c_double
    L.orc_theta_entropy.argtypes = [C.c_double, dp, dp, C.c_double, C.c_double]
    L.orc_entropy_eta.restype = C.c_double
    L.orc_entropy_eta.argtypes = [C.c_double, dp]
    L.orc_dt.restype = C.c_double
    L.orc_dt.argtypes = [C.c_void_p, dp, C.c_double, C.c_double, C.c_int]
    L.orc_integrals.argtypes = [C.c_void_p, dp, dp]
    L.orc_dg_residual.argtypes = [C.c_void_p, dp, C.c_double, dp]
    L.orc_dg_residual_fd.argtypes = [C.c_void_p, dp, C.c_double, dp]
    L.orc_fv_residual.argtypes = [C.c_void_p, dp, C.c_double, dp, dp]
    L.orc_masses.argtypes = [C.c_void_p, dp]
    L.orc_stats_init.argtypes = [dp]
    L.orc_mortar_sparse.argtypes = [C.c_int, C.c_double, dp, dp, dp]
    L.orc_set_mortar_ell_out.argtypes = [dp]
    L.orc_set_mortar_dbg_out.argtypes = [dp]
    L.orc_set_node_dbg_out.argtypes = [dp]
    L.orc_set_iface_dbg_out.argtypes = [dp]
    L.orc_set_force_ell.argtypes = [C.c_double]
    L.orc_face_sparse.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, dp, dp]
    L.orc_set_threads.restype = C.c_int
    L.orc_set_threads.argtypes = [C.c_int]
    return L


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def lgl(N: int):
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    lib().orc_lgl(N, _d(x), _d(w))
    return x, w


def operators(N: int, proj: int = 0):
    """(xi, w, D, Sbar, local weights [np][2np], interpolation [2np][np], projection [np][2np])."""
    np_ = N + 1
    xi, w = np.zeros(np_), np.zeros(np_)
    D, S = np.zeros((np_, np_)), np.zeros((np_, np_))
    wt, I, P = np.zeros((np_, 2 * np_)), np.zeros((2 * np_, np_)), np.zeros((np_, 2 * np_))
    lib().orc_operators(N, proj, _d(xi), _d(w), _d(D), _d(S), _d(wt), _d(I), _d(P))
    return xi, w, D, S, wt, I, P


def logmean(a: float, b: float) -> float:
    return lib().orc_logmean(a, b)


def ranocha(uL, uR, d: int, gamma=1.4):
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    f = np.zeros(4)
    lib().orc_ranocha(gamma, _d(uL), _d(uR), d, _d(f))
    return f


def chandrashekar(uL, uR, d: int, gamma=1.4):
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    f = np.zeros(4)
    lib().orc_chandrashekar(gamma, _d(uL), _d(uR), d, _d(f))
    return f


def llf(uL, uR, n, gamma=1.4):
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    f = np.zeros(4)
    lib().orc_llf(gamma, _d(uL), _d(uR), float(n[0]), float(n[1]), _d(f))
    return f


def theta(u0, a, pmin, hi, gamma=1.4):
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_theta(gamma, _d(u0), _d(a), float(pmin), float(hi))


def theta_entropy(u0, a, K, hi, gamma=1.4):
    """Largest factor in [0, hi] keeping eta(u0 + theta a) >= K (R21)."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_theta_entropy(gamma, _d(u0), _d(a), float(K), float(hi))


def entropy_eta(u, gamma=1.4):
    """Modified specific entropy p rho^-gamma / (gamma - 1) of one state."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_entropy_eta(gamma, _d(u))



def indicator(N, p):
    """Shock indicator alpha in [0, 1] of one element from its nodal pressures
    p[j][i] (y index j, x index i) at the LGL nodes of degree N (reading R20:
    Hennemann et al.'s modal energy indicator, used by the combined limiting
    of Sec. 3.5)."""
    xi, _ = lgl(N)
    pp = np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
    return float(lib().orc_indicator(N, xi.ctypes.data_as(C.POINTER(C.c_double)), pp.ctypes.data_as(C.POINTER(C.c_double))))

def face_sparse(N, ratio, uA, us, gamma=1.4):
    """Low-order fluxes of one interface through the stage's weights and pair
    terms: single face uA[np][4] against ratio faces us[ratio np][4] (ratio 1
    conforming, 2 a 2:1 mortar). Returns (outward fluxes [(1 + ratio) np][4],
    weights [np][ratio np] in reference units)."""
    uA = np.ascontiguousarray(uA, dtype=np.float64)
    us = np.ascontiguousarray(us, dtype=np.float64)
    np_ = N + 1
    F = np.zeros(4 * (1 + ratio) * np_)
    wt = np.zeros(np_ * ratio * np_)
    lib().orc_face_sparse(N, ratio, gamma, _d(uA), _d(us), _d(F), _d(wt))
    return F.reshape((1 + ratio) * np_, 4), wt.reshape(np_, ratio * np_)


def mortar_sparse(N, uL, us, gamma=1.4):
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    us = np.ascontiguousarray(us, dtype=np.float64)
    out = np.zeros(12 * 9)
    lib().orc_mortar_sparse(N, gamma, _d(uL), _d(us), _d(out))
    return out[: 4 * 3 * (N + 1)].reshape(3 * (N + 1), 4)


class Oracle:
    """Oracle context for one mesh, degree N and gamma.

    proj selects the L2 mortar projection (R5): 1 (default) the exact L2
    projection, 0 the LGL-weighted adjoint of interpolation. volume_flux: 0
    Ranocha (R1), 1 Chandrashekar (R23). mortar_low: 0 the sparse local
    weights (Eq. local_weights), 1 the all-to-all weights (Eq. nonlocal_weight,
    R25) in the low-order mortar flux."""

    def __init__(self, mesh, N: int, gamma: float = 1.4, proj: int = 1, volume_flux: int = 0, mortar_low: int = 0):
        self.N, self.np, self.gamma = N, N + 1, gamma
        self.K = mesh.n_elems
        self._keep = [np.ascontiguousarray(mesh.level, dtype=np.int8),
                      np.ascontiguousarray(mesh.ix, dtype=np.int32),
                      np.ascontiguousarray(mesh.iy, dtype=np.int32),
                      np.ascontiguousarray(mesh.bc, dtype=np.int32),
                      np.ascontiguousarray(mesh.bc_prim, dtype=np.float64).reshape(16),
                      np.ascontiguousarray(mesh.dmr_post, dtype=np.float64),
                      np.ascontiguousarray(mesh.dmr_pre, dtype=np.float64)]
        lev, ix, iy, bc, bcp, post, pre = self._keep
        self._L = lib()
        err = C.c_int(0)
        x0, y0, x1, y1 = mesh.box
        self._h = self._L.orc_create(N, gamma, proj, mesh.nx0, mesh.ny0, x0, y0, x1, y1, self.K,
                                   lev.ctypes.data_as(C.POINTER(C.c_int8)), _i(ix), _i(iy), _i(bc),
                                   _d(bcp), _d(post), _d(pre), int(mortar_low), C.byref(err))
        if not self._h:
            raise ValueError(f"oracle mesh rejected (code {err.value})")
        # volume flux: 0 Ranocha (R1), 1 Chandrashekar (R23)
        self._L.orc_set_volume_flux(self._h, int(volume_flux))

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    def _u(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (4, self.K, self.np, self.np), u.shape
        return u

    @property
    def n_mortars(self) -> int:
        return self._L.orc_n_mortars(self._h)

    def mortars(self):
        out = np.zeros((self.n_mortars, 5), dtype=np.int32)
        if self.n_mortars:
            self._L.orc_mortars(self._h, _i(out))
        return out

    def mortar_weights(self):
        """Weights of the low-order mortar flux [np][2 np] (reference units)."""
        out = np.zeros((self.np, 2 * self.np))
        self._L.orc_mortar_weights(self._h, _d(out))
        return out

    def faces(self):
        ft = np.zeros((self.K, 4), dtype=np.int32)
        fn = np.zeros((self.K, 4), dtype=np.int32)
        self._L.orc_faces(self._h, _i(ft), _i(fn))
        return ft, fn

    def graph(self):
        n = self._L.orc_graph_size(self._h)
        nn = self.K * self.np * self.np
        off = np.zeros(nn + 1, dtype=np.int32)
        j = np.zeros(n, dtype=np.int32)
        cx, cy = np.zeros(n), np.zeros(n)
        self._L.orc_graph(self._h, _i(off), _i(j), _d(cx), _d(cy))
        return off, j, cx, cy

    def masses(self):
        m = np.zeros((self.K, self.np, self.np))
        self._L.orc_masses(self._h, _d(m))
        return m

    def rhs(self, u, t=0.0, dt=0.0, limiting=2, beta=0.1, stats=None, bounds=0, entropy=0):
        """Limited residual per unit mass; dt = 0 gives the unlimited DG RHS.
        bounds: 0 bar states, 1 low-order solution; entropy: 1 adds the
        entropy bound to local limiting."""
        u = self._u(u)
        out = np.zeros_like(u)
        st = np.zeros(16) if stats is None else stats
        if stats is None:
            self._L.orc_stats_init(_d(st))
        self._L.orc_rhs(self._h, _d(u), t, dt, limiting, beta, bounds, entropy, _d(out), _d(st))
        return out

    def stage(self, u, t, dt, limiting=2, beta=0.1, stats=None, bounds=0, entropy=0):
        """(mass-weighted limited residual, limited stage state)."""
        u = self._u(u)
        res, ut = np.zeros_like(u), np.zeros_like(u)
        st = np.zeros(16) if stats is None else stats
        if stats is None:
            self._L.orc_stats_init(_d(st))
        self._L.orc_stage(self._h, _d(u), t, dt, limiting, beta, bounds, entropy, _d(res), _d(ut), _d(st))
        return res, ut

    def stage_debug(self, u, t, dt, limiting=2, beta=0.1, bounds=0, entropy=0, force_ell=None):
        """One limited stage with the limiter's intermediate values recorded
        (test use). force_ell in [0, 1] replaces every volume and mortar
        factor. Returns a dict: res (mass-weighted residual), ut (stage
        state), stats, node [nn][8] (rho_FV, rho_min, rho_max, p_min, rho_vol,
        min factor, R+, R-), iface [nif][8] (left node, right node, A_rho,
        exempt, Zalesak factor, theta_left, theta_right, factor; node left
        receives -A, node right +A), mortar [M][3np][16] (node, density cap,
        factor, u_vol[4], scaled correction a[4], rho_min, rho_max, p_min,
        n_i, H_rho) and mortar_ell [M]."""
        u = self._u(u)
        K, np_, N = self.K, self.np, self.N
        nn = K * np_ * np_
        M = self.n_mortars
        node = np.zeros((nn, 8))
        iface = np.zeros((K * 2 * np_ * N, 8))
        mort = np.zeros((max(M, 1), 3 * np_, 16))
        mell = np.zeros(max(M, 1))
        res, ut = np.zeros_like(u), np.zeros_like(u)
        st = np.zeros(16)
        L = self._L
        L.orc_stats_init(_d(st))
        L.orc_set_node_dbg_out(_d(node))
        L.orc_set_iface_dbg_out(_d(iface))
        L.orc_set_mortar_dbg_out(_d(mort))
        L.orc_set_mortar_ell_out(_d(mell))
        L.orc_set_force_ell(-1.0 if force_ell is None else float(force_ell))
        try:
            L.orc_stage(self._h, _d(u), t, dt, limiting, beta, bounds, entropy, _d(res), _d(ut), _d(st))
        finally:
            null = C.POINTER(C.c_double)()
            L.orc_set_node_dbg_out(null)
            L.orc_set_iface_dbg_out(null)
            L.orc_set_mortar_dbg_out(null)
            L.orc_set_mortar_ell_out(null)
            L.orc_set_force_ell(-1.0)
        return dict(res=res, ut=ut, stats=stats_dict(st), node=node, iface=iface, mortar=mort[:M], mortar_ell=mell[:M])

    def dg_residual(self, u, t=0.0, form="evolution"):
        u = self._u(u)
        out = np.zeros_like(u)
        if form == "evolution":
            self._L.orc_dg_residual(self._h, _d(u), t, _d(out))
        else:
            self._L.orc_dg_residual_fd(self._h, _d(u), t, _d(out))
        return out

    def fv_residual(self, u, t=0.0):
        u = self._u(u)
        out = np.zeros_like(u)
        ds = np.zeros((self.K, self.np, self.np))
        self._L.orc_fv_residual(self._h, _d(u), t, _d(out), _d(ds))
        return out, ds

    def dt(self, u, t=0.0, cfl=0.5, rule=0):
        return self._L.orc_dt(self._h, _d(self._u(u)), t, cfl, rule)

    def step(self, u, nsteps, t=0.0, cfl=0.5, dt_rule=0, limiting=2, beta=0.1, bounds=0, entropy=0):
        """Returns (u_new, t_new, dt_history, stats dict)."""
        u = self._u(u).copy()
        tt = np.array([t])
        dts = np.zeros(max(nsteps, 1))
        st = np.zeros(16)
        self._L.orc_stats_init(_d(st))
        self._L.orc_step(self._h, _d(u), nsteps, _d(tt), cfl, dt_rule, limiting, beta, bounds, entropy, _d(dts),
                       _d(st))
        return u, float(tt[0]), dts[:nsteps], dict(zip(ST_NAMES, st[:13].tolist()))

    def integrals(self, u):
        out = np.zeros(4)
        self._L.orc_integrals(self._h, _d(self._u(u)), _d(out))
        return out


def stats_dict(st):
    return dict(zip(ST_NAMES, np.asarray(st)[:13].tolist()))
