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


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
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
        _lib = L
    return _lib


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
        err = C.c_int(0)
        x0, y0, x1, y1 = mesh.box
        self._h = lib().orc_create(N, gamma, proj, mesh.nx0, mesh.ny0, x0, y0, x1, y1, self.K,
                                   lev.ctypes.data_as(C.POINTER(C.c_int8)), _i(ix), _i(iy), _i(bc),
                                   _d(bcp), _d(post), _d(pre), int(mortar_low), C.byref(err))
        if not self._h:
            raise ValueError(f"oracle mesh rejected (code {err.value})")
        # volume flux: 0 Ranocha (R1), 1 Chandrashekar (R23)
        lib().orc_set_volume_flux(self._h, int(volume_flux))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def _u(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (4, self.K, self.np, self.np), u.shape
        return u

    @property
    def n_mortars(self) -> int:
        return lib().orc_n_mortars(self._h)

    def mortars(self):
        out = np.zeros((self.n_mortars, 5), dtype=np.int32)
        if self.n_mortars:
            lib().orc_mortars(self._h, _i(out))
        return out

    def mortar_weights(self):
        """Weights of the low-order mortar flux [np][2 np] (reference units)."""
        out = np.zeros((self.np, 2 * self.np))
        lib().orc_mortar_weights(self._h, _d(out))
        return out

    def faces(self):
        ft = np.zeros((self.K, 4), dtype=np.int32)
        fn = np.zeros((self.K, 4), dtype=np.int32)
        lib().orc_faces(self._h, _i(ft), _i(fn))
        return ft, fn

    def graph(self):
        n = lib().orc_graph_size(self._h)
        nn = self.K * self.np * self.np
        off = np.zeros(nn + 1, dtype=np.int32)
        j = np.zeros(n, dtype=np.int32)
        cx, cy = np.zeros(n), np.zeros(n)
        lib().orc_graph(self._h, _i(off), _i(j), _d(cx), _d(cy))
        return off, j, cx, cy

    def masses(self):
        m = np.zeros((self.K, self.np, self.np))
        lib().orc_masses(self._h, _d(m))
        return m

    def rhs(self, u, t=0.0, dt=0.0, limiting=2, beta=0.1, stats=None, bounds=0, entropy=0):
        """Limited residual per unit mass; dt = 0 gives the unlimited DG RHS.
        bounds: 0 bar states, 1 low-order solution; entropy: 1 adds the
        entropy bound to local limiting."""
        u = self._u(u)
        out = np.zeros_like(u)
        st = np.zeros(16) if stats is None else stats
        if stats is None:
            lib().orc_stats_init(_d(st))
        lib().orc_rhs(self._h, _d(u), t, dt, limiting, beta, bounds, entropy, _d(out), _d(st))
        return out

    def stage(self, u, t, dt, limiting=2, beta=0.1, stats=None, bounds=0, entropy=0):
        """(mass-weighted limited residual, limited stage state)."""
        u = self._u(u)
        res, ut = np.zeros_like(u), np.zeros_like(u)
        st = np.zeros(16) if stats is None else stats
        if stats is None:
            lib().orc_stats_init(_d(st))
        lib().orc_stage(self._h, _d(u), t, dt, limiting, beta, bounds, entropy, _d(res), _d(ut), _d(st))
        return res, ut

    def dg_residual(self, u, t=0.0, form="evolution"):
        u = self._u(u)
        out = np.zeros_like(u)
        if form == "evolution":
            lib().orc_dg_residual(self._h, _d(u), t, _d(out))
        else:
            lib().orc_dg_residual_fd(self._h, _d(u), t, _d(out))
        return out

    def fv_residual(self, u, t=0.0):
        u = self._u(u)
        out = np.zeros_like(u)
        ds = np.zeros((self.K, self.np, self.np))
        lib().orc_fv_residual(self._h, _d(u), t, _d(out), _d(ds))
        return out, ds

    def dt(self, u, t=0.0, cfl=0.5, rule=0):
        return lib().orc_dt(self._h, _d(self._u(u)), t, cfl, rule)

    def step(self, u, nsteps, t=0.0, cfl=0.5, dt_rule=0, limiting=2, beta=0.1, bounds=0, entropy=0):
        """Returns (u_new, t_new, dt_history, stats dict)."""
        u = self._u(u).copy()
        tt = np.array([t])
        dts = np.zeros(max(nsteps, 1))
        st = np.zeros(16)
        lib().orc_stats_init(_d(st))
        lib().orc_step(self._h, _d(u), nsteps, _d(tt), cfl, dt_rule, limiting, beta, bounds, entropy, _d(dts),
                       _d(st))
        return u, float(tt[0]), dts[:nsteps], dict(zip(ST_NAMES, st[:13].tolist()))

    def integrals(self, u):
        out = np.zeros(4)
        lib().orc_integrals(self._h, _d(self._u(u)), _d(out))
        return out


def stats_dict(st):
    return dict(zip(ST_NAMES, np.asarray(st)[:13].tolist()))
