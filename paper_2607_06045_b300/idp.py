"""Python binding of libidpdgsem.so (argument marshalling only).

Mirrors the C ABI of include/idp_dgsem.h: the same entry-point names, with
device arrays passed as torch CUDA tensors (FP64, contiguous, layout
u[4][K][N+1][N+1]) and the stream taken from torch's current stream unless
given. Every computation runs in the library's CUDA kernels; there is no
fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libidpdgsem.so")

IDP_OK, IDP_E_ARG, IDP_E_MESH, IDP_E_CUDA, IDP_E_STATE, IDP_E_DT, IDP_E_NUMERIC, IDP_E_TIMEOUT, IDP_E_UNSUPPORTED = range(9)


class MeshDesc(C.Structure):
    _fields_ = [("nx0", C.c_int32), ("ny0", C.c_int32),
                ("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double), ("y1", C.c_double),
                ("n_leaves", C.c_int32),
                ("level", C.POINTER(C.c_int8)), ("ix", C.POINTER(C.c_int32)), ("iy", C.POINTER(C.c_int32)),
                ("bc", C.c_int32 * 4), ("bc_prim", (C.c_double * 4) * 4),
                ("dmr_post", C.c_double * 4), ("dmr_pre", C.c_double * 4)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("limiting", C.c_int32), ("bounds", C.c_int32), ("dt_rule", C.c_int32),
                ("beta", C.c_double), ("cfl", C.c_double), ("mortar_projection", C.c_int32),
                ("elems_per_block", C.c_int32), ("collect_stats", C.c_int32), ("grid_mode", C.c_int32),
                ("entropy_bound", C.c_int32), ("volume_flux", C.c_int32), ("mortar_low", C.c_int32)]


class AmrParams(C.Structure):
    _fields_ = [("indicator", C.c_int32), ("variable", C.c_int32), ("refine_threshold", C.c_double),
                ("coarsen_threshold", C.c_double), ("min_level", C.c_int32), ("max_level", C.c_int32),
                ("lohner_filter", C.c_double), ("zs_threshold", C.c_double)]


class LimiterStats(C.Structure):
    _fields_ = [("alpha_volume_mean", C.c_double), ("alpha_mortar_mean", C.c_double),
                ("n_stages", C.c_int64), ("n_volume_active", C.c_int64), ("n_mortar_active", C.c_int64),
                ("n_mortar_fallback", C.c_int64), ("n_viol_density", C.c_int64), ("n_viol_pressure", C.c_int64),
                ("n_nonpositive", C.c_int64), ("n_dt_exceed", C.c_int64),
                ("min_rho", C.c_double), ("min_p", C.c_double), ("n_viol_entropy", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

EXPORTS = ["idp_options_default", "idp_dgsem_create", "idp_dgsem_create_batch", "idp_dgsem_layout",
           "idp_dgsem_launch_config",
           "idp_dgsem_rhs", "idp_dgsem_dt", "idp_dgsem_step", "idp_dgsem_step_host", "idp_dgsem_integrals",
           "idp_dgsem_limiter_stats", "idp_dgsem_sync", "idp_dgsem_destroy", "idp_status_str",
           "idp_last_cuda_error", "idp_dgsem_profile", "idp_dgsem_profile_read", "idp_dgsem_profile_kernels",
           "idp_probe_pipes", "idp_eval_math",
           "idp_integrals_noalloc", "idp_amr_params_default", "idp_dgsem_amr_indicator", "idp_amr_plan",
           "idp_amr_transfer", "idp_dgsem_adapt", "idp_dgsem_leaves", "idp_dgsem_mesh_tables"]


EXPORTS3 = ["idp3d_options_default", "idp3d_create", "idp3d_create_octree", "idp3d_layout", "idp3d_mesh_info",
            "idp3d_octree_tables", "idp3d_stage_factors",
            "idp3d_rhs", "idp3d_dt", "idp3d_step", "idp3d_integrals", "idp3d_limiter_stats", "idp3d_destroy"]


class GridDesc3(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("x1", C.c_double), ("y1", C.c_double), ("z1", C.c_double),
                ("bc", C.c_int32 * 6), ("bc_prim", (C.c_double * 5) * 6)]


class Options3(C.Structure):
    _fields_ = [("limiting", C.c_int32), ("beta", C.c_double), ("cfl", C.c_double), ("precision", C.c_int32)]


class LimiterStats3(C.Structure):
    _fields_ = [("alpha_mean", C.c_double), ("n_active", C.c_int64), ("n_viol_density", C.c_int64),
                ("n_viol_pressure", C.c_int64), ("n_nonpositive", C.c_int64), ("n_stages", C.c_int64),
                ("min_rho", C.c_double), ("min_p", C.c_double), ("alpha_mortar", C.c_double),
                ("n_mortar_active", C.c_int64), ("n_mortar_fallback", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2607_06045_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.idp_status_str.restype = C.c_char_p
        L.idp_status_str.argtypes = [C.c_int]
        L.idp_last_cuda_error.restype = C.c_char_p
        L.idp_last_cuda_error.argtypes = []
        L.idp_options_default.argtypes = [C.POINTER(Options)]
        L.idp_dgsem_create.argtypes = [C.POINTER(MeshDesc), C.c_int32, C.c_double, C.POINTER(Options), C.POINTER(vp)]
        L.idp_dgsem_create_batch.argtypes = [C.POINTER(MeshDesc), C.c_int32, C.c_int32, C.c_double,
                                             C.POINTER(Options), C.POINTER(vp)]
        L.idp_dgsem_layout.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int64)]
        L.idp_dgsem_launch_config.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                              C.POINTER(C.c_int32)]
        L.idp_dgsem_rhs.argtypes = [vp, vp, C.c_double, C.c_double, vp, vp]
        L.idp_dgsem_dt.argtypes = [vp, vp, dp, dp, vp]
        L.idp_dgsem_step.argtypes = [vp, vp, C.c_int32, dp, dp, vp]
        L.idp_dgsem_step_host.argtypes = [vp, vp, C.c_int32, dp, dp, vp]
        L.idp_dgsem_integrals.argtypes = [vp, vp, dp, vp]
        L.idp_dgsem_limiter_stats.argtypes = [vp, C.POINTER(LimiterStats), vp]
        L.idp_dgsem_sync.argtypes = [vp, vp]
        L.idp_dgsem_destroy.argtypes = [vp]
        L.idp_dgsem_profile.argtypes = [vp, C.c_int32]
        L.idp_dgsem_profile_read.argtypes = [vp, dp, C.POINTER(C.c_int64), dp, C.POINTER(C.c_int64), C.c_int32]
        L.idp_dgsem_profile_kernels.argtypes = [vp, dp, C.POINTER(C.c_int64), C.c_int32]
        L.idp_probe_pipes.argtypes = [dp, vp]
        L.idp_eval_math.argtypes = [C.c_int32, vp, vp, C.c_int64, vp]
        L.idp_integrals_noalloc.argtypes = [vp, vp, C.c_int64, C.c_int32, vp, C.c_int32, vp, vp]
        ip, i8p = C.POINTER(C.c_int32), C.POINTER(C.c_int8)
        L.idp_amr_params_default.argtypes = [C.POINTER(AmrParams)]
        L.idp_dgsem_amr_indicator.argtypes = [vp, vp, C.POINTER(AmrParams), vp, vp]
        L.idp_amr_plan.argtypes = [C.POINTER(MeshDesc), dp, C.POINTER(AmrParams), C.c_int32, ip, i8p, ip, ip, ip, ip]
        L.idp_amr_transfer.argtypes = [C.c_int32, C.c_double, vp, C.c_int64, vp, C.c_int64, ip, ip, C.c_double,
                                       C.POINTER(C.c_int64), vp]
        i64p = C.POINTER(C.c_int64)
        L.idp_dgsem_adapt.argtypes = [vp, vp, C.POINTER(AmrParams), vp, C.c_int64, i64p, i64p, vp]
        L.idp_dgsem_leaves.argtypes = [vp, i8p, ip, ip]
        L.idp_dgsem_mesh_tables.argtypes = [vp, i64p, ip, C.POINTER(C.c_uint8), ip, ip, ip, ip, ip, ip, ip, ip]
        L.idp3d_options_default.argtypes = [C.POINTER(Options3)]
        L.idp3d_create.argtypes = [C.POINTER(GridDesc3), C.c_int32, C.c_double, C.POINTER(Options3), C.POINTER(vp)]
        L.idp3d_create_octree.argtypes = [C.POINTER(GridDesc3), C.c_int64, i8p, ip, ip, ip, C.c_int32, C.c_double,
                                          C.POINTER(Options3), C.POINTER(vp)]
        L.idp3d_layout.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
        L.idp3d_mesh_info.argtypes = [vp, i64p, i64p]
        L.idp3d_stage_factors.argtypes = [vp, dp, dp, vp]
        L.idp3d_octree_tables.argtypes = [C.POINTER(GridDesc3), C.c_int64, i8p, ip, ip, ip, C.c_int32, i64p, i64p, ip,
                                          ip]
        L.idp3d_rhs.argtypes = [vp, vp, C.c_double, vp, vp]
        L.idp3d_dt.argtypes = [vp, vp, dp, vp]
        L.idp3d_step.argtypes = [vp, vp, C.c_int32, dp, dp, vp]
        L.idp3d_integrals.argtypes = [vp, vp, dp, vp]
        L.idp3d_limiter_stats.argtypes = [vp, C.POINTER(LimiterStats3), vp]
        L.idp3d_destroy.argtypes = [vp]
        L.idp3d_destroy.restype = None
        for f in EXPORTS3:
            if f != "idp3d_destroy":
                getattr(L, f).restype = C.c_int
        L.idp_dgsem_destroy.restype = None
        for f in EXPORTS:
            if f not in ("idp_dgsem_destroy", "idp_status_str", "idp_last_cuda_error"):
                getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


class IdpError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = f"{where}: {lib().idp_status_str(code).decode()} (status {code})"
        if code == IDP_E_CUDA:
            msg += f" [{lib().idp_last_cuda_error().decode()}]"
        super().__init__(msg)


def _check(code, where):
    if code != IDP_OK:
        raise IdpError(code, where)


def idp_probe_pipes(stream=None):
    """[FP64 TFLOP/s, FP32 TFLOP/s, div, sqrt, log cost in DFMA-equivalents]."""
    out = (C.c_double * 5)()
    _check(lib().idp_probe_pipes(out, _stream(stream)), "idp_probe_pipes")
    return list(out)


def idp_eval_math(fn, x, y, stream=None):
    """y = f(x) elementwise on CUDA FP64 tensors with the library's FP64 routines
    (fn 0: 1/x, 1: sqrt, 2: ln)."""
    assert x.is_cuda and y.is_cuda and x.dtype == y.dtype and x.numel() == y.numel()
    _check(lib().idp_eval_math(int(fn), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.numel(),
                               _stream(stream)), "idp_eval_math")


# kernel kinds of one step, in the order of the IDP_K_* constants
KERNELS = ["dt_init", "mortar_flux", "dt", "element", "mortar_limit", "mortar_apply", "time_advance",
           "element_lo", "mortar_lob", "face", "dt_speed", "dt_filter"]

NOALLOC_MAX_ELEMS = 1 << 19


def idp_integrals_noalloc(u, elem_area, N, sim_offsets, out, stream=None):
    """Allocation-free conservation totals; every argument is a caller-owned
    CUDA tensor (u FP64 [4][K][N+1][N+1], elem_area FP64 [K], sim_offsets
    int64 [n_sims+1], out FP64 [n_sims][4]). Returns the status code."""
    import torch
    assert elem_area.is_cuda and elem_area.dtype == torch.float64 and sim_offsets.dtype == torch.int64
    assert out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
    assert elem_area.is_contiguous() and sim_offsets.is_cuda and sim_offsets.is_contiguous()
    # u must hold the elements the areas describe, at degree N
    assert u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()
    assert tuple(u.shape) == (4, elem_area.shape[0], N + 1, N + 1), (tuple(u.shape), elem_area.shape[0], N)
    assert out.numel() >= 4 * (sim_offsets.shape[0] - 1)
    return lib().idp_integrals_noalloc(_ptr(u), C.c_void_p(elem_area.data_ptr()), int(elem_area.shape[0]), int(N),
                                       C.c_void_p(sim_offsets.data_ptr()), int(sim_offsets.shape[0] - 1),
                                       C.c_void_p(out.data_ptr()), _stream(stream))


def options(**kw) -> Options:
    o = Options()
    lib().idp_options_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def mesh_desc(mesh) -> tuple:
    """MeshDesc for a workloads.Mesh plus the arrays it points into."""
    lev = np.ascontiguousarray(mesh.level, dtype=np.int8)
    ix = np.ascontiguousarray(mesh.ix, dtype=np.int32)
    iy = np.ascontiguousarray(mesh.iy, dtype=np.int32)
    d = MeshDesc()
    d.nx0, d.ny0 = int(mesh.nx0), int(mesh.ny0)
    d.x0, d.y0, d.x1, d.y1 = (float(v) for v in mesh.box)
    d.n_leaves = int(lev.shape[0])
    d.level = lev.ctypes.data_as(C.POINTER(C.c_int8))
    d.ix = ix.ctypes.data_as(C.POINTER(C.c_int32))
    d.iy = iy.ctypes.data_as(C.POINTER(C.c_int32))
    for s in range(4):
        d.bc[s] = int(mesh.bc[s])
        for v in range(4):
            d.bc_prim[s][v] = float(np.asarray(mesh.bc_prim)[s][v])
    for v in range(4):
        d.dmr_post[v] = float(mesh.dmr_post[v])
        d.dmr_pre[v] = float(mesh.dmr_pre[v])
    return d, (lev, ix, iy)


def _ptr(t):
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "FP64 contiguous CUDA tensor expected"
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """idp_dgsem context for one mesh (or a batch of meshes)."""

    def __init__(self, meshes, N: int, gamma: float = 1.4, opts: Optional[Options] = None, **kw):
        if opts is None:
            opts = options(**kw)
        self.N, self.np, self.gamma, self.opts = N, N + 1, gamma, opts
        single = not isinstance(meshes, (list, tuple))
        ml = [meshes] if single else list(meshes)
        self.meshes = ml
        descs, self._keep = [], []
        for m in ml:
            d, keep = mesh_desc(m)
            descs.append(d)
            self._keep.append(keep)
        arr = (MeshDesc * len(descs))(*descs)
        h = C.c_void_p()
        if single:
            rc = lib().idp_dgsem_create(C.byref(arr[0]), N, gamma, C.byref(opts), C.byref(h))
        else:
            rc = lib().idp_dgsem_create_batch(arr, len(descs), N, gamma, C.byref(opts), C.byref(h))
        _check(rc, "idp_dgsem_create")
        self._h = h
        K, M, S = C.c_int64(), C.c_int64(), C.c_int32()
        _check(lib().idp_dgsem_layout(h, C.byref(K), C.byref(M), C.byref(S), None), "idp_dgsem_layout")
        self.K, self.M, self.n_sims = K.value, M.value, S.value
        off = (C.c_int64 * (self.n_sims + 1))()
        lib().idp_dgsem_layout(h, None, None, None, off)
        self.sim_offsets = np.array(off[:], dtype=np.int64)

    def close(self):
        if getattr(self, "_h", None):
            lib().idp_dgsem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (4, self.K, self.np, self.np)

    def idp_dgsem_rhs(self, u, t, dt, out, stream=None):
        _check(lib().idp_dgsem_rhs(self._h, _ptr(u), float(t), float(dt), _ptr(out), _stream(stream)), "idp_dgsem_rhs")

    def idp_dgsem_dt(self, u, t=None, stream=None):
        th = np.zeros(self.n_sims) if t is None else np.ascontiguousarray(np.broadcast_to(t, self.n_sims), dtype=np.float64)
        out = np.zeros(self.n_sims)
        dp = C.POINTER(C.c_double)
        _check(lib().idp_dgsem_dt(self._h, _ptr(u), th.ctypes.data_as(dp), out.ctypes.data_as(dp), _stream(stream)),
               "idp_dgsem_dt")
        return out

    def idp_dgsem_step(self, u, n_steps, t, stream=None, check=True):
        """Advance u in place; t: per-sim times (array, updated in place). Returns (status, dt_last)."""
        dp = C.POINTER(C.c_double)
        dtl = np.zeros(self.n_sims)
        rc = lib().idp_dgsem_step(self._h, _ptr(u), int(n_steps), t.ctypes.data_as(dp), dtl.ctypes.data_as(dp),
                                  _stream(stream))
        if check:
            _check(rc, "idp_dgsem_step")
        return rc, dtl

    def idp_dgsem_step_host(self, u_host, n_steps, t, stream=None, check=True):
        """u_host: a (pinned) CPU torch tensor or numpy array, updated in place."""
        dp = C.POINTER(C.c_double)
        dtl = np.zeros(self.n_sims)
        ptr = C.c_void_p(u_host.data_ptr()) if hasattr(u_host, "data_ptr") else u_host.ctypes.data_as(C.c_void_p)
        rc = lib().idp_dgsem_step_host(self._h, ptr, int(n_steps), t.ctypes.data_as(dp), dtl.ctypes.data_as(dp),
                                       _stream(stream))
        if check:
            _check(rc, "idp_dgsem_step_host")
        return rc, dtl

    def idp_dgsem_integrals(self, u, stream=None):
        out = np.zeros((self.n_sims, 4))
        _check(lib().idp_dgsem_integrals(self._h, _ptr(u), out.ctypes.data_as(C.POINTER(C.c_double)),
                                         _stream(stream)), "idp_dgsem_integrals")
        return out

    def idp_dgsem_limiter_stats(self, stream=None, check=False):
        st = LimiterStats()
        rc = lib().idp_dgsem_limiter_stats(self._h, C.byref(st), _stream(stream))
        if check:
            _check(rc, "idp_dgsem_limiter_stats")
        return rc, st.as_dict()

    def idp_dgsem_profile(self, mode=1):
        """0 off; 1 step spans around graph launches; 2 kernel-by-kernel steps with element-pass events."""
        _check(lib().idp_dgsem_profile(self._h, int(mode)), "idp_dgsem_profile")

    def idp_dgsem_profile_read(self, reset=True):
        """(element-pass ms, element launches, step ms, steps) accumulated since the last reset."""
        ms, n, sms, ns = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
        _check(lib().idp_dgsem_profile_read(self._h, C.byref(ms), C.byref(n), C.byref(sms), C.byref(ns),
                                            1 if reset else 0), "idp_dgsem_profile_read")
        return ms.value, n.value, sms.value, ns.value

    def idp_dgsem_profile_kernels(self, reset=False):
        """{kernel kind: (ms, launches)} accumulated in profiling mode 2."""
        ms = (C.c_double * len(KERNELS))()
        n = (C.c_int64 * len(KERNELS))()
        _check(lib().idp_dgsem_profile_kernels(self._h, ms, n, 1 if reset else 0), "idp_dgsem_profile_kernels")
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNELS)}

    def launches_per_step(self):
        """Kernels one SSP-RK3 step launches (mirrors the step sequence)."""
        M = self.M > 0
        lim = self.opts.limiting > 0
        # low-order bounds: a pre-pass over the elements and a mortar gather
        lob = (1 + (1 if M else 0)) if (self.opts.limiting >= 2 and self.opts.bounds == 1) else 0
        # FP64 path, default kernel: the conforming-face kernel before each element pass
        o = self.opts
        ext = (o.limiting >= 2 and (o.bounds == 1 or o.entropy_bound == 1)) or o.volume_flux == 1
        el = 2 if (o.precision == 0 and not ext) else 1
        # mortar flux, dt (its wave-speed pre-pass without a face buffer); the
        # time-step minimum needs no reset launch in a step
        ext_or_f32 = o.precision == 1 or ext
        n = (1 if (M and self.opts.dt_rule == 0) else 0) + 1 + (1 if ext_or_f32 or o.dt_rule != 0 else 0)
        # FP64 path with the face buffer: the time step's FP32 pass before its FP64 pass
        n += 1 if (not ext_or_f32 and o.dt_rule == 0) else 0
        # per stage with mortars and limiting: one mortar limiting-and-apply launch
        n += (1 if (M and self.opts.dt_rule != 0) else 0) + el + lob + (1 if (M and lim) else 0)   # stage 1
        n += 2 * ((1 if M else 0) + el + lob + (1 if (M and lim) else 0))   # stages 2, 3
        return n + 1                                                        # time advance

    def idp_dgsem_launch_config(self):
        """(elements per block, persistent grid 0/1, grid size) of the element pass; zeros before tuning."""
        e, p, g = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().idp_dgsem_launch_config(self._h, C.byref(e), C.byref(p), C.byref(g)),
               "idp_dgsem_launch_config")
        return e.value, p.value, g.value

    def idp_dgsem_sync(self, stream=None):
        return lib().idp_dgsem_sync(self._h, _stream(stream))

    # ---- adaptive mesh refinement -------------------------------------------

    def idp_dgsem_amr_indicator(self, u, params=None, stream=None):
        """Per-element AMR indicator of the device state u (a device tensor of K doubles)."""
        import torch
        p = params if params is not None else amr_params()
        ind = torch.empty(self.K, dtype=torch.float64, device=u.device)
        _check(lib().idp_dgsem_amr_indicator(self._h, _ptr(u), C.byref(p), _ptr(ind), _stream(stream)),
               "idp_dgsem_amr_indicator")
        return ind

    def adapt(self, u, params=None, stream=None):
        """One AMR step of a single-mesh context: indicator (device), plan (host),
        transfer (device) and a context for the adapted mesh with the same
        options. Returns (context, state, (kind, src), scaled families)."""
        import dataclasses
        import torch
        if self.n_sims != 1:
            raise ValueError("adapt works on single-mesh contexts")
        p = params if params is not None else amr_params()
        ind = self.idp_dgsem_amr_indicator(u, p, stream)
        torch.cuda.synchronize()
        lev, ix, iy, kind, src = idp_amr_plan(self.meshes[0], ind.cpu().numpy(), p)
        mesh2 = dataclasses.replace(self.meshes[0], level=lev, ix=ix, iy=iy)
        un, scaled = idp_amr_transfer(self.N, self.gamma, u, kind, src, p.zs_threshold, stream)
        return Context(mesh2, self.N, self.gamma, opts=self.opts), un, (kind, src), scaled


    def idp_dgsem_adapt(self, u, params=None, capacity=None, out=None, stream=None):
        """One AMR step on the device, in this context: the context now steps
        the adapted mesh. u_new is written into `out` (a flat FP64 device
        tensor of at least 4 capacity (N+1)^2 values; allocated for capacity
        = 4 K when None) and returned as a (4, K_new, N+1, N+1) view, with
        the number of scaled families."""
        import torch
        p = params if params is not None else amr_params()
        nn = self.np * self.np
        if out is None:
            cap = int(capacity) if capacity is not None else 4 * self.K
            out = torch.empty(4 * cap * nn, dtype=torch.float64, device=u.device)
        else:
            cap = out.numel() // (4 * nn) if capacity is None else int(capacity)
            assert out.numel() >= 4 * cap * nn
        n, sc = C.c_int64(), C.c_int64()
        rc = lib().idp_dgsem_adapt(self._h, _ptr(u), C.byref(p), _ptr(out), cap, C.byref(n), C.byref(sc),
                                   _stream(stream))
        if rc == 1 and n.value > cap:   # IDP_E_ARG with the count: the buffer is too small
            raise ValueError(f"idp_dgsem_adapt: {n.value} elements exceed the capacity {cap}")
        _check(rc, "idp_dgsem_adapt")
        kn = n.value
        K, M = C.c_int64(), C.c_int64()
        _check(lib().idp_dgsem_layout(self._h, C.byref(K), C.byref(M), None, None), "idp_dgsem_layout")
        self.K, self.M = K.value, M.value
        self.sim_offsets = np.array([0, kn], dtype=np.int64)
        self._leaves_stale = True   # `meshes` fetches the new leaves when read
        return out[: 4 * kn * nn].view(4, kn, self.np, self.np), sc.value

    @property
    def meshes(self):
        """The context's meshes (after idp_dgsem_adapt: the adapted leaves)."""
        if getattr(self, "_leaves_stale", False):
            import dataclasses
            lev, ix, iy = self.leaves()
            self._meshes = [dataclasses.replace(self._meshes[0], level=lev, ix=ix, iy=iy)]
            self._leaves_stale = False
        return self._meshes

    @meshes.setter
    def meshes(self, v):
        self._meshes = v
        self._leaves_stale = False

    def leaves(self):
        """(level, ix, iy) of the context's elements (host arrays)."""
        lev = np.zeros(self.K, np.int8)
        ix, iy = np.zeros(self.K, np.int32), np.zeros(self.K, np.int32)
        ip = C.POINTER(C.c_int32)
        _check(lib().idp_dgsem_leaves(self._h, lev.ctypes.data_as(C.POINTER(C.c_int8)), ix.ctypes.data_as(ip),
                                      iy.ctypes.data_as(ip)), "idp_dgsem_leaves")
        return lev, ix, iy

    def mesh_tables(self, arrays=False):
        """The context's device mesh tables as host arrays (test support)."""
        sizes = np.zeros(6, np.int64)
        i64p, ip = C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        if not arrays:
            _check(lib().idp_dgsem_mesh_tables(self._h, sizes.ctypes.data_as(i64p), *([None] * 10)),
                   "idp_dgsem_mesh_tables")
            return {"sizes": [int(v) for v in sizes]}
        _check(lib().idp_dgsem_mesh_tables(self._h, sizes.ctypes.data_as(i64p), *([None] * 10)),
               "idp_dgsem_mesh_tables")
        K, M, nn, nb, nf, _ = (int(v) for v in sizes)
        t = {"fnbr": np.zeros((K, 4), np.int32), "ftype": np.zeros((K, 4), np.uint8),
             "m_large": np.zeros(M, np.int32), "m_small": np.zeros((M, 2), np.int32), "m_info": np.zeros(M, np.int32),
             "mn_node": np.zeros(nn, np.int32), "mn_slot": np.zeros((nn, 2), np.int32),
             "mb_node_off": np.zeros(nb + 1, np.int32), "mb_for_off": np.zeros(nb + 1, np.int32),
             "mb_foreign": np.zeros(max(nf, 1), np.int32)}
        order = ["fnbr", "ftype", "m_large", "m_small", "m_info", "mn_node", "mn_slot", "mb_node_off", "mb_for_off",
                 "mb_foreign"]
        ptrs = [t[k].ctypes.data_as(C.POINTER(C.c_uint8) if k == "ftype" else ip) for k in order]
        _check(lib().idp_dgsem_mesh_tables(self._h, sizes.ctypes.data_as(i64p), *ptrs), "idp_dgsem_mesh_tables")
        t["mb_foreign"] = t["mb_foreign"][:nf]
        t["sizes"] = [int(v) for v in sizes]
        return t


def amr_params(**kw) -> AmrParams:
    p = AmrParams()
    lib().idp_amr_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def idp_amr_plan(mesh, ind, params=None):
    """(level, ix, iy, kind, src) of the adapted mesh (host arrays)."""
    p = params if params is not None else amr_params()
    d, keep = mesh_desc(mesh)
    ind = np.ascontiguousarray(ind, dtype=np.float64)
    cap = 4 * mesh.n_elems
    lev = np.zeros(cap, np.int8)
    ix, iy, kind = np.zeros(cap, np.int32), np.zeros(cap, np.int32), np.zeros(cap, np.int32)
    src = np.zeros((cap, 4), np.int32)
    n = C.c_int32()
    ip = C.POINTER(C.c_int32)
    _check(lib().idp_amr_plan(C.byref(d), ind.ctypes.data_as(C.POINTER(C.c_double)), C.byref(p), cap, C.byref(n),
                              lev.ctypes.data_as(C.POINTER(C.c_int8)), ix.ctypes.data_as(ip), iy.ctypes.data_as(ip),
                              kind.ctypes.data_as(ip), src.ctypes.data_as(ip)), "idp_amr_plan")
    k = n.value
    return lev[:k].copy(), ix[:k].copy(), iy[:k].copy(), kind[:k].copy(), src[:k].copy()


def idp_amr_transfer(N, gamma, u_old, kind, src, zs_threshold=1e-10, stream=None):
    """(state on the adapted mesh as a new device tensor, scaled families)."""
    import torch
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    src = np.ascontiguousarray(src, dtype=np.int32)
    n_new = kind.shape[0]
    un = torch.empty((4, n_new, N + 1, N + 1), dtype=torch.float64, device=u_old.device)
    sc = C.c_int64()
    ip = C.POINTER(C.c_int32)
    _check(lib().idp_amr_transfer(int(N), float(gamma), _ptr(u_old), int(u_old.shape[1]), _ptr(un), n_new,
                                  kind.ctypes.data_as(ip), src.ctypes.data_as(ip), float(zs_threshold), C.byref(sc),
                                  _stream(stream)), "idp_amr_transfer")
    return un, sc.value


# ---- 3D (include/idp_dgsem3d.h) ----------------------------------------------

def _grid_desc3(mesh) -> GridDesc3:
    octree = hasattr(mesh, "level")
    d = GridDesc3()
    d.nx, d.ny, d.nz = (mesh.nx0, mesh.ny0, mesh.nz0) if octree else (mesh.nx, mesh.ny, mesh.nz)
    d.x0, d.y0, d.z0, d.x1, d.y1, d.z1 = (float(v) for v in mesh.box)
    for s in range(6):
        d.bc[s] = int(mesh.bc[s])
        for v in range(5):
            d.bc_prim[s][v] = float(np.asarray(mesh.bc_prim)[s, v])
    return d


def octree_tables3(mesh, N: int):
    """idp3d_octree_tables on the host (no GPU): (mortar_info [M][7],
    nbr [K][6], number of mortar nodes) of a workloads.Mesh3-like octree."""
    d = _grid_desc3(mesh)
    lev = np.ascontiguousarray(mesh.level, dtype=np.int8)
    ix, iy, iz = (np.ascontiguousarray(a, dtype=np.int32) for a in (mesh.ix, mesh.iy, mesh.iz))
    ip, i8 = C.POINTER(C.c_int32), C.POINTER(C.c_int8)
    args = (C.byref(d), C.c_int64(lev.size), lev.ctypes.data_as(i8), ix.ctypes.data_as(ip), iy.ctypes.data_as(ip),
            iz.ctypes.data_as(ip), N)
    M, MN = C.c_int64(), C.c_int64()
    _check(lib().idp3d_octree_tables(*args, C.byref(M), C.byref(MN), None, None), "idp3d_octree_tables")
    info = np.zeros((max(M.value, 1), 7), np.int32)
    nbr = np.zeros((lev.size, 6), np.int32)
    _check(lib().idp3d_octree_tables(*args, None, None, info.ctypes.data_as(ip), nbr.ctypes.data_as(ip)),
           "idp3d_octree_tables")
    return info[:M.value], nbr, MN.value


def options3(**kw) -> Options3:
    o = Options3()
    lib().idp3d_options_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context3D:
    """idp3d context for a grid of hexahedra (a workloads.Grid3-like object:
    nx, ny, nz, box, bc, bc_prim) or the leaves of a 2:1 octree (a
    workloads.Mesh3-like object: nx0, ny0, nz0, box, level, ix, iy, iz, bc,
    bc_prim) and degree N (1..4)."""

    def __init__(self, grid, N: int, gamma: float = 1.4, opts: Optional[Options3] = None, **kw):
        if opts is None:
            opts = options3(**kw)
        self.grid, self.N, self.np, self.gamma, self.opts = grid, N, N + 1, gamma, opts
        octree = hasattr(grid, "level")
        d = _grid_desc3(grid)
        h = C.c_void_p()
        if octree:
            lev = np.ascontiguousarray(grid.level, dtype=np.int8)
            ix, iy, iz = (np.ascontiguousarray(a, dtype=np.int32) for a in (grid.ix, grid.iy, grid.iz))
            ip = C.POINTER(C.c_int32)
            _check(lib().idp3d_create_octree(C.byref(d), C.c_int64(lev.size), lev.ctypes.data_as(C.POINTER(C.c_int8)),
                                             ix.ctypes.data_as(ip), iy.ctypes.data_as(ip), iz.ctypes.data_as(ip), N,
                                             C.c_double(gamma), C.byref(opts), C.byref(h)), "idp3d_create_octree")
        else:
            _check(lib().idp3d_create(C.byref(d), N, gamma, C.byref(opts), C.byref(h)), "idp3d_create")
        self._h = h
        K, npe = C.c_int64(), C.c_int32()
        lib().idp3d_layout(h, C.byref(K), C.byref(npe))
        self.K, self.nodes_per_elem = K.value, npe.value
        M, MN = C.c_int64(), C.c_int64()
        lib().idp3d_mesh_info(h, C.byref(M), C.byref(MN))
        self.n_mortars, self.n_mortar_nodes = M.value, MN.value

    def close(self):
        if getattr(self, "_h", None):
            lib().idp3d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (5, self.K, self.np, self.np, self.np)

    def idp3d_rhs(self, u, dt, out, stream=None):
        _check(lib().idp3d_rhs(self._h, _ptr(u), float(dt), _ptr(out), _stream(stream)), "idp3d_rhs")

    def idp3d_dt(self, u, stream=None):
        dt = C.c_double()
        _check(lib().idp3d_dt(self._h, _ptr(u), C.byref(dt), _stream(stream)), "idp3d_dt")
        return dt.value

    def idp3d_step(self, u, n_steps, t, stream=None, check=True):
        """n_steps steps in place; t is a length-1 numpy array (updated)."""
        tt = np.ascontiguousarray(t, dtype=np.float64)
        dl = C.c_double()
        rc = lib().idp3d_step(self._h, _ptr(u), int(n_steps), tt.ctypes.data_as(C.POINTER(C.c_double)),
                              C.byref(dl), C.c_void_p(stream) if stream is not None else None)
        t[...] = tt
        if check:
            _check(rc, "idp3d_step")
        return rc, dl.value

    def idp3d_stage_factors(self, stream=None):
        """(shock indicator per element, l_S per mortar) of the last limited stage."""
        a = np.zeros(self.K)
        ell = np.zeros(max(self.n_mortars, 1))
        _check(lib().idp3d_stage_factors(self._h, a.ctypes.data_as(C.POINTER(C.c_double)),
                                         ell.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)),
               "idp3d_stage_factors")
        return a, ell[:self.n_mortars]

    def idp3d_integrals(self, u, stream=None):
        out = np.zeros(5)
        _check(lib().idp3d_integrals(self._h, _ptr(u), out.ctypes.data_as(C.POINTER(C.c_double)),
                                     _stream(stream)), "idp3d_integrals")
        return out

    def idp3d_limiter_stats(self, stream=None):
        st = LimiterStats3()
        rc = lib().idp3d_limiter_stats(self._h, C.byref(st), _stream(stream))
        return rc, st.as_dict()
