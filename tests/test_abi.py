"""CPU checks of the C-ABI library: it loads, exports every function the
header declares, and the host-side validation (mesh, degree, options)
returns the documented statuses before any device work."""
import os
import re

import numpy as np
import pytest

from paper_2607_06045_b300 import build, idp
from paper_2607_06045_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def header_functions(name="idp_dgsem.h"):
    src = open(os.path.join(ROOT, "include", name)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(idp\w*_\w+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = header_functions()
    assert len(names) >= 13
    L = idp.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(idp.EXPORTS)
    names3 = header_functions("idp_dgsem3d.h")
    for n in names3:
        assert hasattr(L, n), n
    assert set(names3) == set(idp.EXPORTS3)
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert headers == ["idp_dgsem.h", "idp_dgsem3d.h"]


def test_launch_config_rejects_null_context():
    L = idp.lib()
    assert L.idp_dgsem_launch_config(None, None, None, None) == 1   # IDP_E_ARG


def test_status_strings_and_defaults():
    L = idp.lib()
    for code in range(9):
        assert L.idp_status_str(code)
    o = idp.options()
    assert o.limiting == 2 and o.beta == 0.1 and o.mortar_projection == 1 and o.precision == 0


def _create(mesh, N=3, **kw):
    d, keep = idp.mesh_desc(mesh)
    import ctypes as C
    h = C.c_void_p()
    o = idp.options(**kw)
    rc = idp.lib().idp_dgsem_create(C.byref(d), N, 1.4, C.byref(o), C.byref(h))
    if rc == idp.IDP_OK:
        idp.lib().idp_dgsem_destroy(h)
    return rc


def test_rejects_unbalanced_mesh():
    # one leaf refined twice next to a level-0 leaf: 2 levels across a face
    m = W.uniform_mesh(2, 2)
    lev = [0, 0, 0]
    ix = [0, 0, 1]
    iy = [0, 1, 1]
    # leaf (0,1,0) refined to level 2 fully (16 leaves)
    for a in range(4):
        for b in range(4):
            lev.append(2); ix.append(4 + a); iy.append(b)
    m.level = np.array(lev, np.int8); m.ix = np.array(ix, np.int32); m.iy = np.array(iy, np.int32)
    assert _create(m) == idp.IDP_E_MESH


def test_rejects_overlap_and_gap():
    m = W.uniform_mesh(2, 2)
    m2 = W.Mesh(nx0=2, ny0=2, box=m.box, level=np.array([0, 0, 0, 0, 1], np.int8),
                ix=np.array([0, 1, 0, 1, 0], np.int32), iy=np.array([0, 0, 1, 1, 0], np.int32))
    assert _create(m2) == idp.IDP_E_MESH           # overlap
    m3 = W.Mesh(nx0=2, ny0=2, box=m.box, level=np.array([0, 0, 0], np.int8),
                ix=np.array([0, 1, 0], np.int32), iy=np.array([0, 0, 1], np.int32))
    assert _create(m3) == idp.IDP_E_MESH           # gap
    m4 = W.Mesh(nx0=2, ny0=2, box=m.box, level=np.array([0, 0, 0, 0], np.int8),
                ix=np.array([0, 1, 0, 2], np.int32), iy=np.array([0, 0, 1, 1], np.int32))
    assert _create(m4) == idp.IDP_E_MESH           # out of range


def test_rejects_bad_arguments():
    m = W.uniform_mesh(2, 2)
    assert _create(m, N=0) == idp.IDP_E_ARG
    assert _create(m, N=8) == idp.IDP_E_ARG
    assert _create(m, limiting=4) == idp.IDP_E_ARG
    assert _create(m, beta=1.5) == idp.IDP_E_ARG
    assert _create(m, cfl=0.0) == idp.IDP_E_ARG
    assert _create(m, elems_per_block=3) == idp.IDP_E_ARG
    assert _create(m, bounds=2) == idp.IDP_E_ARG
    assert _create(m, bounds=-1) == idp.IDP_E_ARG
    assert _create(m, entropy_bound=2) == idp.IDP_E_ARG
    assert _create(m, volume_flux=2) == idp.IDP_E_ARG
    assert _create(m, mortar_low=2) == idp.IDP_E_ARG
    mj = W.uniform_mesh(2, 2, bc=(6, 6, W.BC_PERIODIC, W.BC_PERIODIC))
    assert _create(mj) == idp.IDP_E_ARG
    mb = W.uniform_mesh(2, 2, bc=(W.BC_PERIODIC, W.BC_WALL, W.BC_PERIODIC, W.BC_PERIODIC))
    assert _create(mb) == idp.IDP_E_ARG
    assert _create(m, grid_mode=3) == idp.IDP_E_ARG
    L = idp.lib()
    assert L.idp_eval_math(3, None, None, 1, None) == idp.IDP_E_ARG
    assert L.idp_eval_math(0, None, None, -1, None) == idp.IDP_E_ARG
    assert L.idp_eval_math(0, None, None, 4, None) == idp.IDP_E_ARG
    assert L.idp_eval_math(2, None, None, 0, None) == idp.IDP_OK


def test_rejects_empty_mesh():
    import ctypes as C
    d, keep = idp.mesh_desc(W.uniform_mesh(2, 2))
    d.n_leaves = 0
    h = C.c_void_p()
    assert idp.lib().idp_dgsem_create(C.byref(d), 3, 1.4, C.byref(idp.options()), C.byref(h)) == idp.IDP_E_ARG


def test_valid_mesh_without_gpu_is_a_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    assert _create(W.square_mesh()) == idp.IDP_E_CUDA
