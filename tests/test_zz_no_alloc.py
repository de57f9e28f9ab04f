"""The allocation-free conservation totals (idp_integrals_noalloc) agree with
idp_dgsem_integrals on two calls in a row through the C ABI.

Callers that may not allocate device memory -- code recording a CUDA graph, a
framework with a fixed memory budget, a host callback -- use that entry
point; its scratch is a fixed array inside the library, shared by all calls.
The second call uses a smaller mesh than the first, so a stale partial left
in the shared scratch would show up in its totals."""
import numpy as np
import pytest

from paper_2607_06045_b300 import build, idp
from paper_2607_06045_b300 import workloads as W

pytestmark = pytest.mark.gpu


def areas(meshes):
    out = []
    for m in meshes:
        lev = m.level.astype(np.int64)
        dx = (m.box[2] - m.box[0]) / (float(m.nx0) * (2.0 ** lev))
        dy = (m.box[3] - m.box[1]) / (float(m.ny0) * (2.0 ** lev))
        out.append(dx * dy)
    return np.concatenate(out)


def test_noalloc_integrals_match_context_integrals():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cases = [([W.square_mesh(), W.box_refined_mesh(6, 4, (0.0, 0.0, 1.5, 1.0), (0.2, 0.2, 0.9, 0.6))], 4),
             ([W.uniform_mesh(5, 3, (0.0, 0.0, 2.0, 1.0), bc=(W.BC_OUTFLOW,) * 4)], 3)]
    for call, (meshes, N) in enumerate(cases):
        us = [W.random_state(m, N, seed=call * 10 + k) for k, m in enumerate(meshes)]
        u = W.concat_states(us)
        ctx = idp.Context(meshes if len(meshes) > 1 else meshes[0], N)
        ud = torch.from_numpy(u).cuda()
        ref = ctx.idp_dgsem_integrals(ud)
        area = torch.from_numpy(areas(meshes)).cuda()
        off = torch.from_numpy(ctx.sim_offsets.astype(np.int64)).cuda()
        out = torch.full((len(meshes), 4), float("nan"), dtype=torch.float64, device="cuda")
        rc = idp.idp_integrals_noalloc(ud, area, N, off, out)
        assert rc == idp.IDP_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0.0)
        ctx.close()


def test_noalloc_rejects_oversized_meshes():
    import ctypes as C
    rc = idp.lib().idp_integrals_noalloc(C.c_void_p(8), C.c_void_p(8), idp.NOALLOC_MAX_ELEMS + 1, 3,
                                         C.c_void_p(8), 1, C.c_void_p(8), None)
    assert rc == idp.IDP_E_ARG
