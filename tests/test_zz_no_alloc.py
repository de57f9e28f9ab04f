"""The allocation-free conservation totals (idp_integrals_noalloc) agree with
idp_dgsem_integrals on two calls in a row through the C ABI.

Callers that may not allocate device memory -- code recording a CUDA graph, a
framework with a fixed memory budget, a host callback -- use that entry
point; its scratch is a fixed array inside the library, shared by all calls.
The second call uses a smaller mesh than the first, so a stale partial left
in the shared scratch would show up in its totals. Both calls are also
compared with the oracle's totals, and an offset beyond the mesh is clamped
to the call's own elements."""
import numpy as np
import pytest

import oracle
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
        # and against the oracle's totals of each simulation
        for k, (m, uk) in enumerate(zip(meshes, us)):
            tot = oracle.Oracle(m, N).integrals(uk)
            scale = np.abs(uk).reshape(4, -1).max(axis=1) * areas([m]).sum()
            assert np.all(np.abs(got[k] - tot) <= 1e-13 * scale), (got[k], tot)
        ctx.close()


def test_noalloc_offsets_are_clamped():
    # an offset beyond the mesh sums only this call's partials: the totals
    # equal those of the elements that exist
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m, N = W.square_mesh(), 3
    u = W.random_state(m, N, seed=5)
    ud = torch.from_numpy(u).cuda()
    area = torch.from_numpy(areas([m])).cuda()
    K = m.n_elems
    off = torch.tensor([0, K + 1000], dtype=torch.int64, device="cuda")
    out = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    assert idp.idp_integrals_noalloc(ud, area, N, off, out) == idp.IDP_OK
    torch.cuda.synchronize()
    tot = oracle.Oracle(m, N).integrals(u)
    scale = np.abs(u).reshape(4, -1).max(axis=1) * areas([m]).sum()
    assert np.all(np.abs(out.cpu().numpy()[0] - tot) <= 1e-13 * scale)


def test_noalloc_rejects_oversized_meshes():
    import ctypes as C
    rc = idp.lib().idp_integrals_noalloc(C.c_void_p(8), C.c_void_p(8), idp.NOALLOC_MAX_ELEMS + 1, 3,
                                         C.c_void_p(8), 1, C.c_void_p(8), None)
    assert rc == idp.IDP_E_ARG
