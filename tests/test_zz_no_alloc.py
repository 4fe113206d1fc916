"""p2m_query_noalloc: the allocation-free variant of p2m_query, for callers
that must not call cudaMalloc while they run.  Called through the C ABI and
compared with p2m_query on the same inputs, on two calls in a row (the
second call reuses the static scratch the first one left behind).  This
file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import datagen as dg
from tests import parity_util as pu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_QUERIES = 1 << 20


def _call(pg, mesh, q, out):
    return pg.lib.p2m_query_noalloc(mesh._h, ctypes.c_void_p(q.data_ptr()), q.shape[0],
                                    ctypes.c_void_p(out["dist"].data_ptr()),
                                    ctypes.c_void_p(out["closest"].data_ptr()),
                                    ctypes.c_void_p(out["prim_id"].data_ptr()),
                                    ctypes.c_void_p(out["prim_type"].data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_query_on_two_calls():
    assert torch.cuda.is_available()
    import paper_2308_16084_gb300 as pg
    m = dg.workload(0, n_queries=200_000)
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    tau = pu.tolerance(m.verts)
    for call, sl in enumerate((slice(0, 200_000), slice(3, 150_004))):
        q = torch.from_numpy(np.ascontiguousarray(m.queries[sl])).cuda()
        n = q.shape[0]
        ref = mesh.query(q, closest=True, prim_type=True)
        out = {"dist": torch.full((n,), -1.0, device="cuda"),
               "closest": torch.zeros(n, 3, device="cuda"),
               "prim_id": torch.full((n,), -7, dtype=torch.int32, device="cuda"),
               "prim_type": torch.full((n,), 9, dtype=torch.uint8, device="cuda")}
        torch.cuda.synchronize()
        # the first call of the process may load this library's device code
        # (and with it the static array); from the second call on, nothing
        # the call does may change the device's free memory or torch's pool
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        assert _call(pg, mesh, q, out) == 0, f"call {call}"
        torch.cuda.synchronize()
        if call > 0:
            assert torch.cuda.mem_get_info()[0] == free0, "device memory changed"
            assert torch.cuda.memory_allocated() == alloc0
        assert (out["dist"] - ref["dist"]).abs().max().item() <= tau
        assert (out["closest"] - ref["closest"]).abs().max().item() <= tau
        assert torch.equal(out["prim_id"], ref["prim_id"])
        assert torch.equal(out["prim_type"], ref["prim_type"])


def test_noalloc_rejects_oversize_and_bad_args():
    import paper_2308_16084_gb300 as pg
    m = dg.workload(0, n_queries=16)
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    q = torch.zeros(MAX_QUERIES + 1, 3, device="cuda")
    out = {"dist": torch.empty(MAX_QUERIES + 1, device="cuda"),
           "closest": torch.empty(MAX_QUERIES + 1, 3, device="cuda"),
           "prim_id": torch.empty(MAX_QUERIES + 1, dtype=torch.int32, device="cuda"),
           "prim_type": torch.empty(MAX_QUERIES + 1, dtype=torch.uint8, device="cuda")}
    assert _call(pg, mesh, q, out) == 9  # P2M_ERR_TOO_LARGE
    assert pg.lib.p2m_query_noalloc(mesh._h, None, 4, None, None, None, None, None) == 1
    assert pg.lib.p2m_query_noalloc(None, None, 0, None, None, None, None, None) == 1
