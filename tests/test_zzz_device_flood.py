"""The builder's flooding inspection (Alg. 1) on the device
(device_assist=2): each warp floods one primitive at a time with the steps
of the core the host builder uses, in double precision without fused
multiply-adds, and hands back the primitives its shared-memory buffers
cannot hold.  With device_assist=3 the Voronoi cells are made on the device
too (one thread per cell, cell_core.h).  The layouts they build are the
host's byte for byte: the builds are saved and the files compared (they
hold every table, box code, neighbour list, the inspection count and the
certification's counts)."""
import os
import tempfile

import numpy as np
import pytest

import datagen as dg
from tests import parity_util as pu
from tests.table_util import check_tables_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_16084_gb300 as m
    return m


CASES = {
    "sphere-L3": lambda: dg.workload(0, n_queries=10),
    "displaced-L4": lambda: dg.workload(1, n_queries=10, level=4),
    "heightfield-40": lambda: dg.workload(2, n_queries=10, grid=40),
    "soup-penetrating-L3": lambda: dg.soup_workload("penetrating", level=3, n_queries=10),
    "mixed-L2-wire-L1": lambda: dg.mixed_workload(mesh_level=2, wire_level=1, n_queries=10),
    "fan-120": lambda: dg.high_valence_fan(120),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_device_flood_builds_the_host_layout(pg, name):
    m = CASES[name]()
    kw = dict(segs=m.meta.get("segs"), domain_scale=m.domain_scale,
              domain_margin=m.domain_margin)
    a = pg.P2M(m.verts, m.tris, device_assist=2, **kw)
    b = pg.P2M(m.verts, m.tris, device_assist=1, **kw)
    fa, fb = a.flood_stats(), b.flood_stats()
    assert fa["device"] > 0 and fb["device"] == 0
    assert sum(fa.values()) == sum(fb.values())
    if name.startswith("fan"):
        # the apex's cell does not fit the core's buffers: handed back
        assert fa["host_unbounded"] > 0
    assert a.stats()["inspections"] == b.stats()["inspections"]
    c = pg.P2M(m.verts, m.tris, device_assist=3, **kw)
    cs = c.cell_stats()
    assert cs["device"] > 0 and cs["device"] + cs["host"] == m.verts.shape[0]
    assert cs["packed_on_device"] == 1
    assert a.cell_stats() == b.cell_stats() == {"device": 0, "host": m.verts.shape[0],
                                                "packed_on_device": 0}
    with tempfile.TemporaryDirectory() as d:
        pa, pb, pc = (os.path.join(d, f"{x}.p2m") for x in "abc")
        a.save(pa)
        b.save(pb)
        c.save(pc)
        ba, bb, bc = (open(x, "rb").read() for x in (pa, pb, pc))
    assert len(ba) == len(bb) == len(bc)
    assert ba == bb
    assert bc == bb


@pytest.mark.parametrize("name", ["sphere-L3", "displaced-L4", "heightfield-40",
                                  "soup-penetrating-L3", "mixed-L2-wire-L1"])
def test_device_flood_tables_equal_the_oracle_and_queries_match_bruteforce(pg, name):
    """The device-flooded build against the oracle directly: the same
    interception lists with boxes containing the oracle's, and queries on
    it matching the FP64 brute force."""
    import torch
    m = CASES[name]()
    a = pg.P2M(m.verts, m.tris, device_assist=2, segs=m.meta.get("segs"),
               domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    assert a.flood_stats()["device"] > 0
    o = check_tables_against_oracle(a, m, same_neighbour_count=False)
    rng = np.random.default_rng(31)
    v64 = m.verts.astype(np.float64)
    q = np.concatenate([dg.uniform_in_box(v64, 1.2, 20000, rng),
                        v64[rng.integers(0, v64.shape[0], 5001)] +
                        rng.normal(0, 0.01 * dg.bbox_diagonal(v64), (5001, 3))]).astype(np.float32)
    r = a.query(torch.from_numpy(q).cuda(), closest=True, prim_type=True)
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in r.items()}
    ref = o.bruteforce(q)
    pu.check(m.verts, o.edges(), m.tris, q, gpu, ref, pu.tolerance(m.verts), f"device flood {name}")
