"""Parity of the CUDA query path (through the C ABI) against the FP64 oracle.

Every case compares element by element on the same seeded inputs with the
criterion of parity_util (tau = 1e-5 x bbox diagonal).  Sizes span many
KD-tree leaves, many query tiles and a ragged tail; the full-size workloads
are checked on sampled outputs the oracle computes one by one.
"""
import os
import tempfile

import numpy as np
import pytest

import datagen as dg
import oracle
from tests import parity_util as pu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    import paper_2308_16084_gb300 as m
    return m


def run(mesh, q_np, **kw):
    q = torch.from_numpy(np.ascontiguousarray(q_np, np.float32)).cuda()
    r = mesh.query(q, closest=True, prim_type=True, status=True, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def build(pg, m, **kw):
    return pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin, **kw)


CASES = [(0, {}, None), (1, {"level": 5}, 60000), (2, {"grid": 128}, 60000),
         (3, {"level": 5}, 60000), (1, {"level": 3}, 30001)]


@pytest.mark.parametrize("idx,kw,n", CASES)
@pytest.mark.parametrize("mode", [(0, 0, 0, 0), (1, 1, 1, 0), (0, 1, 0, 0), (1, 0, 1, 1),
                                  (2, 0, 2, 1), (2, 0, 2, 0), (2, 1, 0, 0)])
def test_parity_workloads(pg, idx, kw, n, mode):
    m = dg.workload(idx, n_queries=n, **kw)
    mesh = build(pg, m)
    mesh.tuning = {"nn_walk": mode[0], "warp_cooperative": mode[1], "chunked": mode[2],
                   "group_by_vertex": mode[3]}
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    np.testing.assert_array_equal(mesh.edges(), o.edges())
    ref = o.bruteforce(m.queries)
    gpu = run(mesh, m.queries)
    tau = pu.tolerance(m.verts)
    s = pu.check(m.verts, o.edges(), m.tris, m.queries, gpu, ref, tau, f"workload {idx} {kw}")
    # the rest are float32-unresolvable ties (far queries on face/edge
    # boundaries, where the two best distances differ by ~1e-8)
    assert s["prim_exact"] > 0.98
    lo, hi, _ = mesh.domain()
    outside = ((m.queries < lo) | (m.queries > hi)).any(1)
    np.testing.assert_array_equal((gpu["status"] & 1) == 1, outside)


@pytest.mark.parametrize("idx,kw", [(1, {"level": 4}), (2, {"grid": 40})])
def test_device_assisted_build_equals_host_build(pg, idx, kw):
    """The certification of the Voronoi cells on the device (float32
    proposals, double-precision decisions) gives the host builder's tables
    bit for bit: same lists, same box codes."""
    m = dg.workload(idx, n_queries=10, **kw)
    a = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin,
               device_assist=True)
    b = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin,
               device_assist=False)
    assert a.stats()["n_entries"] == b.stats()["n_entries"]
    for v in range(0, m.verts.shape[0], 3):
        ta, ia, ba = a.interception_list(v)
        tb, ib, bb = b.interception_list(v)
        np.testing.assert_array_equal(ta, tb)
        np.testing.assert_array_equal(ia, ib)
        np.testing.assert_array_equal(ba, bb)


@pytest.mark.parametrize("kind", ["watertight", "gapped", "penetrating"])
def test_parity_triangle_soups(pg, kind):
    """The paper's soup test (Sec. 5): the same surface watertight, as a soup
    of faces apart from each other, and as a soup of faces that cut through
    each other.  Every R-tree mode and both query orders agree bit for bit."""
    m = dg.soup_workload(kind, level=3, n_queries=20001)
    mesh = build(pg, m)
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    ref = o.bruteforce(m.queries)
    gpu = run(mesh, m.queries)
    s = pu.check(m.verts, o.edges(), m.tris, m.queries, gpu, ref, pu.tolerance(m.verts),
                 m.name)
    assert s["prim_exact"] > 0.98
    for mode in ({"chunked": 0, "group_by_vertex": 0}, {"chunked": 1, "group_by_vertex": 1},
                 {"chunked": 2, "group_by_vertex": 0, "nn_walk": 0}):
        mesh.tuning = mode
        got = run(mesh, m.queries)
        for k in ("dist", "closest", "prim_id", "prim_type", "status"):
            np.testing.assert_array_equal(got[k], gpu[k])


@pytest.mark.parametrize("wire_only", [False, True])
def test_parity_mixed_primitives(pg, wire_only):
    """Mixed segments and triangles (Sec. 5): a triangle mesh beside a
    wireframe, and the wireframe alone (no faces at all)."""
    m = dg.mixed_workload(mesh_level=3, wire_level=2, n_queries=30001)
    S = m.meta["segs"]
    V, F = m.verts, m.tris
    if wire_only:
        used = np.unique(S)
        remap = np.full(V.shape[0], -1, np.int64)
        remap[used] = np.arange(used.size)
        V, F, S = V[used], np.zeros((0, 3), np.int32), remap[S].astype(np.int32)
    # the wireframe alone is smaller than the query box: widen its domain
    # and keep the queries that lie inside it
    scale = 4.0 if wire_only else m.domain_scale
    mesh = pg.P2M(V, F, segs=S, domain_scale=scale, domain_margin=m.domain_margin)
    lo, hi, _ = mesh.domain()
    q = m.queries[((m.queries >= lo) & (m.queries <= hi)).all(1)]
    assert q.shape[0] > 25000
    o = oracle.OracleMesh(V, F, segs=S, build_tables=False)
    np.testing.assert_array_equal(mesh.edges(), o.edges())
    ref = o.bruteforce(q)
    gpu = run(mesh, q)
    s = pu.check(V, o.edges(), F, q, gpu, ref, pu.tolerance(V), m.name)
    assert s["prim_exact"] > 0.98
    assert (gpu["prim_type"] == pg.EDGE).sum() > 3000
    assert not (gpu["status"] & pg.Q_OUTSIDE_DOMAIN).any()
    if wire_only:
        assert not (gpu["prim_type"] == pg.FACE).any()


@pytest.mark.parametrize("seed", range(6))
def test_parity_random_soups(pg, seed):
    """Seeded random triangle soups in a box (faces cutting through each
    other), with random segments on half of the seeds, against the oracle's
    plain definition."""
    rng = np.random.default_rng(2000 + seed)
    nt = int(rng.integers(20, 200))
    c = rng.uniform(-1, 1, size=(nt, 1, 3))
    V = (c + rng.uniform(-0.3, 0.3, size=(nt, 3, 3))).reshape(-1, 3)
    F = np.arange(3 * nt, dtype=np.int32).reshape(-1, 3)
    S = None
    if seed % 2:
        ns = int(rng.integers(5, 40))
        a = rng.uniform(-1, 1, size=(ns, 3))
        base = V.shape[0]
        V = np.concatenate([V, a, a + rng.uniform(-0.4, 0.4, size=(ns, 3))], 0)
        S = np.stack([base + np.arange(ns), base + ns + np.arange(ns)], 1).astype(np.int32)
    V = V.astype(np.float32)
    q = dg.uniform_in_box(V.astype(np.float64), 1.2, 20001, rng).astype(np.float32)
    mesh = pg.P2M(V, F, segs=S, domain_scale=1.25, domain_margin=0.05)
    o = oracle.OracleMesh(V, F, segs=S, build_tables=False)
    ref = o.bruteforce(q)
    gpu = run(mesh, q)
    s = pu.check(V, o.edges(), F, q, gpu, ref, pu.tolerance(V), f"random soup {seed}")
    assert s["prim_exact"] > 0.98


def test_parity_against_paper_method(pg):
    """The GPU agrees with the oracle's own P2M query (Alg. A.2) too, and the
    product builder's interception lists equal the oracle's."""
    m = dg.workload(3, n_queries=40000, level=4)
    mesh = build(pg, m)
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    ref = o.query(m.queries, use_boxes=True)
    ref["second"] = o.bruteforce(m.queries)["second"]
    gpu = run(mesh, m.queries)
    pu.check(m.verts, o.edges(), m.tris, m.queries, gpu, ref, pu.tolerance(m.verts), "P2M")
    off, tt, ii, _ = o.table()
    for v in range(0, o.nv, 7):
        t, i, _ = mesh.interception_list(v)
        assert set(zip(t.tolist(), i.tolist())) == \
            set(zip(tt[off[v]:off[v + 1]].tolist(), ii[off[v]:off[v + 1]].tolist()))


@pytest.mark.parametrize("bits", [0, 12, 24])
@pytest.mark.parametrize("threads", [64, 512])
@pytest.mark.parametrize("warp", [0, 1])
@pytest.mark.parametrize("walk", [0, 1, 2])
@pytest.mark.parametrize("chunked", [0, 1, 2])
@pytest.mark.parametrize("group", [0, 1])
def test_tunings_give_identical_results(pg, bits, threads, warp, walk, chunked, group):
    m = dg.workload(0, n_queries=50001)
    mesh = build(pg, m)
    base = run(mesh, m.queries)
    mesh.tuning = {"sort_bits": bits, "block_threads": threads, "warp_cooperative": warp,
                   "nn_walk": walk, "chunked": chunked, "group_by_vertex": group}
    got = run(mesh, m.queries)
    for k in ("dist", "closest", "prim_id", "prim_type", "status"):
        np.testing.assert_array_equal(got[k], base[k])


@pytest.mark.parametrize("streams", [2, 3, 4])
@pytest.mark.parametrize("group", [0, 1])
def test_split_query_gives_identical_results(pg, streams, group):
    """The passes after the first sort run as 2-4 concurrent ranges of the
    sorted queries on forked streams (a ragged count, so the last range is
    shorter; the one-pass path ignores the split): the outputs of one
    pipeline bit for bit, also replayed from a CUDA graph."""
    m = dg.workload(1, n_queries=(1 << 20) + 4097, level=5)
    mesh = build(pg, m)
    mesh.tuning = {"group_by_vertex": group, "streams": 1}
    q = torch.from_numpy(m.queries).cuda()
    base = mesh.query(q, closest=True, prim_type=True, save=True, status=True)
    mesh.tuning = {"streams": streams}
    assert mesh.tuning["streams"] == streams
    got = mesh.query(q, closest=True, prim_type=True, save=True, status=True)
    torch.cuda.synchronize()
    for k in base:
        assert torch.equal(got[k], base[k]), k
    mesh.reserve(q.shape[0])
    out = {k: torch.empty_like(v) for k, v in base.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        mesh.query(q, out=out)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mesh.query(q, out=out)
    for v in out.values():
        v.zero_()
    g.replay()
    torch.cuda.synchronize()
    for k in base:
        assert torch.equal(out[k], base[k]), k


@pytest.mark.parametrize("idx,kw", [(0, {}), (1, {"level": 6}), (2, {"grid": 96})])
@pytest.mark.parametrize("lanes", [2, 4, 8])
@pytest.mark.parametrize("chunked", [0, 1, 2])
@pytest.mark.parametrize("threads", [64, 512])
def test_lanes_per_query_give_identical_results(pg, idx, kw, lanes, chunked, threads):
    """Splitting each query's list over 2, 4 or 8 lanes (the threads-per-
    query axis of the autotuner) changes the order of work, not one bit of
    the outputs; a ragged query count leaves a partial group at the end."""
    m = dg.workload(idx, n_queries=40003, **kw)
    mesh = build(pg, m)
    mesh.tuning = {"chunked": chunked, "block_threads": threads, "lanes_per_query": 1}
    base = run(mesh, m.queries)
    mesh.tuning = {"lanes_per_query": lanes}
    assert mesh.tuning["lanes_per_query"] == lanes
    got = run(mesh, m.queries)
    for k in ("dist", "closest", "prim_id", "prim_type", "status"):
        np.testing.assert_array_equal(got[k], base[k])
    r = mesh.query(torch.from_numpy(m.queries).cuda(), closest=True, prim_type=True, save=True)
    mesh.tuning = {"lanes_per_query": 1}
    r1 = mesh.query(torch.from_numpy(m.queries).cuda(), closest=True, prim_type=True, save=True)
    assert torch.equal(r["save"], r1["save"])


@pytest.mark.parametrize("idx,kw", [(0, {}), (2, {"grid": 96}), (1, {"level": 5})])
@pytest.mark.parametrize("threads", [64, 256])
@pytest.mark.parametrize("chunked", [0, 2])
def test_seed_vertex_sort_gives_identical_results(pg, idx, kw, threads, chunked):
    """Sorting the queries by their seed-grid vertex instead of their Morton
    bucket changes the order of work, not the results."""
    m = dg.workload(idx, n_queries=50001, **kw)
    mesh = build(pg, m)
    mesh.tuning = {"chunked": chunked, "block_threads": threads}
    base = run(mesh, m.queries)
    mesh.tuning = {"sort_key": 1}
    assert mesh.tuning["sort_key"] == 1
    got = run(mesh, m.queries)
    for k in ("dist", "closest", "prim_id", "prim_type", "status"):
        np.testing.assert_array_equal(got[k], base[k])


def test_edge_cases(pg):
    m = dg.workload(0, n_queries=10)
    mesh = build(pg, m)
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    tau = pu.tolerance(m.verts)
    # empty
    q0 = torch.zeros(0, 3, device="cuda")
    r0 = mesh.query(q0)
    assert r0["dist"].numel() == 0
    # single, ragged, exact vertex, exact edge midpoint, far away
    V = m.verts.astype(np.float64)
    E = o.edges()
    special = np.concatenate([
        m.verts[:5],
        (0.5 * (V[E[:5, 0]] + V[E[:5, 1]])).astype(np.float32),
        np.array([[50, 50, 50], [-3, 0.1, 0.2]], np.float32)])
    for q in (special[:1], special, np.repeat(special, 37, 0)[:257]):
        gpu = run(mesh, q)
        ref = o.bruteforce(q)
        # the edge midpoints lie on the shared boundary of an open edge and
        # its open faces by construction: every one of them may come back as
        # a boundary mismatch (its reported primitive is still checked)
        pu.check(m.verts, E, m.tris, q, gpu, ref, tau, "special", boundary_frac=1.0)
    gpu = run(mesh, special)
    assert (gpu["dist"][:5] == 0).all() and (gpu["prim_type"][:5] == pg.VERTEX).all()
    np.testing.assert_array_equal(gpu["prim_id"][:5], np.arange(5))
    assert (gpu["status"][-2] & pg.Q_OUTSIDE_DOMAIN)
    # non-finite inputs: NaN outputs, id -1, status bit
    bad = np.array([[np.nan, 0, 0], [0, np.inf, 0], [0.1, 0.2, 0.3]], np.float32)
    gpu = run(mesh, bad)
    assert np.isnan(gpu["dist"][:2]).all() and (gpu["prim_id"][:2] == -1).all()
    assert (gpu["status"][:2] & pg.Q_NONFINITE).all() and np.isfinite(gpu["dist"][2])


def test_size_limits_rejected_before_any_work(pg):
    """Counts at the 2^31 limit (and negative ones) come back as status codes
    from the argument checks, before any allocation or launch; the small
    buffers passed are never touched."""
    import ctypes
    m = dg.workload(0, n_queries=10)
    mesh = build(pg, m)
    buf = torch.zeros(16, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    big = 1 << 31
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = pg.lib
    assert lib.p2m_query(mesh._h, ptr, big, ptr, None, ptr, None, None, None, st) == 9
    assert lib.p2m_query(mesh._h, ptr, -1, ptr, None, ptr, None, None, None, st) == 1
    assert lib.p2m_nearest_vertex(mesh._h, ptr, big, ptr, st) == 9
    assert lib.p2m_reserve(mesh._h, big) == 9
    out = (ctypes.c_int64 * 6)()
    assert lib.p2m_query_counters(mesh._h, ptr, big, out, st) == 9
    torch.cuda.synchronize()
    assert (buf == 0).all()


def test_determinism_and_save_load(pg):
    m = dg.workload(2, n_queries=40000, grid=64)
    mesh = build(pg, m)
    a = run(mesh, m.queries)
    b = run(mesh, m.queries)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mesh.p2m")
        mesh.save(path)
        mesh2 = pg.P2M.load(path)
        c = run(mesh2, m.queries)
        for k in a:
            np.testing.assert_array_equal(a[k], c[k])
        with open(path, "r+b") as f:
            f.seek(200)
            byte = f.read(1)
            f.seek(200)
            f.write(bytes([byte[0] ^ 0xFF]))
        with pytest.raises(pg.P2MError, match="I/O"):
            pg.P2M.load(path)


def test_host_api_matches_device_api(pg):
    m = dg.workload(0, n_queries=30000)
    mesh = build(pg, m)
    dev = run(mesh, m.queries)
    n = m.queries.shape[0]
    dist = np.zeros(n, np.float32)
    pid = np.zeros(n, np.int32)
    cp = np.zeros((n, 3), np.float32)
    pt = np.zeros(n, np.uint8)
    mesh.query_host(m.queries, dist, pid, cp, pt)
    np.testing.assert_array_equal(dist, dev["dist"])
    np.testing.assert_array_equal(pid, dev["prim_id"])
    np.testing.assert_array_equal(cp, dev["closest"])
    np.testing.assert_array_equal(pt, dev["prim_type"])


def test_pipeline_matches_device_api(pg):
    """Pipelined host batches (slots reused round robin, ragged sizes) give
    the same bits as the device-buffer query."""
    m = dg.workload(0, n_queries=30000)
    mesh = build(pg, m)
    batches = [m.queries, dg.workload(0, n_queries=12345).queries,
               dg.workload(0, n_queries=30000).queries[::-1].copy(), m.queries[:1]]
    pipe = mesh.pipeline(30000, depth=2)
    outs = []
    for qb in batches:
        n = qb.shape[0]
        o = {"q": torch.from_numpy(qb).pin_memory(),
             "dist": torch.empty(n).pin_memory(),
             "prim_id": torch.empty(n, dtype=torch.int32).pin_memory(),
             "closest": torch.empty(n, 3).pin_memory(),
             "prim_type": torch.empty(n, dtype=torch.uint8).pin_memory()}
        pipe.submit(o["q"], o["dist"], o["prim_id"], o["closest"], o["prim_type"])
        outs.append(o)
    pipe.wait()
    for qb, o in zip(batches, outs):
        dev = run(mesh, qb)
        for k in ("dist", "prim_id", "closest", "prim_type"):
            np.testing.assert_array_equal(o[k].numpy(), dev[k])
    big = torch.zeros(30001, 3).pin_memory()
    with pytest.raises(pg.P2MError) as e:
        pipe.submit(big, torch.empty(30001).pin_memory(),
                    torch.empty(30001, dtype=torch.int32).pin_memory())
    assert e.value.code == 9
    pipe.close()


def test_device_pipeline_matches_device_api(pg):
    """Device-buffer batches on the pipe's slots (round robin, ragged sizes,
    overlapping on their streams) give the bits of p2m_query; the launching
    stream joins them before reading."""
    m = dg.workload(1, n_queries=300_000, level=4)
    mesh = build(pg, m)
    q = torch.from_numpy(m.queries).cuda()
    pieces = [q[:300_000], q[7:123_457], q[1000:1001], q[:200_000].flip(0).contiguous()]
    pipe = mesh.pipeline(300_000, depth=3)
    outs = []
    for qb in pieces:
        o = {"dist": torch.empty(qb.shape[0], device="cuda"),
             "prim_id": torch.empty(qb.shape[0], dtype=torch.int32, device="cuda"),
             "closest": torch.empty(qb.shape[0], 3, device="cuda"),
             "prim_type": torch.empty(qb.shape[0], dtype=torch.uint8, device="cuda")}
        pipe.submit_device(qb, o)
        outs.append(o)
    pipe.join()
    for qb, o in zip(pieces, outs):
        ref = mesh.query(qb, closest=True, prim_type=True)
        for k in ("dist", "prim_id", "closest", "prim_type"):
            assert torch.equal(o[k], ref[k]), k
    pipe.wait()
    pipe.close()


# ------------------------------------------------------------------ backward

def test_backward_against_oracle_gradient(pg):
    """grad_q = w (q-c)/d and grad_v_k = -w b_k (q-c)/d (Eq. of the
    distance's derivative) against the oracle's FP64 analytic gradient."""
    m = dg.workload(3, n_queries=50000, level=5)
    mesh = build(pg, m)
    q = torch.from_numpy(m.queries).cuda().requires_grad_(True)
    verts = torch.from_numpy(m.verts).cuda().requires_grad_(True)
    w = torch.from_numpy(m.weights).cuda()
    d, pid = pg.distance(q, verts, mesh)
    (w * d).sum().backward()
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    ref = o.bruteforce(m.queries)
    gq_ref, bv, gv = oracle.gradient(m.queries.astype(np.float64), ref, m.weights.astype(np.float64))
    keep = (ref["dist"] > 1e-4) & (ref["second"] - ref["dist"] > 1e-4)
    gq = q.grad.cpu().numpy()
    gerr = np.abs(gq[keep] - gq_ref[keep]).max(1)
    assert (gerr <= pu.grad_tolerance(ref["dist"][keep], m.verts)).all(), gerr.max()
    # vertex gradient: scatter the oracle's per-query contributions of the
    # same (non-tie) queries and compare with a second GPU pass on them
    qs = torch.from_numpy(m.queries[keep]).cuda()
    ws = torch.from_numpy(m.weights[keep]).cuda()
    v2 = torch.from_numpy(m.verts).cuda().requires_grad_(True)
    d2, _ = pg.distance(qs, v2, mesh)
    (ws * d2).sum().backward()
    gv_ref = np.zeros((m.verts.shape[0], 3))
    bvk, gvk = bv[keep], gv[keep]
    for s in range(3):
        ok = bvk[:, s] >= 0
        np.add.at(gv_ref, bvk[ok, s], gvk[ok, s])
    err = np.abs(v2.grad.cpu().numpy() - gv_ref).max()
    assert err < 1e-3 * max(1.0, np.abs(gv_ref).max()), err


def test_backward_against_finite_differences(pg):
    """FP64 central differences (h = 1e-6) of the oracle's brute-force
    distance on 1k points away from ties and from d = 0."""
    m = dg.workload(3, n_queries=4000, level=4)
    mesh = build(pg, m)
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    ref = o.bruteforce(m.queries)
    keep = np.nonzero((ref["dist"] > 1e-3) & (ref["second"] - ref["dist"] > 1e-3))[0][:1000]
    qn = m.queries[keep]
    q = torch.from_numpy(qn).cuda().requires_grad_(True)
    verts = torch.from_numpy(m.verts).cuda()
    d, _ = pg.distance(q, verts, mesh)
    d.sum().backward()
    gq = q.grad.cpu().numpy()
    h = 1e-6
    q64 = qn.astype(np.float64)
    fd = np.zeros_like(q64)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd[:, k] = (o.bruteforce(q64 + e)["dist"] - o.bruteforce(q64 - e)["dist"]) / (2 * h)
    assert np.abs(gq - fd).max() < 2e-3


# ------------------------------------------------------------------- batched

def _batch_meshes(pg, n_meshes=6):
    ms = dg.batch_workload(n_meshes, tri_range=(1e3, 3e4), query_range=(1e3, 3e4))
    meshes = [build(pg, m) for m in ms]
    return ms, meshes


@pytest.mark.parametrize("group,lanes", [(1, 1), (0, 1), (1, 2), (1, 4)])
def test_batched_matches_single_and_oracle(pg, group, lanes):
    ms, meshes = _batch_meshes(pg)
    qs = [torch.from_numpy(m.queries).cuda() for m in ms]
    # a few non-finite queries in one mesh
    qs[1][:3] = torch.tensor([[float("nan"), 0, 0], [0, float("inf"), 0], [0, 0, -float("inf")]])
    b = pg.P2MBatch(meshes, qs, closest=True, prim_type=True)
    b.tuning = {"group_by_vertex": group, "lanes_per_query": lanes}
    assert b.tuning["group_by_vertex"] == group and b.tuning["lanes_per_query"] == lanes
    out = b.run()
    b.check()
    torch.cuda.synchronize()
    for m, mesh, r, q in zip(ms, meshes, out, qs):
        qn = q.cpu().numpy()
        single = run(mesh, qn)
        np.testing.assert_array_equal(r["dist"].cpu().numpy(), single["dist"])
        np.testing.assert_array_equal(r["prim_id"].cpu().numpy(), single["prim_id"])
        np.testing.assert_array_equal(r["closest"].cpu().numpy(), single["closest"])
        np.testing.assert_array_equal(r["prim_type"].cpu().numpy(), single["prim_type"])
        o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
        sel = np.arange(0, m.queries.shape[0], 5)
        sel = sel[np.isfinite(qn[sel]).all(1)]
        ref = o.bruteforce(m.queries[sel])
        got = {k: v.cpu().numpy()[sel] for k, v in r.items()}
        pu.check(m.verts, o.edges(), m.tris, m.queries[sel], got, ref, pu.tolerance(m.verts),
                 m.name)


def test_batched_autotune_and_graph_replay(pg):
    ms, meshes = _batch_meshes(pg, 4)
    qs = [torch.from_numpy(m.queries).cuda() for m in ms]
    b = pg.P2MBatch(meshes, qs)
    ref = [r["dist"].clone() for r in b.run()]
    ms_best = b.autotune(reps=2)
    assert ms_best > 0
    for r in b.out:
        r["dist"].zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    for r in b.out:
        r["dist"].zero_()
    g.replay()
    torch.cuda.synchronize()
    b.check()
    for r, d0 in zip(b.out, ref):
        assert torch.equal(r["dist"], d0)


# ------------------------------------------------------- full-size workloads

@pytest.fixture(scope="module")
def full1(pg):
    m = dg.workload(1)
    mesh = build(pg, m)
    return m, mesh


def test_full_size_displaced_sphere_sampled(pg, full1):
    """1.3M triangles, 10M queries in the launch configuration the benchmark
    times: every output obeys the invariants, 20,000 sampled outputs match
    the brute-force oracle."""
    m, mesh = full1
    q = torch.from_numpy(m.queries).cuda()
    base = mesh.query(q, closest=True, prim_type=True, save=True)
    mesh.autotune(q, reps=1)  # the benchmark's choice of launch configuration
    r = mesh.query(q, closest=True, prim_type=True, save=True)
    torch.cuda.synchronize()
    for k in base:  # the configuration changes the order of work, not the results
        assert torch.equal(base[k], r[k]), k
    d = r["dist"]
    assert torch.isfinite(d).all()
    assert torch.allclose(torch.linalg.norm(q - r["closest"], dim=1), d, atol=1e-5, rtol=1e-5)
    wts = r["save"][:, 1:]
    assert (wts >= -1e-6).all() and torch.allclose(wts.sum(1), torch.ones_like(d), atol=1e-5)
    rng = np.random.default_rng(1)
    sel = np.sort(rng.choice(m.queries.shape[0], 20000, replace=False))
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    ref = o.bruteforce(m.queries[sel])
    got = {"dist": d.cpu().numpy()[sel], "prim_id": r["prim_id"].cpu().numpy()[sel],
           "prim_type": r["prim_type"].cpu().numpy()[sel],
           "closest": r["closest"].cpu().numpy()[sel]}
    pu.check(m.verts, o.edges(), m.tris, m.queries[sel], got, ref, pu.tolerance(m.verts), "full1")
    # d <= distance to the nearest vertex (Alg. A.2 initialisation)
    nn, _ = o.kdt_nn(m.queries[sel])
    dv = np.linalg.norm(m.queries[sel].astype(np.float64) - m.verts[nn].astype(np.float64), axis=1)
    assert (got["dist"] <= dv + pu.tolerance(m.verts)).all()


def test_full_size_heightfield_sampled(pg):
    """2,093,058-triangle jittered height field with slivers, 16M queries
    Gaussian about the surface: invariants on every output, 20,000 sampled
    outputs against the brute-force oracle."""
    m = dg.workload(2)
    mesh = build(pg, m)
    q = torch.from_numpy(m.queries).cuda()
    r = mesh.query(q, closest=True, prim_type=True)
    torch.cuda.synchronize()
    d = r["dist"]
    assert torch.isfinite(d).all()
    assert torch.allclose(torch.linalg.norm(q - r["closest"], dim=1), d, atol=2e-6, rtol=1e-5)
    sel = np.sort(np.random.default_rng(2).choice(m.queries.shape[0], 20000, replace=False))
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    ref = o.bruteforce(m.queries[sel])
    got = {"dist": d.cpu().numpy()[sel], "prim_id": r["prim_id"].cpu().numpy()[sel],
           "prim_type": r["prim_type"].cpu().numpy()[sel],
           "closest": r["closest"].cpu().numpy()[sel]}
    pu.check(m.verts, o.edges(), m.tris, m.queries[sel], got, ref, pu.tolerance(m.verts), "full2")


def test_full_size_fwd_bwd_sampled(pg):
    """327,680-triangle noisy icosphere, 4M near-surface queries, loss
    sum w_i d_i: forward outputs and the query gradient of 20,000 sampled
    queries against the oracle (away from ties and d = 0), and the vertex
    gradient against the scatter of the oracle's per-query terms."""
    m = dg.workload(3)
    mesh = build(pg, m)
    q = torch.from_numpy(m.queries).cuda().requires_grad_(True)
    verts = torch.from_numpy(m.verts).cuda().requires_grad_(True)
    w = torch.from_numpy(m.weights).cuda()
    d, pid = pg.distance(q, verts, mesh)
    (w * d).sum().backward()
    torch.cuda.synchronize()
    sel = np.sort(np.random.default_rng(3).choice(m.queries.shape[0], 20000, replace=False))
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    ref = o.bruteforce(m.queries[sel])
    got = {"dist": d.detach().cpu().numpy()[sel], "prim_id": pid.cpu().numpy()[sel]}
    again = mesh.query(q.detach()[sel], closest=True, prim_type=True)
    got["prim_type"] = again["prim_type"].cpu().numpy()
    got["closest"] = again["closest"].cpu().numpy()
    pu.check(m.verts, o.edges(), m.tris, m.queries[sel], got, ref, pu.tolerance(m.verts), "full3")
    gq_ref, _, _ = oracle.gradient(m.queries[sel].astype(np.float64), ref,
                                   m.weights[sel].astype(np.float64))
    keep = (ref["dist"] > 1e-4) & (ref["second"] - ref["dist"] > 1e-4)
    gerr = np.abs(q.grad.cpu().numpy()[sel][keep] - gq_ref[keep]).max(1)
    assert (gerr <= pu.grad_tolerance(ref["dist"][keep], m.verts)).all(), gerr.max()
    g = verts.grad
    assert torch.isfinite(g).all()
    # every query's weight reaches the vertices: sum of vertex gradients
    # equals minus the sum of the query gradients (translation invariance)
    np.testing.assert_allclose(g.sum(0).cpu().numpy(), -q.grad.sum(0).cpu().numpy(),
                               rtol=2e-3, atol=2e-2)


def test_full_size_batch_sampled(pg):
    """All 64 meshes of the batch workload (about 5.2M triangles, 24M
    queries) in one persistent launch: 2,000 sampled outputs per mesh against
    the brute-force oracle, and bitwise equality with per-mesh queries."""
    ms = dg.batch_workload(64)
    meshes = [build(pg, m) for m in ms]
    qs = [torch.from_numpy(m.queries).cuda() for m in ms]
    b = pg.P2MBatch(meshes, qs, closest=True, prim_type=True)
    out = b.run()
    b.check()
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    for m, mesh, q, r in zip(ms, meshes, qs, out):
        single = mesh.query(q, closest=False, prim_type=False)
        assert torch.equal(single["dist"], r["dist"]) and torch.equal(single["prim_id"], r["prim_id"])
        sel = np.sort(rng.choice(m.queries.shape[0], min(2000, m.queries.shape[0]), replace=False))
        o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
        ref = o.bruteforce(m.queries[sel])
        got = {k: v.cpu().numpy()[sel] for k, v in r.items()}
        pu.check(m.verts, o.edges(), m.tris, m.queries[sel], got, ref, pu.tolerance(m.verts),
                 m.name)
