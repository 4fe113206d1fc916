"""The C ABI library on the CPU: it loads, exports every entry point that
include/p2m.h declares, validates meshes, and its host builder produces the
same interception table as the oracle (two independent implementations of
Alg. A.1).  No compute call needs a GPU here."""
import ctypes
import os
import re
import tempfile

import numpy as np
import pytest

import datagen as dg
import oracle
from tests.table_util import check_tables_against_oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2308_16084_gb300 as m
    return m


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "p2m.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(p2m_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(pg):
    lib = ctypes.CDLL(pg.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    from paper_2308_16084_gb300 import _lib
    assert set(names) == set(_lib.EXPORTED)


def test_status_strings(pg):
    for code in range(10):
        s = pg.lib.p2m_status_string(code)
        assert s and s != b"unknown status"


def _host(pg, m, **kw):
    return pg.P2M(m.verts, m.tris, segs=m.meta.get("segs"), domain_scale=m.domain_scale,
                  domain_margin=m.domain_margin, device_assist=False, **kw)


@pytest.mark.parametrize("idx,kw", [(0, {}), (1, {"level": 4}), (2, {"grid": 40}),
                                    (3, {"level": 4})])
def test_builder_tables_equal_oracle_tables(pg, idx, kw):
    _check_tables(pg, dg.workload(idx, n_queries=10, **kw))


@pytest.mark.parametrize("kind", ["gapped", "penetrating"])
def test_builder_tables_equal_oracle_tables_on_soups(pg, kind):
    """Triangle soups: every face with its own vertices, apart or cutting
    through each other (all edges are boundary edges)."""
    _check_tables(pg, dg.soup_workload(kind, level=2, n_queries=10))


def test_builder_tables_equal_oracle_tables_on_mixed_input(pg):
    """A triangle mesh beside a wireframe (segments of no face), and the
    wireframe alone."""
    m = dg.mixed_workload(mesh_level=2, wire_level=1, n_queries=10)
    _check_tables(pg, m)
    S = m.meta["segs"]
    used = np.unique(S)
    remap = np.full(m.verts.shape[0], -1, np.int64)
    remap[used] = np.arange(used.size)
    wire = dg.Mesh("wire", m.verts[used], np.zeros((0, 3), np.int32), m.queries,
                   m.domain_scale, m.domain_margin, meta={"segs": remap[S].astype(np.int32)})
    _check_tables(pg, wire)


@pytest.mark.parametrize("seed", range(8))
def test_builder_tables_equal_oracle_tables_on_random_inputs(pg, seed):
    """Seeded random inputs beyond the workloads: a soup of random triangles
    in a box (some cutting through each other), plus random segments on
    half of the seeds."""
    rng = np.random.default_rng(1000 + seed)
    nt = int(rng.integers(8, 40))
    c = rng.uniform(-1, 1, size=(nt, 1, 3))
    tri = c + rng.uniform(-0.35, 0.35, size=(nt, 3, 3))
    V = tri.reshape(-1, 3)
    F = np.arange(3 * nt, dtype=np.int32).reshape(-1, 3)
    segs = None
    if seed % 2:
        ns = int(rng.integers(3, 12))
        a = rng.uniform(-1, 1, size=(ns, 3))
        b = a + rng.uniform(-0.4, 0.4, size=(ns, 3))
        base = V.shape[0]
        V = np.concatenate([V, a, b], 0)
        segs = np.stack([base + np.arange(ns), base + ns + np.arange(ns)], 1).astype(np.int32)
    m = dg.Mesh(f"random-{seed}", V.astype(np.float32), F, np.zeros((1, 3), np.float32),
                1.25, 0.05, meta={} if segs is None else {"segs": segs})
    _check_tables(pg, m)


def test_builder_tables_equal_oracle_tables_on_a_high_valence_fan(pg):
    """A vertex whose Voronoi cell has ~122 faces: the primitives that reach
    it overflow the bounded flooding core's buffers and are flooded by the
    unbounded host code; the rest stay on the core.  The table is the
    oracle's either way."""
    m = dg.high_valence_fan(120)
    _check_tables(pg, m)
    fs = _host(pg, m).flood_stats()
    assert fs["device"] == 0
    assert fs["host_bounded"] > 0 and fs["host_unbounded"] > 0
    assert fs["host_bounded"] + fs["host_unbounded"] == 3 * 120


def test_flood_stats_on_a_regular_mesh(pg):
    """Every edge and face of a regular mesh is flooded by the bounded core
    (nothing overflows it), and a host-only build floods nothing on the
    device."""
    m = dg.workload(0, n_queries=10)
    st = _host(pg, m).flood_stats()
    assert st == {"device": 0, "host_bounded": 1920 + 1280, "host_unbounded": 0}


def test_device_assist_values(pg):
    V, F = dg.octahedron()
    for bad in (-1, 4):
        with pytest.raises(ValueError):
            pg.P2M(V.astype(np.float32), F, device_assist=bad)


def test_invalid_segments_return_status(pg):
    V, F = dg.octahedron()
    for segs in ([[0, 0]], [[0, 99]]):
        with pytest.raises(pg.P2MError) as e:
            pg.P2M(V.astype(np.float32), F, segs=segs, device_assist=False)
        assert e.value.code == 2


def _check_tables(pg, m):
    check_tables_against_oracle(_host(pg, m), m)


def test_builder_thread_count_does_not_change_tables(pg):
    m = dg.workload(3, n_queries=10, level=3)
    a = _host(pg, m, host_threads=1)
    b = _host(pg, m, host_threads=5)
    for v in range(0, a.n_verts, 3):
        ta, ia, ba = a.interception_list(v)
        tb, ib, bb = b.interception_list(v)
        np.testing.assert_array_equal(ta, tb)
        np.testing.assert_array_equal(ia, ib)
        np.testing.assert_array_equal(ba, bb)


@pytest.mark.parametrize("case,code", [("index", 2), ("repeat", 2), ("dup", 3), ("unref", 2),
                                       ("nan", 2), ("empty", 2)])
def test_invalid_meshes_return_status(pg, case, code):
    V, F = dg.octahedron()
    V = V.astype(np.float32)
    F = F.astype(np.int32)
    if case == "index":
        F = F.copy(); F[0, 0] = 99
    elif case == "repeat":
        F = F.copy(); F[0, 1] = F[0, 0]
    elif case == "dup":
        V = np.concatenate([V, V[:1]]); F = np.concatenate([F, [[6, 2, 4]]]).astype(np.int32)
    elif case == "unref":
        V = np.concatenate([V, [[5, 5, 5]]]).astype(np.float32)
    elif case == "nan":
        V = V.copy(); V[0, 0] = np.nan
    elif case == "empty":
        F = np.zeros((0, 3), np.int32)
    with pytest.raises(pg.P2MError) as e:
        pg.P2M(V, F, device_assist=False)
    assert e.value.code == code


def test_domain_beyond_float32_squares_is_too_large(pg):
    """A coordinate (or a domain scale) that puts D beyond +-1e18, where the
    device's float32 squared distances would overflow, is refused with
    P2M_ERR_TOO_LARGE before anything is built."""
    V, F = dg.octahedron()
    V = V.astype(np.float32)
    F = F.astype(np.int32)
    for W, kw in ((np.where(np.arange(18).reshape(6, 3) == 0, 3e38, V).astype(np.float32), {}),
                  (V, {"domain_scale": 1e19})):
        with pytest.raises(pg.P2MError) as e:
            pg.P2M(W, F, device_assist=False, **kw)
        assert e.value.code == 9
    pg.P2M(V * np.float32(1e15), F, device_assist=False, domain_scale=10.0)  # within the limit


def test_bad_options_rejected(pg):
    V, F = dg.octahedron()
    for kw in ({"domain_scale": 0.0}, {"leaf_size": 1}, {"leaf_size": 64}, {"delta_rel": -1.0}):
        with pytest.raises(pg.P2MError) as e:
            pg.P2M(V.astype(np.float32), F.astype(np.int32), device_assist=False, **kw)
        assert e.value.code == 1


def test_save_load_roundtrip_and_corruption(pg):
    m = dg.workload(0, n_queries=10, level=2)
    h = _host(pg, m)
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "m.p2m")
        h.save(p)
        g = pg.P2M.load(p)
        assert g.stats()["n_entries"] == h.stats()["n_entries"]
        for v in range(h.n_verts):
            for x, y in zip(h.interception_list(v), g.interception_list(v)):
                np.testing.assert_array_equal(x, y)
        raw = bytearray(open(p, "rb").read())
        for pos in (3, 100, len(raw) // 2, len(raw) - 3):
            bad = bytearray(raw)
            bad[pos] ^= 0x5A
            open(p, "wb").write(bad)
            with pytest.raises(pg.P2MError) as e:
                pg.P2M.load(p)
            assert e.value.code == 7
        open(p, "wb").write(raw[: len(raw) // 3])
        with pytest.raises(pg.P2MError):
            pg.P2M.load(p)
    with pytest.raises(pg.P2MError):
        pg.P2M.load("/nonexistent/file.p2m")


def test_queries_on_host_only_handle_fail_loudly(pg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = dg.workload(0, n_queries=10, level=1)
    h = _host(pg, m)
    n = 4
    dist = np.zeros(n, np.float32)
    pid = np.zeros(n, np.int32)
    with pytest.raises(pg.P2MError) as e:
        h.query_host(np.zeros((n, 3), np.float32), dist, pid)
    assert e.value.code == 8
    with pytest.raises(pg.P2MError) as e:
        h.pipeline(n)
    assert e.value.code == 8
    # moving the vertices needs the device layout too (checked through the
    # C ABI: the pointer is never read when the handle has no device)
    v = np.zeros((h.n_verts, 3), np.float32)
    assert pg.lib.p2m_update_vertices(h._h, ctypes.c_void_p(v.ctypes.data), h.n_verts, 0,
                                      None) == 8


def test_tuning_fields_are_validated(pg):
    """Every p2m_tuning field is range-checked; a rejected setting leaves the
    previous one in place."""
    m = dg.workload(0, n_queries=10, level=1)
    h = _host(pg, m)
    base = h.tuning
    assert set(base) == {"sort_bits", "block_threads", "warp_cooperative", "nn_walk",
                         "chunked", "group_by_vertex", "sort_key", "lanes_per_query",
                         "streams"}
    h.tuning = {"sort_key": 1, "block_threads": 128, "sort_bits": 12}
    assert h.tuning["sort_key"] == 1 and h.tuning["block_threads"] == 128
    for bad in ({"sort_key": 2}, {"group_by_vertex": 3}, {"chunked": 3}, {"nn_walk": -1},
                {"block_threads": 96}, {"sort_bits": 25}, {"warp_cooperative": 2},
                {"lanes_per_query": 3}, {"lanes_per_query": 16}, {"lanes_per_query": 0},
                {"streams": 0}, {"streams": 5}):
        with pytest.raises(pg.P2MError) as e:
            h.tuning = bad
        assert e.value.code == 1
        assert h.tuning["sort_key"] == 1 and h.tuning["block_threads"] == 128


@pytest.mark.parametrize("name", ["sphere", "soup", "mixed", "fan"])
def test_both_host_flooding_paths_build_the_same_layout(pg, name, monkeypatch, tmp_path):
    """The bounded flooding core (shared with the device) and the unbounded
    host code it hands overflowing primitives to compute the same records:
    forcing every primitive through the unbounded code
    (P2M_FLOOD_UNBOUNDED=1) saves the same layout file byte for byte."""
    m = {"sphere": lambda: dg.workload(3, n_queries=10, level=3),
         "soup": lambda: dg.soup_workload("penetrating", level=2, n_queries=10),
         "mixed": lambda: dg.mixed_workload(mesh_level=2, wire_level=1, n_queries=10),
         "fan": lambda: dg.high_valence_fan(120)}[name]()
    a = _host(pg, m)
    monkeypatch.setenv("P2M_FLOOD_UNBOUNDED", "1")
    b = _host(pg, m)
    fa, fb = a.flood_stats(), b.flood_stats()
    assert fb["host_bounded"] == 0
    assert fa["host_bounded"] + fa["host_unbounded"] == fb["host_unbounded"]
    a.save(str(tmp_path / "a.p2m"))
    b.save(str(tmp_path / "b.p2m"))
    assert (tmp_path / "a.p2m").read_bytes() == (tmp_path / "b.p2m").read_bytes()


def _tiny(name):
    """Edge cases of the flooding: one triangle, one segment, two triangles
    far apart, a zero-area face beside a good one (not flooded)."""
    V, F, S = {
        "one-triangle": ([[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]], None),
        "one-segment": ([[0, 0, 0], [1, 0.2, 0.1]], [], [[0, 1]]),
        "two-triangles-apart": ([[0, 0, 0], [1, 0, 0], [0, 1, 0], [3, 3, 3], [4, 3, 3],
                                 [3, 4, 3.5]], [[0, 1, 2], [3, 4, 5]], None),
        "zero-area-face": ([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0]],
                           [[0, 1, 2], [0, 1, 3]], None),
    }[name]
    return dg.Mesh(name, np.array(V, np.float32), np.array(F, np.int32).reshape(-1, 3),
                   np.zeros((1, 3), np.float32), 1.5, 0.1,
                   meta={} if S is None else {"segs": np.array(S, np.int32)})


@pytest.mark.parametrize("name", ["one-triangle", "one-segment", "two-triangles-apart",
                                  "zero-area-face"])
def test_builder_tables_equal_oracle_tables_on_tiny_inputs(pg, name):
    _check_tables(pg, _tiny(name))


@pytest.mark.parametrize("name", ["sphere", "soup", "mixed", "fan", "lat-long",
                                  "one-triangle", "one-segment", "zero-area-face"])
def test_device_flooding_algorithm_on_the_host_builds_the_same_layout(pg, name, monkeypatch,
                                                                      tmp_path):
    """The device kernel's warp algorithm (flood_warp.h: one point or face
    per lane, loops placed by prefix sums, cap chained by lane 0), run on the
    host with its 32 lanes one after another (P2M_FLOOD_LANES=1), builds the
    default layout byte for byte, handing what overflows its shared-memory
    buffers to the bounded core and the unbounded code."""
    m = {"sphere": lambda: dg.workload(3, n_queries=10, level=3),
         "soup": lambda: dg.soup_workload("penetrating", level=3, n_queries=10),
         "mixed": lambda: dg.mixed_workload(mesh_level=2, wire_level=1, n_queries=10),
         "fan": lambda: dg.high_valence_fan(120),
         "lat-long": lambda: dg.triangulation_pair(10)[1]}.get(name, lambda: _tiny(name))()
    a = _host(pg, m)
    monkeypatch.setenv("P2M_FLOOD_LANES", "1")
    b = _host(pg, m)
    assert sum(a.flood_stats().values()) == sum(b.flood_stats().values())
    a.save(str(tmp_path / "a.p2m"))
    b.save(str(tmp_path / "b.p2m"))
    assert (tmp_path / "a.p2m").read_bytes() == (tmp_path / "b.p2m").read_bytes()


def test_device_flooding_requested_without_a_gpu(pg):
    """device_assist=2 and 3 on a machine without a GPU build on the host
    (the same layout), and a loaded handle reports no flooding split."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = dg.workload(0, n_queries=10)
    a = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin,
               device_assist=2)
    b = _host(pg, m)
    assert a.flood_stats() == b.flood_stats()
    assert a.flood_stats()["device"] == 0
    c = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin,
               device_assist=3)
    assert c.cell_stats() == {"device": 0, "host": m.verts.shape[0], "packed_on_device": 0}
    assert c.flood_stats() == b.flood_stats()
    with tempfile.TemporaryDirectory() as d:
        pa, pb = os.path.join(d, "a.p2m"), os.path.join(d, "b.p2m")
        a.save(pa)
        b.save(pb)
        assert open(pa, "rb").read() == open(pb, "rb").read()
        c = pg.P2M.load(pa)
        assert c.flood_stats() == {"device": 0, "host_bounded": 0, "host_unbounded": 0}
        assert c.stats()["n_entries"] == a.stats()["n_entries"]


def test_builder_spherical_surface_every_vertex_intercepts_every_face(pg):
    """Sec. 6: on a spherical surface each vertex intercepts every triangle
    (tests/golden/spherical_surface_intercepts.txt); the product builder's
    lists hold every face."""
    path = os.path.join(ROOT, "tests", "golden", "spherical_surface_intercepts.txt")
    gens = {"icosphere(0)": lambda: dg.icosphere(0), "icosphere(1)": lambda: dg.icosphere(1),
            "octahedron()": dg.octahedron}
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for name, gen, nv, nf, per in rows:
        V, F = gens[gen]()
        h = pg.P2M(V.astype(np.float32), F.astype(np.int32), device_assist=False)
        assert (h.n_verts, h.n_tris) == (int(nv), int(nf))
        for v in range(h.n_verts):
            t, i, _ = h.interception_list(v)
            assert set(i[t == 2].tolist()) == set(range(int(per))), (name, v)


def test_build_options_and_stats_at_the_c_abi(pg):
    """Through the C ABI itself: device_assist outside 0..3 is INVALID_ARG,
    and the statistics calls reject NULL handles and outputs."""
    V, F = dg.octahedron()
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    desc = pg.MeshDesc(V.ctypes.data, V.shape[0], F.ctypes.data, F.shape[0])
    h = ctypes.c_void_p()
    for bad in (-1, 4, 7):
        opts = pg.BuildOpts(10.0, 0.0, 4e-6, 0, bad, 8)
        assert pg.lib.p2m_build(ctypes.byref(desc), ctypes.byref(opts), ctypes.byref(h)) == 1
    out = (ctypes.c_int64 * 16)()
    assert pg.lib.p2m_flood_stats(None, out) == 1
    assert pg.lib.p2m_cell_stats(None, out) == 1
    assert pg.lib.p2m_stats(None, out) == 1
    m = _host(pg, dg.workload(0, n_queries=10, level=1))
    assert pg.lib.p2m_flood_stats(m._h, None) == 1
    assert pg.lib.p2m_flood_stats(m._h, out) == 0
    assert list(out[:3]) == [0, m.flood_stats()["host_bounded"], 0]
    assert pg.lib.p2m_cell_stats(m._h, None) == 1
    # every cell of the 42 vertices, packed on the host
    assert m.cell_stats() == {"device": 0, "host": 42, "packed_on_device": 0}


@pytest.mark.parametrize("stage", ["cells", "flooding", "packing"])
@pytest.mark.parametrize("threads", [1, 4])
def test_out_of_memory_in_a_build_stage_is_reported(pg, stage, threads, monkeypatch):
    """Host-side fault injection (P2M_INJECT_BAD_ALLOC=<stage>): an
    allocation failure in a worker of a build stage comes back as
    P2M_ERR_OOM, not a crash, and the next build is whole."""
    m = dg.workload(2, n_queries=10, grid=40)
    monkeypatch.setenv("P2M_INJECT_BAD_ALLOC", stage)
    with pytest.raises(pg.P2MError) as e:
        _host(pg, m, host_threads=threads)
    assert e.value.code == 4
    monkeypatch.delenv("P2M_INJECT_BAD_ALLOC")
    _check_tables(pg, m)


_LAYOUT_ARRAYS = ["kd_nodes", "kd_points", "pos_of_vertex", "row_off", "entries", "edge_rec",
                  "face_rec", "edges", "tris", "nb_off", "nb", "chunk_off", "chunks", "nbp",
                  "super_off", "supers"]


def _layout_arrays(raw):
    """Offsets of the arrays of a saved layout: a 184-byte header (magic,
    version, 12 int64 scalars, 19 floats), then per array a uint64 count and
    that many 4-byte elements, then the FNV-1a checksum of everything after
    the version."""
    pos, out = 184, {}
    for name in _LAYOUT_ARRAYS:
        n = int(np.frombuffer(bytes(raw[pos:pos + 8]), np.uint64)[0])
        out[name] = (pos + 8, n)
        pos += 8 + 4 * n
    assert pos == len(raw) - 8
    return out


def _reseal(raw):
    h = 1469598103934665603
    for c in bytes(raw[12:-8]):
        h = ((h ^ c) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    raw[-8:] = np.array([h], np.uint64).tobytes()


def test_load_refuses_inconsistent_contents_with_a_valid_checksum(pg, tmp_path):
    """p2m_load checks every index the kernels follow, not only the
    checksum: a file re-sealed after an index was set out of range is
    refused with P2M_ERR_IO; the untouched file (re-sealed the same way)
    loads."""
    m = dg.workload(0, n_queries=10, level=1)
    h = _host(pg, m)
    p = str(tmp_path / "m.p2m")
    h.save(p)
    raw = bytearray(open(p, "rb").read())
    arr = _layout_arrays(raw)
    ok = bytearray(raw)
    _reseal(ok)
    assert ok == raw
    nv, nf = h.n_verts, h.n_tris

    def u32(name, i, value):
        off, n = arr[name]
        assert 0 <= i < n
        bad = bytearray(raw)
        bad[off + 4 * i:off + 4 * i + 4] = np.array([value], np.uint32).tobytes()
        _reseal(bad)
        return bad

    cases = [u32("entries", 0, (2 << 30) | nf),          # face id past the faces
             u32("entries", 4, 3 << 30),                 # no such primitive type
             u32("row_off", 1, 10 ** 6),                 # rows out of order
             u32("nb", 0, nv), u32("nbp", 3, nv),        # neighbour past the vertices
             u32("kd_points", 3, nv),                    # tree position of no vertex
             u32("edges", 1, nv + 5), u32("tris", 2, nv),
             u32("chunk_off", 1, 0)]
    for k, bad in enumerate(cases):
        q = str(tmp_path / f"bad{k}.p2m")
        open(q, "wb").write(bad)
        with pytest.raises(pg.P2MError) as e:
            pg.P2M.load(q)
        assert e.value.code == 7, k
    q = str(tmp_path / "ok.p2m")
    open(q, "wb").write(ok)
    assert pg.P2M.load(q).stats()["n_entries"] == h.stats()["n_entries"]


def test_package_without_its_library_fails_to_import(tmp_path):
    """No fallback: a copy of the package without libp2m.so raises
    ImportError on import instead of running anything on the CPU."""
    import shutil
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_2308_16084_gb300")
    dst = tmp_path / "paper_2308_16084_gb300"
    shutil.copytree(pkg, dst, ignore=shutil.ignore_patterns("_build", "__pycache__", "*.so"))
    code = ("import sys; sys.path.insert(0, sys.argv[1])\n"
            "try:\n    import paper_2308_16084_gb300\nexcept ImportError as e:\n"
            "    print('IMPORTERROR', 'libp2m.so' in str(e)); sys.exit(0)\n"
            "print('IMPORTED'); sys.exit(1)\n")
    r = subprocess.run([sys.executable, "-c", code, str(tmp_path)], capture_output=True,
                       text=True, timeout=120, cwd=str(tmp_path))
    assert r.returncode == 0 and r.stdout.strip() == "IMPORTERROR True", r.stdout + r.stderr


def test_builder_tables_equal_oracle_tables_on_a_lat_long_sphere(pg):
    """A poorly triangulated closed surface (long thin triangles in pole
    fans): a noisy latitude-longitude sphere, closed (Euler characteristic
    2) and oriented outward, gives the oracle's tables."""
    V, F = dg.uv_sphere(6, 48, 0.05, np.random.default_rng(1234))
    assert V.shape[0] - dg.unique_edges(F).shape[0] + F.shape[0] == 2
    nrm = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    assert ((nrm * V[F].mean(1)).sum(1) > 0).all()
    q_mean, slivers = dg.triangle_quality(V, F)
    assert slivers > 0.2
    m = dg.Mesh("latlong-6x48", V.astype(np.float32), F.astype(np.int32),
                np.zeros((1, 3), np.float32), 1.25, 0.02, meta={})
    _check_tables(pg, m)


@pytest.mark.parametrize("name", ["displaced-L4", "heightfield-40", "soup", "mixed"])
def test_packed_codes_nest(pg, tmp_path, name):
    """The two-level R-tree over each interception list is conservative:
    on every axis the float32 values an entry's 15-bit code test admits (in
    its chunk's frame) lie inside those its chunk's code test admits (in the
    global frame), and a chunk's inside its super-chunk's, so a query the
    entry test admits is never skipped at a chunk or a super-chunk.  Read
    from the saved layout and decided exactly (tests/packed_codes.py)."""
    from tests import packed_codes
    m = {"displaced-L4": lambda: dg.workload(1, n_queries=10, level=4),
         "heightfield-40": lambda: dg.workload(2, n_queries=10, grid=40),
         "soup": lambda: dg.soup_workload("penetrating", level=2, n_queries=10),
         "mixed": lambda: dg.mixed_workload(mesh_level=2, wire_level=1, n_queries=10)}[name]()
    h = _host(pg, m)
    p = str(tmp_path / "m.p2m")
    h.save(p)
    arr, lo, inv = packed_codes.read_layout(p)
    assert packed_codes.check_codes_nest(arr, lo, inv) == h.stats()["n_entries"]


@pytest.mark.parametrize("name,leaf", [("displaced-L4", 8), ("heightfield-40", 3), ("soup", 32)])
def test_kd_tree_boxes_are_the_hulls_of_their_points(pg, tmp_path, name, leaf):
    """The layout's KD tree, which the nearest-vertex modes and the exact
    searches descend: leaf j of the 2^depth leaves holds tree positions
    [j nv / L, (j + 1) nv / L); internal node i (heap order) stores the boxes
    of its children 2i + 1 and 2i + 2.  Every such box is the float32 hull
    of the points below it, the root box that of all; the tree's points are
    the vertices, each once, and pos_of_vertex is the inverse order."""
    from tests import packed_codes
    m = {"displaced-L4": lambda: dg.workload(1, n_queries=10, level=4),
         "heightfield-40": lambda: dg.workload(2, n_queries=10, grid=40),
         "soup": lambda: dg.soup_workload("penetrating", level=2, n_queries=10)}[name]()
    h = _host(pg, m, leaf_size=leaf)
    p = str(tmp_path / "m.p2m")
    h.save(p)
    arr, _, _ = packed_codes.read_layout(p)
    raw = open(p, "rb").read()
    depth = int(np.frombuffer(raw[12:108], np.int64)[3])
    root = np.frombuffer(raw[108:184], np.float32)[7:13]
    nv = h.n_verts
    L = 1 << depth
    kp = arr["kd_points"].reshape(nv, 4)
    ids = kp[:, 3].view(np.int32)
    pts = kp[:, :3].view(np.float32)
    np.testing.assert_array_equal(np.sort(ids), np.arange(nv))
    np.testing.assert_array_equal(pts, np.asarray(m.verts, np.float32)[ids])
    np.testing.assert_array_equal(arr["pos_of_vertex"].view(np.int32)[ids], np.arange(nv))
    assert L <= nv and -(-nv // L) <= max(2, leaf)
    np.testing.assert_array_equal(root, np.concatenate([pts.min(0), pts.max(0)]))
    nodes = arr["kd_nodes"].view(np.float32).reshape(L - 1, 12)
    for i in range(L - 1):
        k = int(np.floor(np.log2(i + 1)))
        span = L >> (k + 1)                    # leaves under each child
        a = (i - ((1 << k) - 1)) * 2 * span    # first leaf of child 2i + 1
        for c, box in enumerate((nodes[i, :6], nodes[i, 6:])):
            lo_leaf = a + c * span
            s, e = (lo_leaf * nv) >> depth, ((lo_leaf + span) * nv) >> depth
            assert e > s
            np.testing.assert_array_equal(box, np.concatenate([pts[s:e].min(0), pts[s:e].max(0)]))
