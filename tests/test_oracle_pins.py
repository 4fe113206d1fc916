"""Pins of the FP64 oracle against facts fixed by the paper and by plain
mathematics (closed forms, brute force, invariants, theorems).  CPU only.

Each test names the passage it pins.  None of them re-types the oracle's
own formulas: the references are closed forms, a different algorithm
(closed-triangle projection with edge clamping), dense sampling, or
brute-force enumeration.
"""
import itertools
import os
import math

import numpy as np
import pytest
from scipy.spatial import ConvexHull

import datagen as dg
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------------------
# helpers written independently of the oracle
# --------------------------------------------------------------------------

def closest_on_closed_triangles(V, F, q):
    """Distance from each q to the union of closed triangles, by projecting
    onto each triangle's plane and, when the projection falls outside,
    clamping onto the three closed edges (a different algorithm from the
    oracle's gated minimum over open primitives)."""
    V = np.asarray(V, np.float64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    best = np.full(q.shape[0], np.inf)

    def seg(p, s0, s1):
        d = s1 - s0
        t = np.clip(((p - s0) * d).sum(-1) / (d * d).sum(-1), 0.0, 1.0)
        x = s0 + t[..., None] * d
        return np.linalg.norm(p - x, axis=-1)

    for i in range(0, q.shape[0], 256):
        p = q[i:i + 256, None, :]
        n = np.cross(b - a, c - a)
        nn = n / np.linalg.norm(n, axis=1, keepdims=True)
        h = ((p - a) * nn).sum(-1)
        x = p - h[..., None] * nn
        # inside test by same-side signs of the three edge cross products
        s0 = (np.cross(b - a, x - a) * n).sum(-1)
        s1 = (np.cross(c - b, x - b) * n).sum(-1)
        s2 = (np.cross(a - c, x - c) * n).sum(-1)
        inside = (s0 >= 0) & (s1 >= 0) & (s2 >= 0)
        dplane = np.abs(h)
        dedge = np.minimum(np.minimum(seg(p, a, b), seg(p, b, c)), seg(p, c, a))
        d = np.where(inside, dplane, dedge)
        best[i:i + 256] = d.min(1)
    return best


def brute_nn(V, q):
    V = np.asarray(V, np.float64)
    out = np.empty(q.shape[0], np.int64)
    for i in range(0, q.shape[0], 512):
        d2 = ((q[i:i + 512, None, :] - V[None]) ** 2).sum(-1)
        out[i:i + 512] = d2.argmin(1)  # first minimum = lowest index on ties
    return out


def rng(seed=0):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# the plain definition (brute force) against closed forms
# --------------------------------------------------------------------------

def test_bruteforce_cube_closed_form():
    """Cube [-1,1]^3: outside d = |max(|q|-1, 0)|, inside d = 1 - max|q_i|;
    the number of coordinates beyond the cube fixes vertex/edge/face
    (Sec. 4.1: primitives are vertices, open edges, open faces)."""
    V, F = dg.cube()
    o = oracle.OracleMesh(V.astype(np.float32), F, build_tables=False)
    q = rng(1).uniform(-2.5, 2.5, size=(4000, 3))
    r = o.bruteforce(q)
    a = np.abs(q)
    outside = (a > 1).any(1)
    d_ref = np.where(outside, np.linalg.norm(np.maximum(a - 1, 0), axis=1), 1 - a.max(1))
    np.testing.assert_allclose(r["dist"], d_ref, rtol=0, atol=1e-12)
    k = (a > 1).sum(1)
    assert (r["ptype"][k == 3] == oracle.VERTEX).all()
    np.testing.assert_allclose(r["cp"][k == 3], np.sign(q[k == 3]), atol=0)
    assert (r["ptype"][k == 2] == oracle.EDGE).all()
    assert np.isin(r["ptype"][k == 1], [oracle.FACE, oracle.EDGE]).all()
    # an edge answer for k == 1 can only be a square's diagonal (a tie)
    E = o.edges()
    e1 = r["pid"][(k == 1) & (r["ptype"] == oracle.EDGE)]
    if e1.size:
        diff = np.abs(V[E[e1, 0]] - V[E[e1, 1]])
        assert ((diff > 0).sum(1) == 2).all()


def test_bruteforce_octahedron_face_regions():
    """Octahedron |x|+|y|+|z| = 1: where the projection onto the octant's
    face plane lands inside the face, d = |s.q - 1| / sqrt(3)."""
    V, F = dg.octahedron()
    o = oracle.OracleMesh(V.astype(np.float32), F, build_tables=False)
    q = rng(2).uniform(-1.5, 1.5, size=(6000, 3))
    s = np.sign(q)
    h = (s * q).sum(1) - 1.0
    p = q - (h / 3.0)[:, None] * s
    inside_face = ((s * p) > 1e-9).all(1)
    r = o.bruteforce(q)
    np.testing.assert_allclose(r["dist"][inside_face], np.abs(h[inside_face]) / math.sqrt(3),
                               rtol=0, atol=1e-12)
    assert (r["ptype"][inside_face] == oracle.FACE).all()


def test_bruteforce_sphere_bounds():
    """Unperturbed icosphere inscribed in the unit sphere with inradius
    r_in: outside |q|-1 <= d <= |q|-r_in, inside r_in-|q| <= d <= 1-|q|."""
    V, F = dg.icosphere(2)
    V32 = V.astype(np.float32)
    Vd = V32.astype(np.float64)
    n = np.cross(Vd[F[:, 1]] - Vd[F[:, 0]], Vd[F[:, 2]] - Vd[F[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    r_in = (n * Vd[F[:, 0]]).sum(1).min()
    rmax = np.linalg.norm(Vd, axis=1).max()
    o = oracle.OracleMesh(V32, F, build_tables=False)
    q = rng(3).uniform(-2, 2, size=(5000, 3))
    rq = np.linalg.norm(q, axis=1)
    d = o.bruteforce(q)["dist"]
    out = rq > rmax
    inn = rq < r_in
    tol = 1e-9
    assert (d[out] >= rq[out] - rmax - tol).all() and (d[out] <= rq[out] - r_in + tol).all()
    assert (d[inn] >= r_in - rq[inn] - tol).all() and (d[inn] <= rmax - rq[inn] + tol).all()


def test_bruteforce_matches_closed_triangle_projection():
    """Gated minimum over open primitives == distance to the union of closed
    triangles computed by projection + edge clamping (different algorithm)."""
    m = dg.workload(0, n_queries=3000, level=2)
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    q = m.queries.astype(np.float64)
    d = o.bruteforce(q)["dist"]
    ref = closest_on_closed_triangles(m.verts.astype(np.float64), m.tris, q)
    np.testing.assert_allclose(d, ref, rtol=0, atol=1e-12)


def test_bruteforce_dense_sampling():
    """Dense barycentric sampling of every triangle never beats the oracle
    and approaches it to within the sampling resolution."""
    r_ = rng(4)
    V = r_.normal(size=(9, 3)).astype(np.float32)
    F = np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8]], np.int32)
    o = oracle.OracleMesh(V, F, build_tables=False)
    q = r_.normal(size=(60, 3)) * 1.5
    d = o.bruteforce(q)["dist"]
    k = 240
    i, j = np.meshgrid(np.arange(k + 1), np.arange(k + 1), indexing="ij")
    ok = (i + j) <= k
    w1, w2 = (i[ok] / k), (j[ok] / k)
    Vd = V.astype(np.float64)
    pts = []
    for f in F:
        a, b, c = Vd[f]
        pts.append(a + w1[:, None] * (b - a) + w2[:, None] * (c - a))
    pts = np.concatenate(pts)
    ds = np.sqrt(((q[:, None, :] - pts[None]) ** 2).sum(-1)).min(1)
    edge = max(np.linalg.norm(Vd[f[0]] - Vd[f[1]]) for f in F) * 2
    assert (ds >= d - 1e-12).all()
    assert (ds - d <= edge / k * 1.5).all()


def test_closest_point_consistency():
    """The reported closest point lies at the reported distance and is the
    barycentric combination of the reported primitive's vertices."""
    m = dg.workload(0, n_queries=2000, level=2)
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    r = o.bruteforce(m.queries)
    q = m.queries.astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(q - r["cp"], axis=1), r["dist"], atol=1e-12)
    Vd = m.verts.astype(np.float64)
    bv = np.where(r["bv"] < 0, 0, r["bv"])
    recon = (r["bw"][:, :, None] * Vd[bv]).sum(1)
    np.testing.assert_allclose(recon, r["cp"], atol=1e-12)
    np.testing.assert_allclose(r["bw"].sum(1), 1.0, atol=1e-12)
    assert (r["bw"] >= 0).all()
    assert (r["second"] >= r["dist"]).all()


# --------------------------------------------------------------------------
# KD tree (Sec. 2.1)
# --------------------------------------------------------------------------

def test_kdt_nearest_equals_brute_force():
    r_ = rng(5)
    V = r_.uniform(-1, 1, size=(3000, 3)).astype(np.float32)
    F = np.stack([np.arange(0, 3000, 3), np.arange(1, 3000, 3), np.arange(2, 3000, 3)], 1)
    o = oracle.OracleMesh(V, F.astype(np.int32), build_tables=False)
    q = r_.uniform(-1.5, 1.5, size=(5000, 3))
    nn, vis = o.kdt_nn(q)
    np.testing.assert_array_equal(nn, brute_nn(V, q))
    assert vis.mean() < 200  # pruning works


def test_kdt_ties_go_to_lowest_index():
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 2], [0, 0, -2]], np.float32)
    F = np.array([[0, 2, 4], [1, 3, 5]], np.int32)
    o = oracle.OracleMesh(V, F, build_tables=False)
    nn, _ = o.kdt_nn(np.zeros((1, 3)))
    assert nn[0] == 0


def test_kdt_ties_on_a_lattice_go_to_lowest_index():
    """Equidistant vertices go to the lowest index (reading 7), where ties
    are everywhere: a shuffled 6x6x6 integer lattice, queried at every
    half-integer point of its box (cube centres tie 8 vertices, face centres
    4, edge midpoints 2; all exact in FP64), against numpy's first minimum
    over the squared distances."""
    r_ = rng(21)
    g = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    V = g[r_.permutation(len(g))].astype(np.float32)
    F = np.arange(len(V), dtype=np.int32).reshape(-1, 3)
    o = oracle.OracleMesh(V, F, build_tables=False)
    h = np.arange(0, 5.01, 0.5)
    q = np.stack(np.meshgrid(h, h, h, indexing="ij"), -1).reshape(-1, 3)
    nn, _ = o.kdt_nn(q)
    np.testing.assert_array_equal(nn, brute_nn(V, q))


def test_primitive_ties_follow_the_type_then_id_order():
    """Equidistant primitives: the paper fixes no order (Sec. 4.1 asks for
    the minimum only); the reading taken is vertex < edge < face, then the
    lower id.  Every coordinate is a dyadic rational, so each tie below is
    exact in FP64; the tied distances are confirmed with the closed-triangle
    projection, one triangle at a time."""
    q = np.array([[0.25, 0.25, 1.0]])
    base = [[0, 0, 0], [1, 0, 0], [0, 1, 0]]  # face 0, at distance 1 under q
    # vertex 3 at distance 1 above q, its triangle rising away from q
    # (its face and its edges are farther): vertex 3 before face 0
    V = np.array(base + [[0.25, 0.25, 2], [0.25, 3, 5], [3, 0.25, 5]], np.float32)
    # the open edge 3-4 passes 1 above q (closest point its midpoint), its
    # triangle rising away: that edge before face 0
    W = np.array(base + [[-1, 0.25, 2], [1.5, 0.25, 2], [0.25, 3, 5]], np.float32)
    F = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    for X in (V, W):
        for tri in F:
            assert closest_on_closed_triangles(X, tri[None], q)[0] == 1.0
    o = oracle.OracleMesh(V, F)
    for r in (o.bruteforce(q), o.query(q), o.query(q, use_boxes=True)):
        assert r["dist"][0] == 1.0 and (r["ptype"][0], r["pid"][0]) == (0, 3)
    o = oracle.OracleMesh(W, F)
    e = [list(x) for x in o.edges()].index([3, 4])
    for r in (o.bruteforce(q), o.query(q), o.query(q, use_boxes=True)):
        assert r["dist"][0] == 1.0 and (r["ptype"][0], r["pid"][0]) == (1, e)
        assert np.array_equal(r["cp"][0], [0.25, 0.25, 2.0])
    # two faces at z = +1 and z = -1 over the same corner, q midway: the
    # lower face id wins, whichever of the two triangles is listed first
    up = [[0, 0, 1], [2, 0, 1], [0, 2, 1]]
    down = [[0, 0, -1], [2, 0, -1], [0, 2, -1]]
    p = np.array([[0.5, 0.5, 0.0]])
    for first, z in ((up, 1.0), (down, -1.0)):
        X = np.array(first + (down if first is up else up), np.float32)
        o = oracle.OracleMesh(X, F)
        for r in (o.bruteforce(p), o.query(p), o.query(p, use_boxes=True)):
            assert r["dist"][0] == 1.0 and (r["ptype"][0], r["pid"][0]) == (2, 0)
            assert np.array_equal(r["cp"][0], [0.5, 0.5, z])


def test_second_best_distance_closed_form():
    """``second``, the best distance over every primitive but the reported
    one (what near-tie detection reads), in closed form: two parallel
    triangles at z = 0 and z = 1/2.  Under both, the best is face 0 at 1 and
    the second face 1 at 3/2 (listed after the best), not face 0's nearest
    edge at sqrt(5); midway between them both faces are at 1/4 (a tie: the
    second is 1/4 too).  Over face 0 alone the second is its nearest edge:
    sqrt(5) under it, sqrt(1 + 1/16) a quarter above (1, 1)."""
    V = np.array([[0, 0, 0], [8, 0, 0], [0, 8, 0],
                  [0, 0, 0.5], [8, 0, 0.5], [0, 8, 0.5]], np.float32)
    F = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    q = np.array([[2.0, 2.0, -1.0], [1.0, 1.0, 0.25]])
    r = oracle.OracleMesh(V, F, build_tables=False).bruteforce(q)
    assert np.allclose(r["dist"], [1.0, 0.25], rtol=0, atol=1e-15)
    assert (r["ptype"] == 2).all() and list(r["pid"]) == [0, 0]
    assert np.allclose(r["second"], [1.5, 0.25], rtol=0, atol=1e-15)
    V1 = V[:3]
    r = oracle.OracleMesh(V1, F[:1], build_tables=False).bruteforce(q)
    assert np.allclose(r["second"], [math.sqrt(5.0), math.sqrt(1.0 + 0.0625)], rtol=0,
                       atol=1e-15)


# --------------------------------------------------------------------------
# convex polytope cutting (Sec. 4.4 "Implementation") and Voronoi cells
# --------------------------------------------------------------------------

def _unique_rows(x, tol):
    out = []
    for p in x:
        if not any(np.linalg.norm(p - u) <= tol for u in out):
            out.append(p)
    return np.array(out).reshape(-1, 3)


def test_clipping_matches_halfspace_enumeration():
    """Corners of a box cut by random half-spaces == all feasible triple-plane
    intersections (brute-force vertex enumeration)."""
    r_ = rng(6)
    lo, hi = np.array([-1.0, -1, -1]), np.array([1.0, 1, 1])
    for trial in range(20):
        k = int(r_.integers(3, 10))
        nrm = r_.normal(size=(k, 3))
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        c = r_.uniform(0.2, 0.9, size=k)
        planes = np.concatenate([nrm, c[:, None]], 1)
        got = _unique_rows(oracle.clip_box(lo, hi, planes), 1e-9)
        allp = list(planes)
        for ax in range(3):
            for s in (-1, 1):
                n = np.zeros(3)
                n[ax] = s
                allp.append(np.array([*n, 1.0]))
        allp = np.array(allp)
        pts = []
        for i, j, l in itertools.combinations(range(allp.shape[0]), 3):
            A = allp[[i, j, l], :3]
            if abs(np.linalg.det(A)) < 1e-12:
                continue
            x = np.linalg.solve(A, allp[[i, j, l], 3])
            if (allp[:, :3] @ x - allp[:, 3] <= 1e-9).all():
                pts.append(x)
        ref = _unique_rows(np.array(pts), 1e-9)
        assert got.shape[0] == ref.shape[0], trial
        for p in ref:
            assert np.linalg.norm(got - p, axis=1).min() < 1e-9


def test_voronoi_cells_equal_all_bisector_cells():
    """Cell(v) from k-nearest seeding + corner certification == D cut by the
    bisectors of ALL other vertices (same volume, same neighbours)."""
    r_ = rng(7)
    n = 180
    V = r_.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    F = np.stack([np.arange(0, n, 3), np.arange(1, n, 3), np.arange(2, n, 3)], 1).astype(np.int32)
    o = oracle.OracleMesh(V, F, domain_scale=1.5, delta_rel=0.0)
    Vd = V.astype(np.float64)
    lo, hi = o.domain_lo, o.domain_hi
    for v in range(0, n, 9):
        w = np.array([i for i in range(n) if i != v])
        nrm = Vd[w] - Vd[v]
        ln = np.linalg.norm(nrm, axis=1)
        nrm /= ln[:, None]
        c = (nrm * (0.5 * (Vd[w] + Vd[v]))).sum(1)
        corners = oracle.clip_box(lo, hi, np.concatenate([nrm, c[:, None]], 1))
        vol = ConvexHull(corners).volume
        assert abs(vol - o.cell_volume(v)) <= 1e-9 * vol
        # neighbours: bisector planes carrying >= 3 corners of the cell
        on = np.abs(corners @ nrm.T - c[None, :]) < 1e-9
        ref = set(w[on.sum(0) >= 3].tolist())
        assert ref == set(o.cell_neighbors(v).tolist()), v
    vol_all = sum(o.cell_volume(v) for v in range(n))
    assert abs(vol_all - np.prod(hi - lo)) < 1e-9 * np.prod(hi - lo)


def test_voronoi_cells_from_delaunay_equal_all_bisector_cells():
    """Cell(v) clipped by the bisectors of its qhull Delaunay neighbours ==
    D cut by the bisectors of ALL other vertices (same volume, same
    neighbours): the construction the large-mesh oracle builds use."""
    r_ = rng(8)
    n = 180
    V = r_.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    F = np.stack([np.arange(0, n, 3), np.arange(1, n, 3), np.arange(2, n, 3)], 1).astype(np.int32)
    o = oracle.OracleMesh(V, F, domain_scale=1.5, delta_rel=0.0, voronoi="delaunay")
    Vd = V.astype(np.float64)
    lo, hi = o.domain_lo, o.domain_hi
    for v in range(0, n, 7):
        w = np.array([i for i in range(n) if i != v])
        nrm = Vd[w] - Vd[v]
        nrm /= np.linalg.norm(nrm, axis=1)[:, None]
        c = (nrm * (0.5 * (Vd[w] + Vd[v]))).sum(1)
        corners = oracle.clip_box(lo, hi, np.concatenate([nrm, c[:, None]], 1))
        vol = ConvexHull(corners).volume
        assert abs(vol - o.cell_volume(v)) <= 1e-9 * vol
        on = np.abs(corners @ nrm.T - c[None, :]) < 1e-9
        assert set(w[on.sum(0) >= 3].tolist()) == set(o.cell_neighbors(v).tolist()), v


@pytest.mark.parametrize("idx,kw", [(0, {}), (1, {"level": 4}), (2, {"grid": 40}),
                                    (3, {"level": 4})])
def test_delaunay_cells_give_the_certified_tables(idx, kw):
    """The oracle built from qhull's Delaunay neighbours has the certified
    construction's Voronoi neighbours and cell volumes, the same
    interception lists with Region boxes equal to rounding, and its Alg. A.2
    query equals the brute force bit for bit."""
    m = dg.workload(idx, n_queries=20000, **kw)
    a = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    b = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin, voronoi="delaunay")
    assert a.n_neighbor_pairs == b.n_neighbor_pairs
    for v in range(0, a.nv, 3):
        assert set(a.cell_neighbors(v).tolist()) == set(b.cell_neighbors(v).tolist()), v
        va = a.cell_volume(v)
        assert abs(va - b.cell_volume(v)) <= 1e-9 * va
    ta, tb = _table_set(a), _table_set(b)
    assert ta.keys() == tb.keys()
    diag = float(np.linalg.norm(a.domain_hi - a.domain_lo))
    worst = max(np.abs(ta[k] - tb[k]).max() for k in ta)
    assert worst <= 1e-12 * diag
    bf = b.bruteforce(m.queries)
    r = b.query(m.queries, use_boxes=True)
    np.testing.assert_array_equal(r["dist"], bf["dist"])
    np.testing.assert_array_equal(r["pid"], bf["pid"])


def test_delaunay_candidates_are_validated():
    """orc_create_ex refuses a neighbour list it cannot use: offsets that do
    not start at 0 or decrease, ids out of range, a vertex listed as its own
    neighbour, or offsets without ids."""
    import ctypes
    lib = oracle._load()
    m = dg.workload(0, n_queries=10, level=1)
    V = m.verts.astype(np.float64)
    F = np.ascontiguousarray(m.tris, np.int32)
    nv = V.shape[0]
    good_off, good_ids = oracle.delaunay_neighbors(V)

    def create(off, ids):
        st = ctypes.c_int(0)
        h = lib.orc_create_ex(V.ctypes.data, nv, F.ctypes.data, F.shape[0], None, 0, 1.25, 0.0,
                              4e-6, 1, 1, None if off is None else off.ctypes.data,
                              None if ids is None else ids.ctypes.data, ctypes.byref(st))
        if h:
            lib.orc_destroy(h)
        return st.value

    assert create(good_off, good_ids) == 0
    bad = good_off.copy()
    bad[0] = 1
    assert create(bad, good_ids) == 1
    bad = good_off.copy()
    bad[5] = bad[6] + 1
    assert create(bad, good_ids) == 1
    ids = good_ids.copy()
    ids[3] = nv
    assert create(good_off, ids) == 2
    ids = good_ids.copy()
    ids[good_off[4]] = 4
    assert create(good_off, ids) == 1
    assert create(good_off, None) == 1


def test_voronoi_volume_sum_workload0():
    m = dg.workload(0, n_queries=10)
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    tot = sum(o.cell_volume(v) for v in range(o.nv))
    D = np.prod(o.domain_hi - o.domain_lo)
    assert abs(tot - D) < 1e-9 * D


# --------------------------------------------------------------------------
# interception table: Thm. 2, Thm. 5/6 soundness, Thm. 7 completeness
# --------------------------------------------------------------------------

def _table_set(o):
    off, t, i, b = o.table()
    s = {}
    for v in range(o.nv):
        for j in range(off[v], off[v + 1]):
            s[(v, int(t[j]), int(i[j]))] = b[j]
    return s


@pytest.fixture(scope="module")
def small_meshes():
    out = {}
    m = dg.workload(0, n_queries=10)
    out["noisy-L3"] = (m.verts, m.tris, m.domain_scale, m.domain_margin)
    V, F = dg.icosphere(2)
    out["sphere-L2"] = (V.astype(np.float32), F.astype(np.int32), 1.5, 0.0)
    V, F = dg.cube()
    out["cube"] = (V.astype(np.float32), F.astype(np.int32), 3.0, 0.0)
    V, F = dg.octahedron()
    out["octahedron"] = (V.astype(np.float32), F.astype(np.int32), 3.0, 0.0)
    m = dg.workload(2, n_queries=10, grid=24)
    out["heightfield-24"] = (m.verts, m.tris, m.domain_scale, m.domain_margin)
    return out


@pytest.mark.parametrize("name", ["noisy-L3", "cube", "heightfield-24"])
def test_widened_cells_are_the_cells_pushed_out_by_delta(small_meshes, name):
    """The widened cell of v, which the flooding clips (the conservative
    relaxation by delta): D grown by delta, cut by the bisector of every
    Voronoi neighbour pushed delta away from v.  Each corner the oracle
    reports keeps every one of those constraints and lies on at least three
    of them (a corner of that polytope), checked from the positions."""
    V, F, s, mg = small_meshes[name]
    o = oracle.OracleMesh(V, F, s, mg)
    P = o.V
    lo, hi = o.domain_lo - o.delta, o.domain_hi + o.delta
    tol = 1e-9 * float(np.linalg.norm(o.domain_hi - o.domain_lo))
    for v in range(o.nv):
        X = o.cell_corners(v)
        nb = o.cell_neighbors(v)
        assert len(X) >= 4 and len(nb) >= 1
        n = P[nb] - P[v]
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        mid = 0.5 * (P[nb] + P[v])
        slack = np.concatenate([X @ n.T - (n * mid).sum(1) - o.delta, lo - X, X - hi], 1)
        assert slack.max() <= tol, (name, v)
        assert ((np.abs(slack) <= tol).sum(1) >= 3).all(), (name, v)


@pytest.mark.parametrize("name", ["noisy-L3", "sphere-L2", "cube", "octahedron", "heightfield-24"])
def test_incident_primitives_are_intercepted(small_meshes, name):
    """Thm. 2: every vertex intercepts its incident edges and faces."""
    V, F, s, mg = small_meshes[name]
    o = oracle.OracleMesh(V, F, s, mg)
    T = _table_set(o)
    E = o.edges()
    for e, (a, b) in enumerate(E):
        assert (a, oracle.EDGE, e) in T and (b, oracle.EDGE, e) in T
    for f, tri in enumerate(F):
        for v in tri:
            assert (int(v), oracle.FACE, f) in T


@pytest.mark.parametrize("name", ["noisy-L3", "sphere-L2", "cube", "octahedron", "heightfield-24"])
def test_table_complete_by_sampling(small_meshes, name):
    """Thm. 7 (flooding finds every interceptor), checked empirically: for
    sampled points of D, the brute-force closest primitive p and nearest
    vertex v satisfy p in IT[v] (or p = v), and the point lies in the
    Region box of (v, p) (Sec. 4.6)."""
    V, F, s, mg = small_meshes[name]
    o = oracle.OracleMesh(V, F, s, mg)
    T = _table_set(o)
    q = rng(8).uniform(o.domain_lo, o.domain_hi, size=(40000, 3))
    r = o.bruteforce(q)
    nn = brute_nn(V, q)
    for i in range(q.shape[0]):
        t, pid = int(r["ptype"][i]), int(r["pid"][i])
        if t == oracle.VERTEX:
            assert pid == nn[i] or abs(r["dist"][i] - np.linalg.norm(q[i] - V[nn[i]])) < 1e-12
            continue
        key = (int(nn[i]), t, pid)
        assert key in T, (name, i, key)
        b = T[key]
        assert (q[i] >= b[:3]).all() and (q[i] <= b[3:]).all(), (name, i)


def test_table_sound_against_exhaustive_filter():
    """Thm. 5/6: every flooded pair passes the convexity filter, and the
    flood never reports a pair that exhaustive inspection of all V x (E+F)
    pairs rejects."""
    m = dg.workload(0, n_queries=10, level=2)
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    T = _table_set(o)
    exhaustive = set()
    for v in range(o.nv):
        for e in range(o.ne):
            if o.intercepts(v, oracle.EDGE, e)[0]:
                exhaustive.add((v, oracle.EDGE, e))
        for f in range(o.nf):
            if o.intercepts(v, oracle.FACE, f)[0]:
                exhaustive.add((v, oracle.FACE, f))
    assert set(T.keys()) <= exhaustive
    # flooding reaches nearly every filter-accepted pair on this mesh
    assert len(T) >= 0.9 * len(exhaustive)


# --------------------------------------------------------------------------
# the query (Alg. A.2) equals the plain definition
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["noisy-L3", "sphere-L2", "cube", "octahedron", "heightfield-24"])
@pytest.mark.parametrize("use_boxes", [False, True])
def test_query_equals_bruteforce(small_meshes, name, use_boxes):
    V, F, s, mg = small_meshes[name]
    o = oracle.OracleMesh(V, F, s, mg)
    q = rng(9).uniform(o.domain_lo, o.domain_hi, size=(20000, 3)).astype(np.float32)
    bf = o.bruteforce(q)
    r = o.query(q, use_boxes=use_boxes)
    np.testing.assert_array_equal(r["dist"], bf["dist"])
    np.testing.assert_array_equal(r["ptype"], bf["ptype"])
    np.testing.assert_array_equal(r["pid"], bf["pid"])
    # invariant of Alg. A.2: d_min starts at the nearest-vertex distance
    qd = q.astype(np.float64)
    dv = np.linalg.norm(qd - V.astype(np.float64)[r["nn"]], axis=1)
    assert (r["dist"] <= dv).all()


@pytest.mark.parametrize("idx,kw", [(0, {}), (1, {"level": 4}), (2, {"grid": 48}),
                                    (3, {"level": 4})])
def test_query_equals_bruteforce_workloads(idx, kw):
    m = dg.workload(idx, n_queries=20000, **kw)
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    bf = o.bruteforce(m.queries)
    for ub in (False, True):
        r = o.query(m.queries, use_boxes=ub)
        np.testing.assert_array_equal(r["dist"], bf["dist"])
        np.testing.assert_array_equal(r["pid"], bf["pid"])


# --------------------------------------------------------------------------
# gradient against central finite differences
# --------------------------------------------------------------------------

def test_gradient_matches_finite_differences():
    """dd/dq = (q-c)/d and dd/dv_k = -b_k (q-c)/d against FP64 central
    differences (h = 1e-6) of the brute-force distance, away from ties and
    from d = 0."""
    m = dg.workload(3, n_queries=400, level=3)
    Vd = m.verts.astype(np.float64)
    o = oracle.OracleMesh(Vd, m.tris, build_tables=False)
    q = m.queries.astype(np.float64)
    r = o.bruteforce(q)
    keep = (r["second"] - r["dist"] > 1e-4) & (r["dist"] > 1e-4)
    idx = np.nonzero(keep)[0][:60]
    h = 1e-6
    gq, bv, gv = oracle.gradient(q, r)
    for i in idx:
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            dp = o.bruteforce((q[i] + e)[None])["dist"][0]
            dm = o.bruteforce((q[i] - e)[None])["dist"][0]
            assert abs((dp - dm) / (2 * h) - gq[i, k]) < 1e-6
    for i in idx[:15]:
        for slot in range(3):
            v = bv[i, slot]
            if v < 0:
                continue
            for k in range(3):
                Vp = Vd.copy()
                Vp[v, k] += h
                Vm = Vd.copy()
                Vm[v, k] -= h
                dp = oracle.OracleMesh(Vp, m.tris, build_tables=False).bruteforce(q[i][None])["dist"][0]
                dm = oracle.OracleMesh(Vm, m.tris, build_tables=False).bruteforce(q[i][None])["dist"][0]
                assert abs((dp - dm) / (2 * h) - gv[i, slot, k]) < 1e-5


# --------------------------------------------------------------------------
# robustness of the input checks
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case,msg", [
    ("index", "index out of range"), ("repeat", "repeated index"),
    ("dup", "duplicate vertex"), ("unref", "unreferenced vertex"),
    ("nan", "non-finite"), ("empty", "no triangles")])
def test_invalid_meshes_rejected(case, msg):
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
    with pytest.raises(ValueError, match=msg):
        oracle.OracleMesh(V, F)


# --------------------------------------------------------------------------
# mixed segments and triangles (Sec. 5): segments are edges of no face
# --------------------------------------------------------------------------

def test_segment_closed_forms():
    """A lone segment from (0,0,0) to (2,0,0): distances by hand."""
    V = np.array([[0, 0, 0], [2, 0, 0]], np.float32)
    # margin 2 x the bbox diagonal: every query below lies inside D
    o = oracle.OracleMesh(V, np.zeros((0, 3), np.int32), 4.0, 2.0, segs=[[0, 1]])
    assert (np.abs(o.domain_lo) >= 3).all() and (o.domain_hi >= 3).all()
    assert (o.nf, o.ne) == (0, 1)
    q = np.array([[1, 3, 0], [3, 1, 0], [-1, 0, 0], [0.5, 0, -2]], np.float32)
    want_d = [3.0, np.sqrt(2.0), 1.0, 2.0]
    want_t = [oracle.EDGE, oracle.VERTEX, oracle.VERTEX, oracle.EDGE]
    want_i = [0, 1, 0, 0]
    want_c = [[1, 0, 0], [2, 0, 0], [0, 0, 0], [0.5, 0, 0]]
    for r in (o.bruteforce(q), o.query(q, use_boxes=True)):
        np.testing.assert_allclose(r["dist"], want_d, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(r["ptype"], want_t)
        np.testing.assert_array_equal(r["pid"], want_i)
        np.testing.assert_allclose(r["cp"], want_c, rtol=0, atol=1e-12)


def test_mixed_triangle_and_segment_closed_form():
    """Triangle (0,0,0),(1,0,0),(0,1,0) under the segment (0,0,2)-(1,1,2):
    edge ids follow the canonical order, so the segment is edge 3."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 2], [1, 1, 2]], np.float32)
    o = oracle.OracleMesh(V, [[0, 1, 2]], 4.0, 0.5, segs=[[3, 4]])
    np.testing.assert_array_equal(o.edges(), [[0, 1], [0, 2], [1, 2], [3, 4]])
    q = np.array([[0.25, 0.25, 1.2], [0.25, 0.25, 0.5], [2, 2, 2]], np.float32)
    qd = q.astype(np.float64)
    want_d = [2 - qd[0, 2], qd[1, 2], np.sqrt(2.0)]
    for r in (o.bruteforce(q), o.query(q, use_boxes=True)):
        np.testing.assert_allclose(r["dist"], want_d, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(r["ptype"], [oracle.EDGE, oracle.FACE, oracle.VERTEX])
        np.testing.assert_array_equal(r["pid"], [3, 0, 4])
        np.testing.assert_allclose(r["cp"], [[qd[0, 0], qd[0, 1], 2], [qd[1, 0], qd[1, 1], 0],
                                             [1, 1, 2]], rtol=0, atol=1e-12)


def test_segment_on_a_face_side_is_that_edge():
    V, F = dg.octahedron()
    V = V.astype(np.float32)
    o1 = oracle.OracleMesh(V, F, build_tables=False)
    o2 = oracle.OracleMesh(V, F, segs=[list(F[0, :2])], build_tables=False)
    assert o2.ne == o1.ne
    q = rng(11).uniform(-2, 2, size=(2000, 3))
    a, b = o1.bruteforce(q), o2.bruteforce(q)
    for k in ("dist", "ptype", "pid"):
        np.testing.assert_array_equal(a[k], b[k])


def test_mixed_tables_and_query():
    """Mesh + wireframe: the P2M query equals the plain definition, every
    vertex intercepts its incident segments (Thm. 2), and sampled points
    find their closest primitive in the list of their nearest vertex."""
    m = dg.mixed_workload(mesh_level=2, wire_level=1, n_queries=20000)
    S = m.meta["segs"]
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin, segs=S)
    bf = o.bruteforce(m.queries)
    assert (bf["ptype"] == oracle.EDGE).sum() > 1000
    for ub in (False, True):
        r = o.query(m.queries, use_boxes=ub)
        np.testing.assert_array_equal(r["dist"], bf["dist"])
        np.testing.assert_array_equal(r["pid"], bf["pid"])
    T = _table_set(o)
    E = {tuple(e): k for k, e in enumerate(o.edges().tolist())}
    for a, b in S.tolist():
        e = E[(min(a, b), max(a, b))]
        assert (a, oracle.EDGE, e) in T and (b, oracle.EDGE, e) in T
    q = rng(12).uniform(o.domain_lo, o.domain_hi, size=(20000, 3))
    r = o.bruteforce(q)
    nn = brute_nn(m.verts, q)
    for i in range(q.shape[0]):
        t, pid = int(r["ptype"][i]), int(r["pid"][i])
        if t != oracle.VERTEX:
            b = T[(int(nn[i]), t, pid)]
            assert (q[i] >= b[:3]).all() and (q[i] <= b[3:]).all()


@pytest.mark.parametrize("segs,msg", [([[0, 0]], "repeated index"),
                                      ([[0, 99]], "index out of range")])
def test_invalid_segments_rejected(segs, msg):
    V, F = dg.octahedron()
    with pytest.raises(ValueError, match=msg):
        oracle.OracleMesh(V.astype(np.float32), F, segs=segs)


def test_vertex_used_only_by_a_segment_is_referenced():
    V, F = dg.octahedron()
    V = np.concatenate([V, [[3, 0, 0]]]).astype(np.float32)
    o = oracle.OracleMesh(V, F, segs=[[0, 6]], build_tables=False)
    assert o.ne == 13


# --------------------------------------------------------------------------
# statistics the paper reports as ranges (sanity only; parity unpinned:
# the paper's models are not available)
# --------------------------------------------------------------------------

def test_statistics_in_paper_ranges():
    """Sec. 5.1: list lengths mostly 20-100; Sec. 6: about 85 % of the
    vertices visited by flooding are not interceptors."""
    m = dg.workload(0, n_queries=10)
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    off = o.table()[0]
    L = np.diff(off)
    assert 20 <= L.mean() <= 100
    reject = 1 - o.n_entries / o.n_inspections
    assert 0.6 <= reject <= 0.95


# --------------------------------------------------------------------------
# ConvexPoly and the Region boxes (Sec. 4.4, 4.6)
# --------------------------------------------------------------------------

def _in_space_perp(V, F, E, ptype, pid, x, tol):
    """Membership in Space-perp(p) written from Eq. 4/5 directly: a face's
    prism (projection inside the triangle), an edge's slab between the
    endpoint planes and on the far side of every adjacent face."""
    if ptype == oracle.FACE:
        a, b, c = V[F[pid]]
        n = np.cross(b - a, c - a)
        ok = np.ones(x.shape[0], bool)
        for p0, p1 in ((a, b), (b, c), (c, a)):
            inward = np.cross(n, p1 - p0)
            inward /= np.linalg.norm(inward)
            ok &= (x - p0) @ inward >= -tol
        return ok
    a, b = V[E[pid, 0]], V[E[pid, 1]]
    u = (b - a) / np.linalg.norm(b - a)
    s = (x - a) @ u
    ok = (s >= -tol) & (s <= np.linalg.norm(b - a) + tol)
    for f in np.nonzero((F == E[pid, 0]).any(1) & (F == E[pid, 1]).any(1))[0]:
        third = [w for w in F[f] if w not in E[pid]][0]
        c = V[third]
        w = (c - a) - ((c - a) @ u) * u       # in-plane direction into the face
        w /= np.linalg.norm(w)
        ok &= (x - a) @ w <= tol
    return ok


def test_convexpoly_volume_matches_sampling():
    """ConvexPoly(v,p) = Cell(v) ∩ Space-perp(p): its volume matches a Monte
    Carlo estimate whose membership test uses the nearest vertex and the
    Space-perp definitions directly."""
    m = dg.workload(0, n_queries=10, level=2)
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    V = m.verts.astype(np.float64)
    E = o.edges()
    r_ = rng(11)
    off, t, ids, boxes = o.table()
    checked = 0
    for j in r_.choice(off[-1], size=40, replace=False):
        v = int(np.searchsorted(off, j, side="right") - 1)
        cor = o.convexpoly(v, int(t[j]), int(ids[j]))
        if cor.shape[0] < 4:
            continue
        try:
            vol = ConvexHull(cor).volume
        except Exception:
            continue
        lo, hi = cor.min(0), cor.max(0)
        x = r_.uniform(lo, hi, size=(20000, 3))
        nn = brute_nn(V, x)
        inside = (nn == v) & _in_space_perp(V, m.tris, E, int(t[j]), int(ids[j]), x, 0.0)
        est = inside.mean() * np.prod(hi - lo)
        err = 4 * np.sqrt(max(inside.mean(), 1e-4) / x.shape[0]) * np.prod(hi - lo)
        assert abs(est - vol) <= err + 1e-3 * vol, (v, t[j], ids[j], est, vol)
        checked += 1
    assert checked >= 20


def test_region_box_contains_relaxed_region_corners():
    """The Region box of (v,p) contains every ConvexPoly corner where v is
    not nearer than the primitive's line or plane (the relaxed Bisect^e side
    of Thm. 5/6), with the delta padding on every side."""
    m = dg.workload(0, n_queries=10, level=2)
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    V = m.verts.astype(np.float64)
    E = o.edges()
    diag = np.linalg.norm(o.domain_hi - o.domain_lo)
    eta = 2 * o.delta * diag + o.delta ** 2
    off, t, ids, boxes = o.table()
    n_seen = 0
    for j in range(0, off[-1], 7):
        v = int(np.searchsorted(off, j, side="right") - 1)
        cor = o.convexpoly(v, int(t[j]), int(ids[j]))
        if t[j] == oracle.EDGE:
            a, b = V[E[ids[j]]]
            u = (b - a) / np.linalg.norm(b - a)
            w = cor - a
            dist2 = (w * w).sum(1) - (w @ u) ** 2
        else:
            a, b, c = V[m.tris[ids[j]]]
            n = np.cross(b - a, c - a)
            n /= np.linalg.norm(n)
            dist2 = ((cor - a) @ n) ** 2
        g = ((cor - V[v]) ** 2).sum(1) - dist2 + eta
        sel = cor[g > 0]
        if sel.size == 0:
            continue
        bx = boxes[j]
        assert (sel >= bx[:3] + 0.5 * o.delta).all() and (sel <= bx[3:] - 0.5 * o.delta).all()
        n_seen += 1
    assert n_seen > 100


def _spherical_fixture():
    rows = []
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "spherical_surface_intercepts.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, gen, nv, nf, per = line.split()
            rows.append((name, gen, int(nv), int(nf), int(per)))
    return rows


def _spherical_mesh(gen):
    V, F = {"icosphere(0)": lambda: dg.icosphere(0), "icosphere(1)": lambda: dg.icosphere(1),
            "octahedron()": dg.octahedron}[gen]()
    return V.astype(np.float32), F.astype(np.int32)


@pytest.mark.parametrize("row", _spherical_fixture(), ids=lambda r: r[0])
def test_spherical_surface_every_vertex_intercepts_every_face(row):
    """Sec. 6: on a spherical surface each vertex intercepts every triangle
    (tests/golden/spherical_surface_intercepts.txt).  Every Voronoi cell
    reaches the sphere's centre, which projects inside every face."""
    name, gen, nv, nf, per = row
    V, F = _spherical_mesh(gen)
    o = oracle.OracleMesh(V, F, 10.0, 0.0)
    assert (o.nv, o.nf) == (nv, nf)
    off, tt, ii, _ = o.table()
    for v in range(o.nv):
        faces = set(ii[off[v]:off[v + 1]][tt[off[v]:off[v + 1]] == 2].tolist())
        assert faces == set(range(per)), (name, v)


def test_region_box_is_tight():
    """Reading of Sec. 4.6: the Region box is the exact bounding box of
    ConvexPoly ∩ {g > 0} (g = |x-v|^2 - Dist(x)^2 + eta), padded by delta.
    A linear function over ConvexPoly minus a convex set peaks on the
    polytope's boundary, down to its edges, so dense samples along every
    edge of the polytope's convex hull (a different construction: scipy's
    hull, points kept where g > 0) reach the box's faces to within the
    sampling step.  Catches a box taken over the whole polytope."""
    m = dg.workload(0, n_queries=10, level=2)
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    V = m.verts.astype(np.float64)
    E = o.edges()
    diag = np.linalg.norm(o.domain_hi - o.domain_lo)
    eta = 2 * o.delta * diag + o.delta ** 2
    off, t, ids, boxes = o.table()
    tt = np.linspace(0.0, 1.0, 2001)[:, None]
    n_seen = n_partial = 0
    for j in range(0, off[-1], 11):
        v = int(np.searchsorted(off, j, side="right") - 1)
        cor = o.convexpoly(v, int(t[j]), int(ids[j]))
        try:
            hull = ConvexHull(cor)
        except Exception:
            continue  # a flat polytope
        pairs = set()
        for s in hull.simplices:
            for a, b in ((s[0], s[1]), (s[1], s[2]), (s[0], s[2])):
                pairs.add((min(a, b), max(a, b)))
        pairs = np.array(sorted(pairs))
        pts = (cor[pairs[:, 0]][None] * (1 - tt[..., None]) +
               cor[pairs[:, 1]][None] * tt[..., None]).reshape(-1, 3)
        step = np.linalg.norm(cor[pairs[:, 1]] - cor[pairs[:, 0]], axis=1).max() / 2000
        if t[j] == oracle.EDGE:
            a, b = V[E[ids[j]]]
            u = (b - a) / np.linalg.norm(b - a)
            w = pts - a
            dist2 = (w * w).sum(1) - (w @ u) ** 2
        else:
            a, b, c = V[m.tris[ids[j]]]
            n = np.cross(b - a, c - a)
            n /= np.linalg.norm(n)
            dist2 = ((pts - a) @ n) ** 2
        g = ((pts - V[v]) ** 2).sum(1) - dist2 + eta
        sel = pts[g > 0]
        if sel.shape[0] == 0:
            continue  # an incident primitive kept by Thm. 2 alone
        bx = boxes[j].astype(np.float64)
        lo, hi = bx[:3] + o.delta, bx[3:] - o.delta
        tol = step + 1e-6 * diag  # sampling step, float32 rounding of the stored box
        assert (sel.min(0) >= lo - tol).all() and (sel.max(0) <= hi + tol).all(), j
        assert (np.abs(sel.min(0) - lo) <= tol).all() and (np.abs(sel.max(0) - hi) <= tol).all(), j
        n_seen += 1
        n_partial += bool((g <= 0).any())
    assert n_seen > 100 and n_partial > 20
