"""The seeded synthetic workloads (the input recipe): the mesh and query
sizes of the five workloads, what the generators promise about them, and
their determinism.  CPU only."""
import numpy as np
import pytest

import datagen as dg


def n_edges(f):
    """Unique undirected edges of a triangle list."""
    f = np.asarray(f, np.int64)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    e.sort(1)
    return np.unique(e[:, 0] * (int(f.max()) + 1) + e[:, 1]).shape[0]


@pytest.mark.parametrize("idx,V,F,E", [
    (0, 642, 1_280, 1_920),                   # icosphere level 3: 10 4^k + 2, 20 4^k, 30 4^k
    (1, 655_362, 1_310_720, 1_966_080),       # icosphere level 8
    (2, 1_048_576, 2_093_058, 3_141_633),     # 1024^2 grid: n^2, 2 (n-1)^2, 3 (n-1)^2 + 2 (n-1)
    (3, 163_842, 327_680, 491_520),           # icosphere level 7
])
def test_workload_mesh_sizes(idx, V, F, E):
    m = dg.workload(idx, n_queries=1000)
    assert m.verts.shape == (V, 3) and m.verts.dtype == np.float32
    assert m.tris.shape == (F, 3) and m.tris.dtype == np.int32
    assert n_edges(m.tris) == E
    assert np.isfinite(m.verts).all()
    assert np.array_equal(np.unique(m.tris), np.arange(V))  # every vertex used
    assert m.queries.shape == (1000, 3) and m.queries.dtype == np.float32


def test_workload_query_counts_and_distributions():
    m = dg.workload(0)
    assert m.queries.shape[0] == 100_000
    m = dg.workload(1, level=3)
    assert m.queries.shape[0] == 10_000_000
    # uniform in the bounding box scaled 1.5x about its centre
    lo, hi = m.verts.min(0), m.verts.max(0)
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo) * 1.5
    q = m.queries[:200_000]
    assert (q >= c - h - 1e-6).all() and (q <= c + h + 1e-6).all()
    assert np.allclose(q.mean(0), c, atol=0.01 * h.max())
    assert np.allclose(q.std(0), 2 * h / np.sqrt(12), rtol=0.02)


def test_workloads_are_seeded():
    for idx in (0, 2, 3):
        a = dg.workload(idx, n_queries=5000, level=3, grid=32)
        b = dg.workload(idx, n_queries=5000, level=3, grid=32)
        assert np.array_equal(a.verts, b.verts) and np.array_equal(a.tris, b.tris)
        assert np.array_equal(a.queries, b.queries)
    a = dg.workload(0, n_queries=5000)
    c = dg.workload(3, n_queries=5000, level=3)
    assert not np.array_equal(a.verts, c.verts)  # separate streams per workload


def test_batch_workload_shape():
    """64 meshes whose triangle counts follow a log-uniform target in
    [1k, 500k], rounded to an icosphere level 3..7 (1,280 to 327,680
    triangles) or to a grid (968 to 500,000), about 5.1M in all, and whose
    query counts are log-uniform in [10k, 2M] (shrunk here by query_scale)."""
    ms = dg.batch_workload(query_scale=1e-3)
    assert len(ms) == 64
    F = np.array([m.tris.shape[0] for m in ms])
    assert F.min() >= 968 and F.max() <= 500_000
    assert 4.5e6 <= F.sum() <= 5.8e6
    N = np.array([m.queries.shape[0] for m in ms])
    assert (N >= 10).all() and (N <= 2_000).all()
