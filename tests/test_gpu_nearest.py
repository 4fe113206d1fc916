"""Step a2 on its own: the device KD-tree nearest vertex (p2m_nearest_vertex)
equals the FP64 nearest vertex of the oracle's KD tree."""
import numpy as np
import pytest

import datagen as dg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("idx,kw", [(0, {}), (1, {"level": 6}), (2, {"grid": 128}),
                                    (3, {"level": 5})])
@pytest.mark.parametrize("walk", [0, 1, 2])
def test_nearest_vertex_matches_oracle(idx, kw, walk):
    """Every search: KD-tree backtracking, KD descent + Voronoi walk, seed
    grid + Voronoi walk (queries outside D fall back to backtracking)."""
    import paper_2308_16084_gb300 as pg
    m = dg.workload(idx, n_queries=60000, **kw)
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    mesh.tuning = {"nn_walk": walk}
    q = torch.from_numpy(m.queries).cuda()
    nn = mesh.nearest_vertex(q).cpu().numpy()
    o = oracle.OracleMesh(m.verts, m.tris, build_tables=False)
    ref, _ = o.kdt_nn(m.queries)
    V = m.verts.astype(np.float64)
    qd = m.queries.astype(np.float64)
    gap = np.linalg.norm(qd - V[nn], axis=1) - np.linalg.norm(qd - V[ref], axis=1)
    # identical, or an equidistant vertex within float32 rounding
    assert (gap <= 1e-6 * np.linalg.norm(qd, axis=1).max()).all()
    assert (nn == ref).mean() > 0.9999


def test_nearest_vertex_special_inputs():
    import paper_2308_16084_gb300 as pg
    m = dg.workload(0, n_queries=10)
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    q = torch.from_numpy(np.concatenate([m.verts[:7], [[np.nan, 0, 0]]]).astype(np.float32)).cuda()
    nn = mesh.nearest_vertex(q).cpu().numpy()
    np.testing.assert_array_equal(nn[:7], np.arange(7))
    assert nn[7] == -1
    assert mesh.nearest_vertex(torch.zeros(0, 3, device="cuda")).numel() == 0
