"""p2m_update_vertices: the differentiable path's geometry refresh.

The vertex-dependent records (KD tree, neighbour positions, edge and face
records) follow new positions while the interception lists and Region boxes
stay those of the build.  Checked through the C ABI:
  - positions equal to the build's change no output bit;
  - after a small seeded move, every query whose build-time list still
    covers the moved mesh's closest primitive matches the FP64 brute force
    on the moved mesh (parity criterion of parity_util); "covers" means, for
    the nearest vertex v the GPU walks to on the moved mesh, that the
    closest primitive is v itself, or is in the oracle's build-time list of
    v with q inside the oracle's FP64 Region box of that entry (the
    product's lists equal the oracle's and its 15-bit box codes contain the
    oracle's boxes, so the product tests that entry).  Every other query
    gets an upper bound of the true distance;
  - the autograd entry point queries the positions it is given.
"""
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


def _run(mesh, q):
    r = mesh.query(q, closest=True, prim_type=True, status=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


@pytest.mark.parametrize("idx,kw", [(3, {"level": 4}), (2, {"grid": 48})])
def test_unchanged_positions_change_nothing(pg, idx, kw):
    m = dg.workload(idx, n_queries=50001, **kw)
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    q = torch.from_numpy(m.queries).cuda()
    base = _run(mesh, q)
    v = torch.from_numpy(m.verts).cuda()
    for refresh in (False, True):
        mesh.update_vertices(v, refresh_seed_grid=refresh)
        got = _run(mesh, q)
        for k in base:
            np.testing.assert_array_equal(got[k], base[k], err_msg=f"{k} refresh={refresh}")


def test_bad_arguments_rejected(pg):
    m = dg.workload(0, n_queries=10)
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    v = torch.from_numpy(m.verts).cuda()
    lib = pg.lib
    import ctypes
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = ctypes.c_void_p(v.data_ptr())
    assert lib.p2m_update_vertices(mesh._h, None, mesh.n_verts, 0, st) == 1
    assert lib.p2m_update_vertices(mesh._h, ptr, mesh.n_verts - 1, 0, st) == 1
    assert lib.p2m_update_vertices(mesh._h, ptr, mesh.n_verts, 2, st) == 1
    assert lib.p2m_update_vertices(None, ptr, mesh.n_verts, 0, st) == 1


@pytest.mark.parametrize("refresh", [False, True])
def test_moved_vertices_match_bruteforce_where_covered(pg, refresh):
    m = dg.workload(3, n_queries=60000, level=4)
    diag = dg.bbox_diagonal(m.verts)
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    o_old = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin)
    off, tt, ti, bb = o_old.table()
    rng = np.random.default_rng(77)
    moved = (m.verts.astype(np.float64) +
             rng.uniform(-1, 1, size=m.verts.shape) * 2e-4 * diag).astype(np.float32)
    mesh.update_vertices(torch.from_numpy(moved).cuda(), refresh_seed_grid=refresh)
    q = torch.from_numpy(m.queries).cuda()
    gpu = _run(mesh, q)
    nn = mesh.nearest_vertex(q).cpu().numpy()
    o_new = oracle.OracleMesh(moved, m.tris, build_tables=False)
    ref = o_new.bruteforce(m.queries)
    tau = pu.tolerance(moved)
    # every answer is the distance to some primitive: never below the truth
    assert (gpu["dist"] >= ref["dist"] - tau).all()
    qd = m.queries.astype(np.float64)
    covered = np.zeros(qd.shape[0], bool)
    for i in range(qd.shape[0]):
        v, t, p = int(nn[i]), int(ref["ptype"][i]), int(ref["pid"][i])
        if t == pu.VERTEX:
            covered[i] = p == v
            continue
        a, b = off[v], off[v + 1]
        hit = np.nonzero((tt[a:b] == t) & (ti[a:b] == p))[0]
        if hit.size:
            box = bb[a + hit[0]]
            covered[i] = bool((qd[i] >= box[:3]).all() and (qd[i] <= box[3:]).all())
    assert covered.mean() > 0.95, covered.mean()
    sel = np.nonzero(covered)[0]
    sub = {k: v[sel] for k, v in gpu.items()}
    rsub = {k: v[sel] for k, v in ref.items()}
    pu.check(moved, o_new.edges(), m.tris, m.queries[sel], sub, rsub, tau, "moved vertices")


def test_autograd_queries_the_positions_it_is_given(pg):
    m = dg.workload(3, n_queries=20000, level=4)
    diag = dg.bbox_diagonal(m.verts)
    mesh = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    rng = np.random.default_rng(5)
    moved = (m.verts.astype(np.float64) +
             rng.uniform(-1, 1, size=m.verts.shape) * 2e-4 * diag).astype(np.float32)
    q = torch.from_numpy(m.queries).cuda().requires_grad_(True)
    vm = torch.from_numpy(moved).cuda().requires_grad_(True)
    d, pid = pg.distance(q, vm, mesh)
    d.sum().backward()
    torch.cuda.synchronize()
    # the same positions through the explicit update: the same bits
    mesh.update_vertices(torch.from_numpy(moved).cuda())
    r = mesh.query(q.detach(), closest=True, prim_type=True)
    assert torch.equal(r["dist"], d.detach()) and torch.equal(r["prim_id"], pid)
    # and the build's positions again give the build's answers
    v0 = torch.from_numpy(m.verts).cuda()
    d0, _ = pg.distance(q.detach(), v0, mesh)
    mesh2 = pg.P2M(m.verts, m.tris, domain_scale=m.domain_scale, domain_margin=m.domain_margin)
    assert torch.equal(d0, mesh2.query(q.detach())["dist"])
    assert torch.isfinite(vm.grad).all() and torch.isfinite(q.grad).all()
