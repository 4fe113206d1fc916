"""A built handle's interception table against the oracle's (two
independent implementations of Alg. A.1): the same lists, and float32
Region boxes that contain the oracle's FP64 boxes and stay within a few
codes of them."""
import numpy as np

import oracle


def check_tables_against_oracle(h, m, same_neighbour_count=True):
    """same_neighbour_count: also require the oracle's count of Voronoi
    neighbour pairs.  Builds whose cells the device certifies may keep a
    different set of sliver faces (a bisector applied in another order can
    leave a face of rounding-level area), so they compare the tables
    only."""
    o = oracle.OracleMesh(m.verts, m.tris, m.domain_scale, m.domain_margin,
                          segs=m.meta.get("segs"))
    np.testing.assert_array_equal(h.edges(), o.edges())
    st = h.stats()
    assert st["n_entries"] == o.n_entries
    if same_neighbour_count:
        assert st["neighbour_pairs"] == o.n_neighbor_pairs
    off, tt, ii, bb = o.table()
    delta = h.domain()[2]
    assert abs(delta - o.delta) <= 1e-6 * o.delta
    for v in range(o.nv):
        t, i, b = h.interception_list(v)
        a = set(zip(t.tolist(), i.tolist()))
        r = set(zip(tt[off[v]:off[v + 1]].tolist(), ii[off[v]:off[v + 1]].tolist()))
        assert a == r, v
        # float32 Region boxes contain the oracle's FP64 boxes, up to the
        # scatter of two independent computations of crossing points, which
        # near tangential crossings is of order sqrt(eps) and stays far below
        # the delta padding of every box
        order_r = np.lexsort((ii[off[v]:off[v + 1]], tt[off[v]:off[v + 1]]))
        order_a = np.lexsort((i, t))
        ob = bb[off[v]:off[v + 1]][order_r]
        hb = b[order_a].astype(np.float64)
        tol = 1e-2 * delta
        assert (hb[:, :3] <= ob[:, :3] + tol).all() and (hb[:, 3:] >= ob[:, 3:] - tol).all()
        # and the integer box codes stay tight: a few codes of the chunk's
        # frame (at most 2^-12 of the domain) beyond the FP64 box
        slack = 2.0 ** -12 * (np.asarray(h.domain()[1]) - np.asarray(h.domain()[0]))
        assert (hb[:, :3] >= ob[:, :3] - slack - tol).all()
        assert (hb[:, 3:] <= ob[:, 3:] + slack + tol).all()
    return o
