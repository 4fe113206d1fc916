"""Parity criterion between the CUDA path and the FP64 oracle.

The bar (tolerance tau = 1e-5 x bounding-box diagonal):
  - distance within tau of the oracle's;
  - primitive (type, id) identical, except where the oracle's two best
    primitives are within tau of each other (a near tie), or where the
    primitive the kernel reports lies, in FP64, within tau of the oracle's
    distance (an open face or edge whose float32 gate landed on the other
    side of a boundary it shares with the oracle's primitive); the second
    kind ("boundary mismatches") is counted and bounded;
  - closest point within tau of the oracle's wherever the primitive matches;
    wherever it does not, within tau of the FP64 closest point on the
    primitive the kernel reports (taken as a closed set), whose distance must
    itself be within tau of the oracle's distance.
"""
import json
import os

import numpy as np

VERTEX, EDGE, FACE = 0, 1, 2

# boundary mismatches allowed per query checked (plus a small absolute
# slack for short samples); they come from float32 gates on open sets.  On
# the GB300 none occurred in any seeded workload case; only queries placed
# on an edge on purpose produce them.
BOUNDARY_FRAC = 0.001
BOUNDARY_SLACK = 3


def tolerance(verts):
    v = np.asarray(verts, np.float64)
    return 1e-5 * float(np.linalg.norm(v.max(0) - v.min(0)))


def _segment_closest(p, a, b):
    d = b - a
    s = np.clip(np.einsum("ij,ij->i", p - a, d) / np.einsum("ij,ij->i", d, d), 0.0, 1.0)
    return a + s[:, None] * d


def closed_closest(V, E, F, q, ptype, pid):
    """FP64 closest point on the closed primitive (vertex, segment or
    triangle) named by (ptype, pid), and its distance to q.  Written here
    from the definitions, independently of both implementations: a triangle
    projects onto its plane when the foot lies inside all three edge
    half-planes, and otherwise onto the nearest of its three closed sides."""
    V = np.asarray(V, np.float64)
    q = np.asarray(q, np.float64).reshape(-1, 3)
    ptype = np.asarray(ptype).astype(np.int64)
    pid = np.asarray(pid).astype(np.int64)
    n = q.shape[0]
    cp = np.full((n, 3), np.nan)
    ok = np.zeros(n, bool)
    iv = np.nonzero((ptype == VERTEX) & (pid >= 0) & (pid < V.shape[0]))[0]
    cp[iv] = V[pid[iv]]
    ok[iv] = True
    ie = np.nonzero((ptype == EDGE) & (pid >= 0) & (pid < len(E)))[0]
    if ie.size:
        e = np.asarray(E)[pid[ie]]
        cp[ie] = _segment_closest(q[ie], V[e[:, 0]], V[e[:, 1]])
        ok[ie] = True
    iff = np.nonzero((ptype == FACE) & (pid >= 0) & (pid < len(F)))[0]
    if iff.size:
        f = np.asarray(F)[pid[iff]]
        a, b, c = V[f[:, 0]], V[f[:, 1]], V[f[:, 2]]
        p = q[iff]
        nrm = np.cross(b - a, c - a)
        nn = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
        h = np.einsum("ij,ij->i", p - a, nn)
        foot = p - h[:, None] * nn
        inside = np.ones(iff.size, bool)
        for e0, e1 in ((a, b), (b, c), (c, a)):
            inside &= np.einsum("ij,ij->i", np.cross(e1 - e0, foot - e0), nrm) >= 0
        best = np.full(iff.size, np.inf)
        bestp = np.zeros((iff.size, 3))
        for e0, e1 in ((a, b), (b, c), (c, a)):
            x = _segment_closest(p, e0, e1)
            dx = np.linalg.norm(p - x, axis=1)
            take = dx < best
            best[take] = dx[take]
            bestp[take] = x[take]
        cp[iff] = np.where(inside[:, None], foot, bestp)
        ok[iff] = True
    dist = np.where(ok, np.linalg.norm(q - np.nan_to_num(cp), axis=1), np.inf)
    return cp, dist


def closed_distance(V, E, F, q, ptype, pid):
    """FP64 distance from q to the closed primitive (vertex, segment,
    triangle)."""
    return closed_closest(V, E, F, q, ptype, pid)[1]


def grad_tolerance(dist, verts, base=2e-3):
    """Per-query bound on |grad_q - grad_q_oracle| for grad_q = (q - c)/d:
    a base error plus the direction error that a float32 closest point
    carries, about 8 ulps of the largest coordinate divided by d."""
    scale = float(np.abs(np.asarray(verts, np.float64)).max())
    return base + 8.0 * 2.0 ** -23 * scale / np.asarray(dist, np.float64)


def _log(label, summary):
    path = os.environ.get("P2M_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"label": label, **summary}) + "\n")


def check(V, E, F, q, gpu, ref, tau, label="", boundary_frac=BOUNDARY_FRAC):
    """Assert the parity bar; returns a dict of summary numbers."""
    d = np.asarray(gpu["dist"], np.float64)
    dr = ref["dist"]
    n = int(d.shape[0])
    assert np.isfinite(d).all(), f"{label}: non-finite distances"
    derr = np.abs(d - dr)
    worst = int(derr.argmax()) if n else 0
    assert derr.max(initial=0.0) <= tau, f"{label}: |d - d_oracle| = {derr.max()} > {tau} at {worst}"
    gt = np.asarray(gpu["prim_type"]) if "prim_type" in gpu else None
    gi = np.asarray(gpu["prim_id"])
    same = (gi == ref["pid"]) if gt is None else (gt == ref["ptype"]) & (gi == ref["pid"])
    near_tie = (ref["second"] - ref["dist"]) < tau if "second" in ref else np.zeros_like(same)
    mism = np.nonzero(~same)[0]
    bad = np.nonzero(~same & ~near_tie)[0]
    max_cp_err_mism = 0.0
    if mism.size and gt is not None:
        cp_c, cd = closed_closest(V, E, F, q[mism], gt[mism], gi[mism])
        far = mism[cd > dr[mism] + tau]
        assert far.size == 0, (f"{label}: {far.size} reported primitives farther than the "
                               f"oracle's distance + tau, first at {far[:5]}")
        if "closest" in gpu:
            e = np.linalg.norm(np.asarray(gpu["closest"], np.float64)[mism] - cp_c, axis=1)
            max_cp_err_mism = float(e.max())
            off = mism[e > tau]
            assert off.size == 0, (f"{label}: closest point of {off.size} mismatched queries "
                                   f"more than tau from their reported primitive, first at "
                                   f"{off[:5]} ({e.max()})")
    elif mism.size:
        # no primitive types given: ids must still match outside near ties
        assert bad.size == 0, f"{label}: {bad.size} id mismatches beyond the tie rule"
    limit = boundary_frac * n + BOUNDARY_SLACK
    assert bad.size <= limit, (f"{label}: {bad.size} boundary mismatches, more than the "
                               f"bound {limit:.0f} for {n} queries")
    max_cp_err = 0.0
    if "closest" in gpu:
        cerr = np.linalg.norm(np.asarray(gpu["closest"], np.float64) - ref["cp"], axis=1)
        max_cp_err = float(cerr[same].max(initial=0.0))
        assert max_cp_err <= tau, f"{label}: closest point error {max_cp_err}"
    s = {"n": n, "max_dist_err": float(derr.max(initial=0.0)),
         "prim_exact": float(same.mean()) if n else 1.0, "near_ties": int(near_tie.sum()),
         "mismatches": int(mism.size), "boundary_mismatches": int(bad.size),
         "boundary_bound": float(limit), "max_closest_err": max_cp_err,
         "max_closest_err_mismatched": max_cp_err_mism, "tau": float(tau)}
    _log(label, s)
    return s
