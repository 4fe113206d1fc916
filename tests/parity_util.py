"""Parity criterion between the CUDA path and the FP64 oracle.

The bar (tolerance tau = 1e-5 x bounding-box diagonal):
  - distance within tau of the oracle's;
  - primitive (type, id) identical, except where the oracle's two best
    primitives are within tau of each other (a near tie), or where the
    primitive the kernel reports lies, in FP64, within tau of the oracle's
    distance (an open face or edge whose float32 gate landed on the other
    side of a boundary it shares with the oracle's primitive);
  - closest point within tau of the oracle's wherever the primitive matches.
"""
import numpy as np

VERTEX, EDGE, FACE = 0, 1, 2


def tolerance(verts):
    v = np.asarray(verts, np.float64)
    return 1e-5 * float(np.linalg.norm(v.max(0) - v.min(0)))


def closed_distance(V, E, F, q, ptype, pid):
    """FP64 distance from q to the closed primitive (vertex, segment,
    triangle), computed here independently of both implementations."""
    V = np.asarray(V, np.float64)
    q = np.asarray(q, np.float64)
    out = np.full(q.shape[0], np.inf)
    for i in range(q.shape[0]):
        t, k = int(ptype[i]), int(pid[i])
        p = q[i]
        if t == VERTEX and 0 <= k < V.shape[0]:
            out[i] = np.linalg.norm(p - V[k])
        elif t == EDGE and 0 <= k < E.shape[0]:
            a, b = V[E[k, 0]], V[E[k, 1]]
            d = b - a
            s = np.clip(np.dot(p - a, d) / np.dot(d, d), 0, 1)
            out[i] = np.linalg.norm(p - (a + s * d))
        elif t == FACE and 0 <= k < F.shape[0]:
            a, b, c = V[F[k, 0]], V[F[k, 1]], V[F[k, 2]]
            n = np.cross(b - a, c - a)
            nn = n / np.linalg.norm(n)
            h = np.dot(p - a, nn)
            x = p - h * nn
            inside = all(np.dot(np.cross(e1 - e0, x - e0), n) >= 0
                         for e0, e1 in ((a, b), (b, c), (c, a)))
            if inside:
                out[i] = abs(h)
            else:
                best = np.inf
                for e0, e1 in ((a, b), (b, c), (c, a)):
                    d = e1 - e0
                    s = np.clip(np.dot(p - e0, d) / np.dot(d, d), 0, 1)
                    best = min(best, np.linalg.norm(p - (e0 + s * d)))
                out[i] = best
    return out


def check(V, E, F, q, gpu, ref, tau, label=""):
    """Assert the parity bar; returns a dict of summary numbers."""
    d = np.asarray(gpu["dist"], np.float64)
    dr = ref["dist"]
    assert np.isfinite(d).all(), f"{label}: non-finite distances"
    derr = np.abs(d - dr)
    worst = int(derr.argmax())
    assert derr.max() <= tau, f"{label}: |d - d_oracle| = {derr.max()} > {tau} at {worst}"
    same = (np.asarray(gpu["prim_type"]) == ref["ptype"]) & (np.asarray(gpu["prim_id"]) == ref["pid"])
    near_tie = (ref["second"] - ref["dist"]) < tau if "second" in ref else np.zeros_like(same)
    bad = np.nonzero(~same & ~near_tie)[0]
    if bad.size:
        cd = closed_distance(V, E, F, q[bad], np.asarray(gpu["prim_type"])[bad],
                             np.asarray(gpu["prim_id"])[bad])
        still = bad[cd > dr[bad] + tau]
        assert still.size == 0, (f"{label}: {still.size} primitive mismatches beyond the tie "
                                 f"rule, first at {still[:5]}")
    if "closest" in gpu:
        cerr = np.linalg.norm(np.asarray(gpu["closest"], np.float64) - ref["cp"], axis=1)
        assert cerr[same].max(initial=0.0) <= tau, f"{label}: closest point error {cerr[same].max()}"
    return {"n": int(d.shape[0]), "max_dist_err": float(derr.max()),
            "prim_exact": float(same.mean()), "near_ties": int(near_tie.sum()),
            "boundary_mismatches": int(bad.size)}
