"""Seeded synthetic inputs for the point-to-mesh query workloads.

This module draws meshes and query points only.  It holds none of the
P2M method's arithmetic (no distances, no Voronoi cells, no tables), so
both the FP64 oracle and the CUDA path can take their inputs from it
without sharing any of the method's code.

Every generator works in float64 and rounds once to float32 at the end,
which is the storage precision of both paths.  Seeds are derived from
``numpy.random.SeedSequence(16084)``: one child sequence per workload,
and from it independent sub-streams for the mesh, the queries and the
loss weights.

The paper's evaluation meshes (Camel, Armadillo, Sponza, Lucy, Dragon,
Thingi10K, Bear, Water-Bottle) are not available here.  The synthetic
workloads below stand in for their roles: smooth closed surfaces
(icospheres with radial displacement), poorly triangulated meshes
(jittered fractal height fields with slivers, Table 5 of the paper),
size diversity (the 64-mesh batch, Thingi10K), and the query
distribution of Sec. 5 (uniform in a scaled bounding box) together with
near-surface queries.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ROOT_SEED = 16084


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
        [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
        [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v, f


def icosphere(level: int):
    """Unit icosphere: the icosahedron subdivided ``level`` times, every new
    edge midpoint projected back onto the unit sphere.  Faces are oriented
    outward.  V = 10*4^k + 2, F = 20*4^k."""
    v, f = _icosahedron()
    for _ in range(level):
        nv = v.shape[0]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        pairs = np.stack([np.stack([a, b], 1), np.stack([b, c], 1),
                          np.stack([c, a], 1)], 0).reshape(-1, 2)
        key = np.sort(pairs, axis=1)
        uniq, inv = np.unique(key, axis=0, return_inverse=True)
        inv = inv.reshape(3, -1)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], 0)
        ab, bc, ca = inv[0] + nv, inv[1] + nv, inv[2] + nv
        f = np.concatenate([
            np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
            np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)], 0)
    return v, f


def noisy_icosphere(level: int, amplitude: float, rng):
    """Icosphere with every vertex radius drawn as 1 + U(-a, a)."""
    v, f = icosphere(level)
    r = 1.0 + rng.uniform(-amplitude, amplitude, size=v.shape[0])
    return v * r[:, None], f


def uv_sphere(n_lat: int, n_lon: int, amplitude: float, rng):
    """Unit sphere triangulated by latitude and longitude: two poles and
    n_lat - 1 rings of n_lon vertices, each band of quads split along one
    diagonal, triangle fans at the poles.  Near the poles the triangles are
    long and thin: a poor triangulation of the surface icosphere() covers
    well (the poor/good contrast of Sec. 5.5).  Radii 1 + U(-a, a), as
    noisy_icosphere.  Faces are oriented outward."""
    th = np.pi * np.arange(1, n_lat) / n_lat
    ph = 2 * np.pi * np.arange(n_lon) / n_lon
    ring = np.stack([np.sin(th)[:, None] * np.cos(ph)[None, :],
                     np.sin(th)[:, None] * np.sin(ph)[None, :],
                     np.cos(th)[:, None] * np.ones_like(ph)[None, :]], -1).reshape(-1, 3)
    v = np.concatenate([[[0.0, 0.0, 1.0]], ring, [[0.0, 0.0, -1.0]]], 0)
    south = v.shape[0] - 1

    def at(i, j):  # ring i (0 = nearest the north pole), longitude j
        return 1 + i * n_lon + j % n_lon

    f = [[0, at(0, j), at(0, j + 1)] for j in range(n_lon)]
    for i in range(n_lat - 2):
        for j in range(n_lon):
            a, b, c, d = at(i, j), at(i, j + 1), at(i + 1, j), at(i + 1, j + 1)
            f += [[a, c, d], [a, d, b]]
    f += [[south, at(n_lat - 2, j + 1), at(n_lat - 2, j)] for j in range(n_lon)]
    f = np.array(f, dtype=np.int64)
    v = v * (1.0 + rng.uniform(-amplitude, amplitude, size=(v.shape[0], 1)))
    nrm = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = (nrm * v[f].mean(1)).sum(1) < 0
    f[flip] = f[flip][:, ::-1]
    return v, f


def displaced_icosphere(level: int, amplitude: float, rng, n_terms: int = 8):
    """Icosphere with a smooth low-frequency radial displacement
    r(u) = 1 + a * s(u), s(u) = sum_j a_j cos(w_j d_j.u + phi_j), scaled so that
    max |s| over the vertices is 1.  Gives uneven triangle sizes."""
    v, f = icosphere(level)
    aj = rng.standard_normal(n_terms)
    wj = rng.uniform(1.0, 3.0, n_terms)
    dj = rng.standard_normal((n_terms, 3))
    dj /= np.linalg.norm(dj, axis=1, keepdims=True)
    pj = rng.uniform(0.0, 2.0 * math.pi, n_terms)
    s = np.zeros(v.shape[0])
    for j in range(n_terms):
        s += aj[j] * np.cos(wj[j] * (v @ dj[j]) + pj[j])
    s /= np.abs(s).max()
    return v * (1.0 + amplitude * s)[:, None], f


def _grid_triangles(n: int):
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    v00 = (i * n + j).ravel()
    v01 = v00 + 1
    v10 = v00 + n
    v11 = v10 + 1
    t1 = np.stack([v00, v01, v11], 1)
    t2 = np.stack([v00, v11, v10], 1)
    return np.stack([t1, t2], 1).reshape(-1, 3)


def fractal_heightfield(n: int, rng, peak_to_peak: float = 0.2,
                        spectral_exponent: float = 1.2,
                        jitter_fraction: float = 0.2,
                        jitter_radius: float = 0.45):
    """n x n grid on [0,1]^2 with heights from spectral synthesis (amplitude
    proportional to |f|^-exponent, random phases), normalised to the given
    peak-to-peak range.  ``jitter_fraction`` of the interior vertices move
    in-plane uniformly inside a disk of radius ``jitter_radius`` * h,
    h = 1/(n-1); jitters that would fold a triangle over in the plane are
    drawn again.  The diagonal of every grid quad has one fixed direction."""
    fx = np.fft.fftfreq(n) * n
    fr = np.sqrt(fx[:, None] ** 2 + fx[None, :] ** 2)
    amp = np.zeros_like(fr)
    amp[fr > 0] = fr[fr > 0] ** (-spectral_exponent)
    coef = amp * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    hgt = np.real(np.fft.ifft2(coef))
    hgt = (hgt - hgt.min()) * (peak_to_peak / (hgt.max() - hgt.min()))
    h = 1.0 / (n - 1)
    g = np.arange(n) * h
    yy, xx = np.meshgrid(g, g, indexing="ij")
    xy = np.stack([xx.ravel(), yy.ravel()], 1)
    f = _grid_triangles(n)

    interior = (np.arange(1, n - 1)[:, None] * n + np.arange(1, n - 1)[None, :]).ravel()
    n_j = int(round(jitter_fraction * interior.size))
    chosen = rng.choice(interior, size=n_j, replace=False) if n_j > 0 else \
        np.zeros(0, np.int64)
    disp = np.zeros_like(xy)

    def draw(idx):
        r = jitter_radius * h * np.sqrt(rng.uniform(size=idx.size))
        th = rng.uniform(0.0, 2.0 * math.pi, size=idx.size)
        disp[idx, 0] = r * np.cos(th)
        disp[idx, 1] = r * np.sin(th)

    draw(chosen)
    is_chosen = np.zeros(n * n, bool)
    is_chosen[chosen] = True
    min_area = 1e-3 * h * h
    for it in range(200):
        p = xy + disp
        a, b, c = p[f[:, 0]], p[f[:, 1]], p[f[:, 2]]
        area2 = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - \
                (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
        bad = area2 <= 2.0 * min_area
        if not bad.any():
            break
        redo = np.unique(f[bad].ravel())
        redo = redo[is_chosen[redo]]
        if it >= 150:
            disp[redo] = 0.0
        else:
            draw(redo)
    p = xy + disp
    v = np.stack([p[:, 0], p[:, 1], hgt.ravel()], 1)
    return v, f


def cube():
    """Axis-aligned cube [-1,1]^3 with 12 outward triangles."""
    v = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)],
                 dtype=np.float64)

    def idx(x, y, z):
        return ((x + 1) // 2) * 4 + ((y + 1) // 2) * 2 + ((z + 1) // 2)

    quads = []
    for ax in range(3):
        for s in (-1, 1):
            o = [a for a in range(3) if a != ax]
            cs = []
            for (u, w) in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
                c = [0, 0, 0]
                c[ax] = s
                c[o[0]] = u
                c[o[1]] = w
                cs.append(idx(*c))
            quads.append(cs)
    f = []
    for q in quads:
        f.append([q[0], q[1], q[2]])
        f.append([q[0], q[2], q[3]])
    f = np.array(f, dtype=np.int64)
    # orient outward
    cen = v[f].mean(1)
    nrm = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = (nrm * cen).sum(1) < 0
    f[flip] = f[flip][:, ::-1]
    return v, f


def octahedron():
    """Regular octahedron |x|+|y|+|z| = 1 with 8 outward triangles."""
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float64)
    f = []
    for xi in (0, 1):
        for yi in (2, 3):
            for zi in (4, 5):
                f.append([xi, yi, zi])
    f = np.array(f, dtype=np.int64)
    nrm = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    cen = v[f].mean(1)
    flip = (nrm * cen).sum(1) < 0
    f[flip] = f[flip][:, ::-1]
    return v, f


# ----------------------------------------------------------------------------
# queries
# ----------------------------------------------------------------------------

def bbox(v):
    return v.min(0), v.max(0)


def uniform_in_box(v, scale, n, rng):
    lo, hi = bbox(v)
    c = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo) * scale
    return c + rng.uniform(-1.0, 1.0, size=(n, 3)) * half


def surface_points(v, f, n, rng):
    """Area-weighted uniform points on the triangles."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    cdf = np.cumsum(area)
    cdf /= cdf[-1]
    fi = np.searchsorted(cdf, rng.uniform(size=n), side="right")
    fi = np.minimum(fi, f.shape[0] - 1)
    r1 = np.sqrt(rng.uniform(size=n))
    r2 = rng.uniform(size=n)
    w0, w1, w2 = 1.0 - r1, r1 * (1.0 - r2), r1 * r2
    return w0[:, None] * a[fi] + w1[:, None] * b[fi] + w2[:, None] * c[fi]


def near_surface(v, f, n, radius, rng):
    """Surface point plus a uniform offset in the ball of the given radius."""
    p = surface_points(v, f, n, rng)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(size=n) ** (1.0 / 3.0)
    return p + d * r[:, None]


def gaussian_about_surface(v, f, n, sigma, rng):
    p = surface_points(v, f, n, rng)
    return p + rng.standard_normal((n, 3)) * sigma


def bbox_diagonal(v):
    lo, hi = bbox(v)
    return float(np.linalg.norm(hi - lo))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclass
class Mesh:
    name: str
    verts: np.ndarray        # (V,3) float32
    tris: np.ndarray         # (F,3) int32
    queries: np.ndarray      # (N,3) float32
    domain_scale: float      # query domain D = bbox scaled about its centre ...
    domain_margin: float     # ... plus this fraction of the bbox diagonal per side
    weights: np.ndarray | None = None   # (N,) float32 loss weights (differentiable workload)
    meta: dict = field(default_factory=dict)


def _streams(index: int, n: int):
    child = np.random.SeedSequence(ROOT_SEED).spawn(5)[index]
    return [np.random.default_rng(s) for s in child.spawn(n)]


def _finish(name, v, f, q, scale, margin, w=None, meta=None):
    return Mesh(name, np.ascontiguousarray(v, np.float32),
                np.ascontiguousarray(f, np.int32),
                np.ascontiguousarray(q, np.float32), float(scale), float(margin),
                None if w is None else np.ascontiguousarray(w, np.float32),
                meta or {})


WORKLOADS = {
    0: "icosphere-L3-noise0.05-100k",
    1: "icosphere-L8-displaced0.2-10M-uniform1.5",
    2: "heightfield-1024-jitter0.2-16M-gauss0.01",
    3: "icosphere-L7-noise0.05-4M-near-fwdbwd",
    4: "batch64-icosphere-heightfield-1k..500k",
}


def workload(index: int, n_queries: int | None = None, level: int | None = None,
             grid: int | None = None):
    """Build one of the five workloads.  ``n_queries``, ``level`` and ``grid``
    shrink it for tests (same recipe, fewer queries or a coarser mesh)."""
    rm, rq, rw = _streams(index, 3)
    if index == 0:
        k = 3 if level is None else level
        v, f = noisy_icosphere(k, 0.05, rm)
        n = 100_000 if n_queries is None else n_queries
        nu = int(round(0.9 * n))
        q = np.concatenate([uniform_in_box(v, 1.2, nu, rq),
                            near_surface(v, f, n - nu, 0.01, rq)], 0)
        return _finish(WORKLOADS[0], v, f, q, 1.25, 0.0)
    if index == 1:
        k = 8 if level is None else level
        v, f = displaced_icosphere(k, 0.2, rm)
        n = 10_000_000 if n_queries is None else n_queries
        q = uniform_in_box(v, 1.5, n, rq)
        return _finish(WORKLOADS[1], v, f, q, 1.5, 0.01)
    if index == 2:
        g = 1024 if grid is None else grid
        v, f = fractal_heightfield(g, rm)
        n = 16_000_000 if n_queries is None else n_queries
        sigma = 0.01 * bbox_diagonal(v)
        q = gaussian_about_surface(v, f, n, sigma, rq)
        return _finish(WORKLOADS[2], v, f, q, 1.0, 0.12, meta={"sigma": sigma})
    if index == 3:
        k = 7 if level is None else level
        v, f = noisy_icosphere(k, 0.05, rm)
        n = 4_000_000 if n_queries is None else n_queries
        q = near_surface(v, f, n, 0.01, rq)
        w = rw.uniform(0.0, 1.0, size=n)
        return _finish(WORKLOADS[3], v, f, q, 1.25, 0.0, w=w)
    raise ValueError("workload 4 is a batch: use batch_workload()")


def _soup_streams(n: int):
    # children 5 and 6 of the root sequence: apart from the five workloads'
    child = np.random.SeedSequence(ROOT_SEED).spawn(7)[5]
    return [np.random.default_rng(s) for s in child.spawn(n)]


def triangle_soup(kind: str, level: int, rng):
    """The three versions of a closed surface the paper's soup test uses
    (Sec. 5, triangle soups): 'watertight' (a noisy icosphere), 'gapped'
    (every face with its own three vertices, shrunk to 80 % about its
    centroid, so no two faces touch) and 'penetrating' (own vertices, grown
    to 160 % and turned by up to 30 degrees about a random axis through the
    centroid, so neighbouring faces cut through each other)."""
    v, f = noisy_icosphere(level, 0.05, rng)
    if kind == "watertight":
        return v, f
    tri = v[f]                                   # (F, 3, 3)
    c = tri.mean(1, keepdims=True)
    if kind == "gapped":
        tri = c + 0.8 * (tri - c)
    elif kind == "penetrating":
        axis = rng.normal(size=(f.shape[0], 3))
        axis /= np.linalg.norm(axis, axis=1, keepdims=True)
        ang = rng.uniform(-math.pi / 6, math.pi / 6, size=f.shape[0])
        k = axis[:, None, :]
        p = 1.6 * (tri - c)
        cos, sin = np.cos(ang)[:, None, None], np.sin(ang)[:, None, None]
        # Rodrigues' rotation of every corner about the face's axis
        p = p * cos + np.cross(k, p) * sin + k * (p * k).sum(-1, keepdims=True) * (1 - cos)
        tri = c + p
    else:
        raise ValueError(kind)
    return tri.reshape(-1, 3), np.arange(3 * f.shape[0]).reshape(-1, 3)


def soup_workload(kind: str, level: int = 5, n_queries: int = 1_000_000):
    """Triangle-soup workload: level 5 gives 20,480 faces (the size of the
    paper's Bear model); half the queries uniform in the bbox scaled 1.2x,
    half within 0.01 x bbox diagonal of the surface."""
    rm, rq = _soup_streams(2)
    v, f = triangle_soup(kind, level, rm)
    nu = n_queries // 2
    q = np.concatenate([uniform_in_box(v, 1.2, nu, rq),
                        near_surface(v, f, n_queries - nu, 0.01 * bbox_diagonal(v), rq)], 0)
    return _finish(f"soup-{kind}-L{level}", v, f, q, 1.25, 0.02, meta={"kind": kind})


def triangulation_pair(n_queries: int = 1_000_000):
    """The same surface triangulated well and poorly (Sec. 5.5, Table 5):
    a noisy icosphere at level 5 (10,242 vertices, mean Q 0.74, no triangle
    with a smallest angle under 10 degrees) and a noisy latitude-longitude
    sphere of 31 rings of 320 vertices (9,922 vertices, mean Q 0.44, 21 % of
    its triangles under 10 degrees).  Both with radial noise 0.05; the same
    queries for both: half uniform in the bbox scaled 1.2x, half within
    0.01 x bbox diagonal of the icosphere."""
    child = np.random.SeedSequence(ROOT_SEED).spawn(10)[9]
    rg, rp, rq = [np.random.default_rng(s) for s in child.spawn(3)]
    vg, fg = noisy_icosphere(5, 0.05, rg)
    vp, fp = uv_sphere(32, 320, 0.05, rp)
    nu = n_queries // 2
    q = np.concatenate([uniform_in_box(vg, 1.2, nu, rq),
                        near_surface(vg, fg, n_queries - nu, 0.01 * bbox_diagonal(vg), rq)], 0)
    return (_finish("icosphere-L5-noise0.05", vg, fg, q, 1.25, 0.02),
            _finish("latlong-sphere-32x320-noise0.05", vp, fp, q, 1.25, 0.02))


def unique_edges(f):
    """Sorted unique (min, max) vertex pairs of the sides of triangles f."""
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], 0)
    return np.unique(np.sort(e, axis=1), axis=0)


def points_on_segments(v, s, n, radius, rng):
    """Uniform point of a length-weighted random segment plus a uniform
    offset in the ball of the given radius."""
    a, b = v[s[:, 0]], v[s[:, 1]]
    w = np.linalg.norm(b - a, axis=1)
    k = rng.choice(s.shape[0], size=n, p=w / w.sum())
    t = rng.uniform(size=(n, 1))
    p = a[k] + t * (b[k] - a[k])
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return p + d * (radius * rng.uniform(size=n) ** (1.0 / 3.0))[:, None]


def mixed_workload(mesh_level: int = 6, wire_level: int = 4, n_queries: int = 1_000_000):
    """Mixed segments and triangles (Sec. 5, mixed primitives): a noisy
    icosphere (the triangle mesh) beside the wireframe of a displaced one
    (segments only, no faces), as the paper combines a triangle mesh with
    another model's wireframe.  Half the queries uniform in the bbox scaled
    1.2x, a quarter near each part.  Returns the Mesh (tris = the triangles)
    and the segments as meta['segs'] (indices into verts)."""
    rm, rq = _soup_streams(2)[::-1]
    v1, f1 = noisy_icosphere(mesh_level, 0.05, rm)
    v2, f2 = displaced_icosphere(wire_level, 0.2, rm)
    v2 = 0.8 * v2 + np.array([2.2, 0.0, 0.0])
    segs = unique_edges(f2) + v1.shape[0]
    v = np.concatenate([v1, v2], 0)
    nu, nm = n_queries // 2, n_queries // 4
    q = np.concatenate([uniform_in_box(v, 1.2, nu, rq),
                        near_surface(v1, f1, nm, 0.02, rq),
                        points_on_segments(v, segs, n_queries - nu - nm, 0.02, rq)], 0)
    return _finish(f"mixed-L{mesh_level}-wire-L{wire_level}", v, f1, q, 1.25, 0.02,
                   meta={"segs": np.ascontiguousarray(segs, np.int32)})


def high_valence_fan(n_rim: int = 120, seed: int = 7):
    """A flat fan: an apex above the centre of n_rim nearly co-circular rim
    vertices (radius and height jittered by 2e-5), one triangle per rim
    side.  Every rim vertex is a Voronoi neighbour of the apex, so the
    apex's cell has about n_rim + 2 faces: a stress case for bounded work
    buffers (the builder's flooding hands such primitives to unbounded code).
    Queries: none (tables-only workload); domain 1.5x the bbox."""
    rng = np.random.default_rng(seed)
    th = 2 * math.pi * np.arange(n_rim) / n_rim
    r = 1 + rng.uniform(-2e-5, 2e-5, n_rim)
    rim = np.stack([r * np.cos(th), r * np.sin(th), rng.uniform(-2e-5, 2e-5, n_rim)], 1)
    v = np.concatenate([[[0.0, 0.0, 0.1]], rim], 0).astype(np.float32)
    f = np.array([[0, 1 + i, 1 + (i + 1) % n_rim] for i in range(n_rim)], np.int32)
    return Mesh(f"fan-{n_rim}", v, f, np.zeros((1, 3), np.float32), 1.5, 0.05, meta={})


def batch_workload(n_meshes: int = 64, tri_range=(1e3, 5e5), query_range=(1e4, 2e6),
                   query_scale: float = 1.0):
    """64 meshes of uneven size: a coin picks a noisy icosphere (level
    clamp(round(log4(T/20)), 3, 7)) or a jittered fractal height field
    (n = round(sqrt(T/2)) + 1) for a log-uniform triangle target T; query
    counts are log-uniform; half the queries are uniform in the bbox scaled
    1.2x and half lie within 0.01 * diagonal of the surface.
    ``query_scale`` shrinks the query counts for tests."""
    child = np.random.SeedSequence(ROOT_SEED).spawn(5)[4]
    rp = np.random.default_rng(child.spawn(1)[0])
    meshes = []
    specs = []
    for i in range(n_meshes):
        T = math.exp(rp.uniform(math.log(tri_range[0]), math.log(tri_range[1])))
        N = int(round(math.exp(rp.uniform(math.log(query_range[0]),
                                          math.log(query_range[1])))))
        coin = rp.uniform() < 0.5
        specs.append((T, N, coin))
    subs = child.spawn(1 + n_meshes)[1:]
    for i, (T, N, coin) in enumerate(specs):
        rm, rq = [np.random.default_rng(s) for s in subs[i].spawn(2)]
        if coin:
            k = int(min(7, max(3, round(math.log(T / 20.0, 4)))))
            v, f = noisy_icosphere(k, 0.05, rm)
            name = f"icosphere-L{k}"
        else:
            g = int(round(math.sqrt(T / 2.0))) + 1
            v, f = fractal_heightfield(g, rm)
            name = f"heightfield-{g}"
        n = max(1, int(round(N * query_scale)))
        nu = n // 2
        diag = bbox_diagonal(v)
        q = np.concatenate([uniform_in_box(v, 1.2, nu, rq),
                            near_surface(v, f, n - nu, 0.01 * diag, rq)], 0)
        meshes.append(_finish(f"batch{i:02d}-{name}", v, f, q, 1.25, 0.02))
    return meshes


def triangle_quality(v, f):
    """Q(t) = 6/sqrt(3) * S / (p * h) (S area, p half-perimeter, h longest
    edge) and the share of triangles whose smallest angle is below 10 degrees
    (mesh-quality statistics of Sec. 5.5)."""
    v = v.astype(np.float64)
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    la = np.linalg.norm(b - c, axis=1)
    lb = np.linalg.norm(c - a, axis=1)
    lc = np.linalg.norm(a - b, axis=1)
    S = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    p = 0.5 * (la + lb + lc)
    h = np.maximum(np.maximum(la, lb), lc)
    Q = 6.0 / math.sqrt(3.0) * S / (p * h)
    cosA = np.clip((lb ** 2 + lc ** 2 - la ** 2) / (2 * lb * lc), -1, 1)
    cosB = np.clip((la ** 2 + lc ** 2 - lb ** 2) / (2 * la * lc), -1, 1)
    cosC = np.clip((la ** 2 + lb ** 2 - lc ** 2) / (2 * la * lb), -1, 1)
    amin = np.degrees(np.arccos(np.maximum(np.maximum(cosA, cosB), cosC)))
    return float(Q.mean()), float((amin < 10.0).mean())
