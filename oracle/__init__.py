"""Plain FP64 CPU oracle of the P2M point-to-mesh method.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2308_16084_gb300``) never imports it and shares no
code with it.

The C part (``p2m_oracle.c``) holds the paper's method and the brute-force
definition; this module compiles it with gcc on first use, marshals numpy
arrays through ctypes, and adds the analytic gradient (Sec. 4.1 defines the
closest point; the gradient follows from it, see ``gradient``).

Functions whose result has no independent pin say so in their docstring
("parity unpinned"); everything else is pinned by the ``-m "not gpu"``
tests (brute force on tiny meshes, closed forms, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "p2m_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libp2m_oracle.so")
_lock = threading.Lock()
_lib = None

VERTEX, EDGE, FACE = 0, 1, 2
STATUS = {0: "ok", 1: "bad argument", 2: "index out of range", 3: "repeated index",
          4: "duplicate vertex", 5: "unreferenced vertex", 6: "non-finite coordinate",
          7: "out of memory", 8: "no triangles or segments"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (plain C, no target
    specific flags, FMA contraction off so x86 and Arm agree)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and \
            os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                          os.path.getmtime(os.path.join(_HERE, "p2m_oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [P, i64, P, i64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, P]
            lib.orc_create_mixed.restype = P
            lib.orc_create_mixed.argtypes = [P, i64, P, i64, P, i64, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, P]
            lib.orc_create_ex.restype = P
            lib.orc_create_ex.argtypes = [P, i64, P, i64, P, i64, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, P, P, P]
            lib.orc_destroy.argtypes = [P]
            lib.orc_info.argtypes = [P, P, P]
            lib.orc_edges.argtypes = [P, P]
            lib.orc_bruteforce.argtypes = [P, P, i64, ctypes.c_int] + [P] * 7
            lib.orc_query.argtypes = [P, P, i64, ctypes.c_int, ctypes.c_int] + [P] * 8
            lib.orc_kdt_nn.argtypes = [P, P, i64, P, P]
            lib.orc_table.argtypes = [P, P, P, P, P]
            lib.orc_cell_neighbors.argtypes = [P, ctypes.c_int32, P, ctypes.c_int]
            lib.orc_cell_corners.argtypes = [P, ctypes.c_int32, P, ctypes.c_int]
            lib.orc_cell_volume.restype = ctypes.c_double
            lib.orc_cell_volume.argtypes = [P, ctypes.c_int32]
            lib.orc_intercepts.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P]
            lib.orc_convexpoly.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P,
                                            ctypes.c_int]
            lib.orc_clip_box.argtypes = [P, P, P, ctypes.c_int, P, ctypes.c_int]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def default_threads() -> int:
    return os.cpu_count() or 1


def delaunay_neighbors(V):
    """Delaunay neighbours of every vertex as CSR (offsets int64, ids int32),
    from qhull's 3-D Delaunay triangulation (scipy.spatial.Delaunay, a
    library step like the TetGen call of the paper's preprocessing, Sec. 5).
    The bisectors of a vertex's Delaunay neighbours bound its Voronoi cell."""
    from scipy.spatial import Delaunay
    d = Delaunay(np.asarray(V, np.float64))
    indptr, idx = d.vertex_neighbor_vertices
    off = np.ascontiguousarray(indptr, np.int64)
    ids = np.ascontiguousarray(idx, np.int32)
    return off, ids


class OracleMesh:
    """Oracle state for one mesh: topology, KD tree and (optionally) the
    Voronoi cells, the interception table and the Region boxes (Alg. A.1).

    Vertices are float32 inputs widened exactly to float64 (float64 input is
    kept as it is, for finite-difference tests)."""

    def __init__(self, verts, tris, domain_scale=10.0, domain_margin=0.0,
                 delta_rel=4e-6, build_tables=True, threads=None, segs=None,
                 voronoi="certified"):
        """voronoi: "certified" (k-nearest seeding, every cell corner
        certified by a nearest-vertex search) or "delaunay" (the cell of v
        clipped by the bisectors of its Delaunay neighbours from qhull, for
        large meshes).  Either gives the Voronoi cells of V clipped to D."""
        self._lib = _load()
        self.V = self._widen(verts)
        self.F = np.ascontiguousarray(np.asarray(tris, np.int32).reshape(-1, 3))
        self.S = np.ascontiguousarray(
            np.zeros((0, 2), np.int32) if segs is None else np.asarray(segs, np.int32).reshape(-1, 2))
        self.threads = default_threads() if threads is None else int(threads)
        if voronoi not in ("certified", "delaunay"):
            raise ValueError(f"oracle: unknown Voronoi construction {voronoi!r}")
        cand_off = cand = None
        self.delaunay_s = 0.0
        if build_tables and voronoi == "delaunay":
            import time
            t0 = time.perf_counter()
            cand_off, cand = delaunay_neighbors(self.V)
            self.delaunay_s = time.perf_counter() - t0
        st = ctypes.c_int(0)
        self._h = self._lib.orc_create_ex(
            _p(self.V), self.V.shape[0], _p(self.F), self.F.shape[0], _p(self.S),
            self.S.shape[0], float(domain_scale), float(domain_margin), float(delta_rel),
            int(bool(build_tables)), self.threads, _p(cand_off), _p(cand), ctypes.byref(st))
        self.status = st.value
        if not self._h:
            raise ValueError(f"oracle: invalid mesh ({STATUS.get(st.value, st.value)})")
        info = np.zeros(16, np.int64)
        dom = np.zeros(7, np.float64)
        self._lib.orc_info(self._h, _p(info), _p(dom))
        self.nv, self.nf, self.ne, self.n_entries = (int(x) for x in info[:4])
        self.n_degenerate = int(info[4])
        self.n_neighbor_pairs = int(info[5])
        self.n_inspections = int(info[6])
        self.times_ms = {"topology": int(info[7]), "kdt": int(info[8]),
                         "voronoi": int(info[9]), "inspection": int(info[10])}
        self.domain_lo = dom[:3].copy()
        self.domain_hi = dom[3:6].copy()
        self.delta = float(dom[6])
        self.has_tables = bool(build_tables)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # ---------------------------------------------------------------- topology
    def edges(self):
        """Canonical edge list: unique (min, max) vertex pairs, sorted."""
        E = np.zeros((self.ne, 2), np.int32)
        self._lib.orc_edges(self._h, _p(E))
        return E

    # ------------------------------------------------------------------ results
    def _alloc(self, n):
        return dict(dist=np.zeros(n), cp=np.zeros((n, 3)), ptype=np.zeros(n, np.int32),
                    pid=np.zeros(n, np.int64), bv=np.zeros((n, 3), np.int32),
                    bw=np.zeros((n, 3)))

    @staticmethod
    def _widen(a):
        """float32 inputs are widened exactly; float64 inputs (finite
        difference tests only) are taken as they are."""
        a = np.asarray(a)
        if a.dtype != np.float64:
            a = a.astype(np.float32).astype(np.float64)
        return np.ascontiguousarray(a.reshape(-1, 3))

    _q = _widen

    def bruteforce(self, q, threads=None):
        """Plain definition: min over all vertices, open edges and open
        faces of the gated distance (Sec. 4.1; gating of Alg. A.2).  Also
        returns ``second``: the best distance over every other primitive."""
        q = self._q(q)
        n = q.shape[0]
        r = self._alloc(n)
        r["second"] = np.zeros(n)
        self._lib.orc_bruteforce(self._h, _p(q), n, self.threads if threads is None else threads,
                                 _p(r["dist"]), _p(r["cp"]), _p(r["ptype"]), _p(r["pid"]),
                                 _p(r["bv"]), _p(r["bw"]), _p(r["second"]))
        return r

    def query(self, q, use_boxes=False, threads=None, counters=False):
        """Alg. A.2: KD-tree nearest vertex, then its interception list."""
        if not self.has_tables:
            raise RuntimeError("oracle built without tables")
        q = self._q(q)
        n = q.shape[0]
        r = self._alloc(n)
        r["nn"] = np.zeros(n, np.int32)
        cnt = np.zeros((n, 4), np.int64) if counters else None
        self._lib.orc_query(self._h, _p(q), n, self.threads if threads is None else threads,
                            int(bool(use_boxes)), _p(r["dist"]), _p(r["cp"]), _p(r["ptype"]),
                            _p(r["pid"]), _p(r["bv"]), _p(r["bw"]), _p(r["nn"]), _p(cnt))
        if counters:
            r["counters"] = cnt
        return r

    def kdt_nn(self, q):
        q = self._q(q)
        n = q.shape[0]
        nn = np.zeros(n, np.int32)
        vis = np.zeros(n, np.int64)
        self._lib.orc_kdt_nn(self._h, _p(q), n, _p(nn), _p(vis))
        return nn, vis

    # ------------------------------------------------------------------ tables
    def table(self):
        """Interception table as CSR: offsets (V+1), types, ids, boxes (n,6)."""
        off = np.zeros(self.nv + 1, np.int64)
        t = np.zeros(self.n_entries, np.int32)
        i = np.zeros(self.n_entries, np.int32)
        b = np.zeros((self.n_entries, 6))
        self._lib.orc_table(self._h, _p(off), _p(t), _p(i), _p(b))
        return off, t, i, b

    def cell_neighbors(self, v):
        buf = np.zeros(1024, np.int32)
        k = self._lib.orc_cell_neighbors(self._h, int(v), _p(buf), 1024)
        return buf[:k].copy()

    def cell_corners(self, v):
        buf = np.zeros((4096, 3))
        k = self._lib.orc_cell_corners(self._h, int(v), _p(buf), 4096)
        return buf[:k].copy()

    def cell_volume(self, v):
        return float(self._lib.orc_cell_volume(self._h, int(v)))

    def convexpoly(self, v, ptype, pid):
        """Corners of ConvexPoly(v,p) = Cell(v) ∩ Space-perp(p) (widened)."""
        buf = np.zeros((4096, 3))
        k = self._lib.orc_convexpoly(self._h, int(v), int(ptype), int(pid), _p(buf), 4096)
        return buf[:k].copy()

    def intercepts(self, v, ptype, pid):
        box = np.zeros(6)
        nc = ctypes.c_int32(0)
        r = self._lib.orc_intercepts(self._h, int(v), int(ptype), int(pid), _p(box),
                                     ctypes.byref(nc))
        return bool(r == 1), box, int(nc.value)


def clip_box(lo, hi, planes):
    """Corners of the box [lo,hi] cut by half-spaces n.x <= c (rows n,c)."""
    lib = _load()
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    pl = np.ascontiguousarray(np.asarray(planes, np.float64).reshape(-1, 4))
    out = np.zeros((4096, 3))
    k = lib.orc_clip_box(_p(lo), _p(hi), _p(pl), pl.shape[0], _p(out), 4096)
    return out[:k].copy()


def gradient(q, result, grad_dist=None):
    """Analytic gradient of d(q) = |q - c(q)| at the closest point c.

    dd/dq = (q - c)/d.  For the vertices of the closest primitive, with c =
    sum_k b_k v_k, dd/dv_k = -b_k (q - c)/d: by the envelope argument the
    change of the optimal barycentric weights moves c inside the primitive,
    orthogonally to q - c, so only the explicit dependence remains.  (The
    paper defines no gradient; this is the derivative of its distance.)
    Returns (grad_q (n,3), list of (vertex ids (n,3), grad (n,3,3))).
    """
    q = np.asarray(q, np.float64).reshape(-1, 3)
    cp = result["cp"]
    d = result["dist"]
    g = np.ones(q.shape[0]) if grad_dist is None else np.asarray(grad_dist, np.float64)
    u = (q - cp) / d[:, None]
    gq = g[:, None] * u
    gv = -(g[:, None, None] * result["bw"][:, :, None]) * u[:, None, :]
    return gq, result["bv"], gv
