"""GB300 point-to-mesh distance queries (query stage of P2M, Zong et al.,
ACM TOG 2023) behind the C ABI of ``libp2m.so`` (include/p2m.h).

This module only marshals arguments: every step of the query runs in the
library's CUDA kernels, and the preprocessing in its host builder.  PyTorch
supplies device memory and streams.  There is no fallback: if the library is
missing, importing this package raises ``ImportError``; on a machine without
a GPU, handles can still be built (tables only) but queries raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._lib import LIB_PATH, P2MError, check, lib  # noqa: F401

VERTEX, EDGE, FACE = 0, 1, 2
Q_OUTSIDE_DOMAIN, Q_NONFINITE = 1, 2


class BuildOpts(ctypes.Structure):
    """p2m_build_opts of include/p2m.h."""
    _fields_ = [("domain_scale", ctypes.c_float), ("domain_margin", ctypes.c_float),
                ("delta_rel", ctypes.c_float), ("host_threads", ctypes.c_int),
                ("device_assist", ctypes.c_int), ("leaf_size", ctypes.c_int)]


class MeshDesc(ctypes.Structure):
    """p2m_mesh of include/p2m.h (host pointers and counts)."""
    _fields_ = [("verts", ctypes.c_void_p), ("n_verts", ctypes.c_int64),
                ("tris", ctypes.c_void_p), ("n_tris", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    """p2m_tuning of include/p2m.h: the query path's launch configuration."""
    _fields_ = [("sort_bits", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("warp_cooperative", ctypes.c_int), ("nn_walk", ctypes.c_int),
                ("chunked", ctypes.c_int), ("group_by_vertex", ctypes.c_int),
                ("sort_key", ctypes.c_int), ("lanes_per_query", ctypes.c_int),
                ("streams", ctypes.c_int)]


class BatchIO(ctypes.Structure):
    """p2m_batch_io of include/p2m.h: one mesh's device buffers in a batch."""
    _fields_ = [("q", ctypes.c_void_p), ("n", ctypes.c_int64), ("dist", ctypes.c_void_p),
                ("closest", ctypes.c_void_p), ("prim_id", ctypes.c_void_p),
                ("prim_type", ctypes.c_void_p)]


class BatchTuning(ctypes.Structure):
    """p2m_batch_tuning of include/p2m.h."""
    _fields_ = [("sort_bits", ctypes.c_int), ("tile", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("grid_ctas", ctypes.c_int),
                ("group_by_vertex", ctypes.c_int), ("lanes_per_query", ctypes.c_int)]


def _stream(stream=None):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return ctypes.c_void_p(None)  # the library reports the missing device
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class P2M:
    """A preprocessed mesh on the current CUDA device.

    ``P2M(verts, tris, domain_scale=10, domain_margin=0, delta_rel=4e-6,
    host_threads=0, device_assist=3, leaf_size=8)`` runs the paper's
    preprocessing (Alg. A.1) through ``p2m_build``.  ``verts`` (V,3) float32
    and ``tris`` (F,3) int32 may be numpy arrays or CPU tensors.
    ``device_assist``: False/0 host only, True/1 Voronoi-cell certification
    on the GPU, 2 the flooding (Alg. 1) on the GPU as well, 3 (default) the
    whole Voronoi-cell stage too; every setting gives the same layout."""

    def __init__(self, verts=None, tris=None, *, segs=None, domain_scale=10.0,
                 domain_margin=0.0, delta_rel=4e-6, host_threads=0, device_assist=3,
                 leaf_size=8, _handle=None):
        self._h = None
        if _handle is not None:
            self._h = _handle
        else:
            V = np.ascontiguousarray(np.asarray(verts, dtype=np.float32).reshape(-1, 3))
            F = np.ascontiguousarray(np.asarray(
                np.zeros((0, 3)) if tris is None else tris, dtype=np.int32).reshape(-1, 3))
            desc = MeshDesc(V.ctypes.data, V.shape[0], F.ctypes.data, F.shape[0])
            assist = int(device_assist)
            if assist not in (0, 1, 2, 3):
                raise ValueError("device_assist must be 0, 1, 2 or 3")
            opts = BuildOpts(domain_scale, domain_margin, delta_rel, host_threads, assist,
                             leaf_size)
            h = ctypes.c_void_p()
            if segs is None:
                check(lib.p2m_build(ctypes.byref(desc), ctypes.byref(opts), ctypes.byref(h)),
                      "p2m_build")
            else:
                S = np.ascontiguousarray(np.asarray(segs, dtype=np.int32).reshape(-1, 2))
                check(lib.p2m_build_mixed(ctypes.byref(desc), S.ctypes.data, S.shape[0],
                                          ctypes.byref(opts), ctypes.byref(h)),
                      "p2m_build_mixed")
            self._h = h
        st = self.stats()
        self.n_verts, self.n_tris, self.n_edges = st["n_verts"], st["n_tris"], st["n_edges"]

    @classmethod
    def load(cls, path):
        """A layout saved by save(), checked (checksum and every index the
        kernels follow) and uploaded to the current device when there is
        one."""
        h = ctypes.c_void_p()
        check(lib.p2m_load(os.fsencode(path), ctypes.byref(h)), "p2m_load")
        return cls(_handle=h)

    def save(self, path):
        """Write the built layout to `path` (versioned, checksummed)."""
        check(lib.p2m_save(self._h, os.fsencode(path)), "p2m_save")

    def close(self):
        """Release the handle and its device memory (idempotent)."""
        if self._h:
            lib.p2m_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- info
    def stats(self):
        """Statistics of the built layout (p2m_stats): sizes, table entries,
        longest list, device bytes, KD tree, neighbour pairs, flooding
        inspections, build times in ms, certification rounds and queries,
        degenerate faces."""
        out = (ctypes.c_int64 * 16)()
        check(lib.p2m_stats(self._h, out), "p2m_stats")
        keys = ["n_verts", "n_tris", "n_edges", "n_entries", "max_list", "device_bytes",
                "kd_leaves", "kd_depth", "neighbour_pairs", "inspections", "build_ms",
                "cells_ms", "inspect_ms", "cert_rounds", "cert_queries", "n_degenerate"]
        return dict(zip(keys, list(out)))

    def flood_stats(self):
        """How the build's flooding was split: primitives flooded on the
        device, by the host's bounded core, by its unbounded code."""
        out = (ctypes.c_int64 * 3)()
        check(lib.p2m_flood_stats(self._h, out), "p2m_flood_stats")
        return {"device": out[0], "host_bounded": out[1], "host_unbounded": out[2]}

    def cell_stats(self):
        """How the build's Voronoi cells were split (made on the device, on
        the host) and whether the table was packed on the device."""
        out = (ctypes.c_int64 * 3)()
        check(lib.p2m_cell_stats(self._h, out), "p2m_cell_stats")
        return {"device": out[0], "host": out[1], "packed_on_device": out[2]}

    def domain(self):
        """(lo, hi, delta): the query domain D and the widening margin."""
        out = (ctypes.c_float * 7)()
        check(lib.p2m_domain(self._h, out), "p2m_domain")
        return np.array(out[:3]), np.array(out[3:6]), float(out[6])

    def edges(self):
        """The canonical edge list, (E,2) int32: unique (min, max) vertex
        pairs in lexicographic order; edge ids index it."""
        n = ctypes.c_int64()
        check(lib.p2m_get_edges(self._h, None, ctypes.byref(n)), "p2m_get_edges")
        E = np.zeros((n.value, 2), np.int32)
        check(lib.p2m_get_edges(self._h, E.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)),
              "p2m_get_edges")
        return E

    def interception_list(self, v):
        """(types, ids, boxes) of vertex v's interception list."""
        n = ctypes.c_int64()
        check(lib.p2m_get_list(self._h, int(v), None, None, None, 0, ctypes.byref(n)),
              "p2m_get_list")
        t = np.zeros(n.value, np.int32)
        i = np.zeros(n.value, np.int32)
        b = np.zeros((n.value, 6), np.float32)
        check(lib.p2m_get_list(self._h, int(v), t.ctypes.data_as(ctypes.c_void_p),
                               i.ctypes.data_as(ctypes.c_void_p),
                               b.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)),
              "p2m_get_list")
        return t, i, b

    # --------------------------------------------------------------- tuning
    @property
    def tuning(self):
        """The query launch configuration as a dict (p2m_get_tuning);
        assigning a dict with some of its fields changes those
        (p2m_set_tuning range-checks them)."""
        t = Tuning()
        check(lib.p2m_get_tuning(self._h, ctypes.byref(t)), "p2m_get_tuning")
        return {"sort_bits": t.sort_bits, "block_threads": t.block_threads,
                "warp_cooperative": t.warp_cooperative, "nn_walk": t.nn_walk,
                "chunked": t.chunked, "group_by_vertex": t.group_by_vertex,
                "sort_key": t.sort_key, "lanes_per_query": t.lanes_per_query,
                "streams": t.streams}

    @tuning.setter
    def tuning(self, d):
        cur = self.tuning
        cur.update(d)
        t = Tuning(cur["sort_bits"], cur["block_threads"], cur["warp_cooperative"],
                   cur["nn_walk"], cur["chunked"], cur["group_by_vertex"], cur["sort_key"],
                   cur["lanes_per_query"], cur["streams"])
        check(lib.p2m_set_tuning(self._h, ctypes.byref(t)), "p2m_set_tuning")

    def autotune(self, q, reps=3, stream=None):
        """Time the launch configurations on the (N,3) CUDA queries q and
        keep the fastest; returns its time in ms."""
        ms = ctypes.c_float()
        check(lib.p2m_autotune(self._h, _ptr(q), q.shape[0], reps, _stream(stream),
                               ctypes.byref(ms)), "p2m_autotune")
        return ms.value

    def set_timing(self, enable=True):
        """Record CUDA events around every phase of the following queries
        (read them with timing_summary())."""
        check(lib.p2m_set_timing(self._h, int(bool(enable))), "p2m_set_timing")

    def timing_summary(self):
        """Per-phase totals of the queries made since the previous summary
        (timing enabled): dict with calls, sort_ms, nn_ms, regroup_ms,
        list_ms, output_ms (the one-pass kernel counts as list_ms)."""
        out = (ctypes.c_double * 6)()
        check(lib.p2m_timing_summary(self._h, out), "p2m_timing_summary")
        return {"calls": int(out[0]), "sort_ms": float(out[1]), "nn_ms": float(out[2]),
                "regroup_ms": float(out[3]), "list_ms": float(out[4]),
                "output_ms": float(out[5])}

    def counters(self, q, stream=None):
        """Work totals of a query batch: internal KD nodes visited, vertices
        examined, list entries scanned, edges tested, faces tested, chunk
        boxes tested."""
        out = (ctypes.c_int64 * 6)()
        check(lib.p2m_query_counters(self._h, _ptr(q), q.shape[0], out, _stream(stream)),
              "p2m_query_counters")
        return dict(zip(["nodes", "points", "entries", "edges", "faces", "chunks"], list(out)))

    def reserve(self, n):
        """Allocate the query scratch for batches of up to n points now, so
        that later queries of that size allocate nothing."""
        check(lib.p2m_reserve(self._h, int(n)), "p2m_reserve")

    # ---------------------------------------------------------------- query
    def query(self, q, *, closest=True, prim_type=True, save=False, status=False,
              out=None, stream=None):
        """Closest-point query of a (N,3) float32 CUDA tensor.  Returns a dict
        of CUDA tensors: dist, prim_id and optionally closest, prim_type,
        save (N,4: typed id bits + barycentric weights), status."""
        import torch
        assert q.is_cuda and q.dtype == torch.float32 and q.is_contiguous()
        n = q.shape[0]
        dev = q.device
        r = out if out is not None else {}
        if "dist" not in r:
            r["dist"] = torch.empty(n, dtype=torch.float32, device=dev)
            r["prim_id"] = torch.empty(n, dtype=torch.int32, device=dev)
            if closest:
                r["closest"] = torch.empty(n, 3, dtype=torch.float32, device=dev)
            if prim_type:
                r["prim_type"] = torch.empty(n, dtype=torch.uint8, device=dev)
            if save:
                r["save"] = torch.empty(n, 4, dtype=torch.float32, device=dev)
            if status:
                r["status"] = torch.empty(n, dtype=torch.uint8, device=dev)
        check(lib.p2m_query(self._h, _ptr(q), n, _ptr(r["dist"]), _ptr(r.get("closest")),
                            _ptr(r["prim_id"]), _ptr(r.get("prim_type")), _ptr(r.get("save")),
                            _ptr(r.get("status")), _stream(stream)), "p2m_query")
        return r

    def nearest_vertex(self, q, stream=None):
        """Nearest vertex id of each point of a (N,3) float32 CUDA tensor."""
        import torch
        out = torch.empty(q.shape[0], dtype=torch.int32, device=q.device)
        check(lib.p2m_nearest_vertex(self._h, _ptr(q), q.shape[0], _ptr(out), _stream(stream)),
              "p2m_nearest_vertex")
        return out

    def query_host(self, q, dist, prim_id, closest=None, prim_type=None, stream=None):
        """End-to-end query on HOST buffers (numpy or pinned CPU tensors):
        copies in, queries, copies out, synchronises."""
        def p(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.data_ptr())
            return a.ctypes.data_as(ctypes.c_void_p)
        check(lib.p2m_query_host(self._h, p(q), int(q.shape[0]), p(dist), p(closest),
                                 p(prim_id), p(prim_type), _stream(stream)), "p2m_query_host")

    def pipeline(self, max_n, depth=2):
        """A P2MPipe of `depth` slots for host-buffer batches of up to max_n
        queries."""
        return P2MPipe(self, max_n, depth)

    def update_vertices(self, verts, refresh_seed_grid=False, stream=None):
        """Move the vertices to `verts` ((V,3) float32 CUDA tensor, original
        order): KD tree, neighbour positions and edge and face records are
        recomputed on the device; the interception tables stay those of the
        build (p2m_update_vertices).  refresh_seed_grid also recomputes the
        seed grids of the nearest-vertex walk."""
        _update_vertices(self, verts, refresh_seed_grid, stream)

    def backward(self, q, res, grad_dist, grad_q=True, grad_verts=None, stream=None):
        """Gradients of sum(grad_dist * dist): returns (grad_q, grad_verts);
        grad_verts is accumulated into the given (V,3) tensor if passed."""
        import torch
        n = q.shape[0]
        gq = torch.empty(n, 3, dtype=torch.float32, device=q.device) if grad_q else None
        check(lib.p2m_backward(self._h, _ptr(q), _ptr(res["dist"]), _ptr(res["closest"]),
                               _ptr(res["save"]), _ptr(grad_dist), n, _ptr(gq), _ptr(grad_verts),
                               _stream(stream)), "p2m_backward")
        return gq, grad_verts


def _update_vertices(mesh, verts, refresh_seed_grid=False, stream=None):
    import torch
    assert verts.is_cuda and verts.dtype == torch.float32, "verts: float32 CUDA tensor"
    v = verts.detach().contiguous()
    assert v.shape == (mesh.n_verts, 3), f"verts: expected ({mesh.n_verts}, 3)"
    check(lib.p2m_update_vertices(mesh._h, _ptr(v), mesh.n_verts, int(bool(refresh_seed_grid)),
                                  _stream(stream)), "p2m_update_vertices")
    return v


def _torch_autograd():
    import torch

    class P2MFunction(torch.autograd.Function):
        """d = dist(q, mesh) with gradients to the query points and to the
        vertex positions.  The forward saves only (typed primitive id,
        barycentric weights), the closest points and the distances; the
        backward kernel recomputes nothing of the query."""

        @staticmethod
        def forward(ctx, q, verts, mesh):
            # the query runs on the positions it is given: the mesh's vertex
            # records are refreshed from `verts` first (p2m_update_vertices;
            # the interception tables stay those of the build)
            keep = _update_vertices(mesh, verts)
            r = mesh.query(q.contiguous(), closest=True, prim_type=False, save=True)
            ctx.keep = keep  # the refresh's source stays alive until its kernels ran
            ctx.mesh = mesh
            ctx.n_verts = verts.shape[0]
            ctx.save_for_backward(q, r["dist"], r["closest"], r["save"])
            ctx.mark_non_differentiable(r["prim_id"])
            return r["dist"], r["prim_id"]

        @staticmethod
        def backward(ctx, gdist, _gid):
            q, dist, cp, save = ctx.saved_tensors
            gv = None
            if ctx.needs_input_grad[1]:
                gv = torch.zeros(ctx.n_verts, 3, dtype=torch.float32, device=q.device)
            gq, gv = ctx.mesh.backward(q, {"dist": dist, "closest": cp, "save": save},
                                       gdist.contiguous(), grad_q=ctx.needs_input_grad[0],
                                       grad_verts=gv)
            return gq, gv, None

    return P2MFunction


_autograd_cls = None


def distance(q, verts, mesh):
    """Differentiable point-to-mesh distance: returns (dist, prim_id).  The
    query runs on the vertex positions `verts` (the mesh's geometry is
    refreshed from them, its interception tables are the build's), and
    gradients flow to q and to verts."""
    global _autograd_cls
    if _autograd_cls is None:
        _autograd_cls = _torch_autograd()
    return _autograd_cls.apply(q, verts, mesh)


def _host_ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


class P2MPipe:
    """Pipelined queries on HOST buffers: each submit() copies a batch in,
    queries it and copies the results out on the next of `depth` slots
    (own stream and scratch), without waiting for the other slots, so the
    copies of one batch overlap the kernels of another.  Buffers should be
    pinned; they belong to the pipe until wait()."""

    def __init__(self, mesh, max_n, depth=2):
        self.mesh = mesh  # keeps the handle alive
        p = ctypes.c_void_p()
        check(lib.p2m_pipe_create(mesh._h, int(max_n), int(depth), ctypes.byref(p)),
              "p2m_pipe_create")
        self._p = p

    def submit(self, q, dist, prim_id, closest=None, prim_type=None):
        """Queue one batch: q (N,3) float32 in, dist / prim_id (and closest,
        prim_type when given) out, all host buffers."""
        check(lib.p2m_pipe_submit(self._p, _host_ptr(q), int(q.shape[0]), _host_ptr(dist),
                                  _host_ptr(closest), _host_ptr(prim_id), _host_ptr(prim_type)),
              "p2m_pipe_submit")

    def submit_device(self, q, out, stream=None):
        """Queue one batch on DEVICE tensors: q (N,3) float32, out a dict with
        dist and prim_id (and closest, prim_type) CUDA tensors.  It starts
        after the work enqueued so far on `stream` (default: the current
        one); batches on different slots may run concurrently."""
        check(lib.p2m_pipe_submit_device(self._p, _ptr(q), int(q.shape[0]), _ptr(out["dist"]),
                                         _ptr(out.get("closest")), _ptr(out["prim_id"]),
                                         _ptr(out.get("prim_type")), _stream(stream)),
              "p2m_pipe_submit_device")

    def join(self, stream=None):
        """Make `stream` (default: the current one) wait for every batch
        submitted so far."""
        check(lib.p2m_pipe_join(self._p, _stream(stream)), "p2m_pipe_join")

    def wait(self):
        """Block until every submitted batch's results are in its buffers."""
        check(lib.p2m_pipe_wait(self._p), "p2m_pipe_wait")

    def close(self):
        """Release the pipe's slots (idempotent)."""
        if getattr(self, "_p", None):
            lib.p2m_pipe_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class P2MBatch:
    """Many meshes and their query sets in one persistent launch."""

    def __init__(self, meshes, queries, closest=False, prim_type=False):
        import torch
        self.meshes = list(meshes)
        self.queries = list(queries)
        self.out = []
        ios = (BatchIO * len(self.meshes))()
        for k, (m, q) in enumerate(zip(self.meshes, self.queries)):
            n = q.shape[0]
            r = {"dist": torch.empty(n, dtype=torch.float32, device=q.device),
                 "prim_id": torch.empty(n, dtype=torch.int32, device=q.device)}
            if closest:
                r["closest"] = torch.empty(n, 3, dtype=torch.float32, device=q.device)
            if prim_type:
                r["prim_type"] = torch.empty(n, dtype=torch.uint8, device=q.device)
            self.out.append(r)
            ios[k] = BatchIO(q.data_ptr(), n, r["dist"].data_ptr(),
                             r["closest"].data_ptr() if closest else None,
                             r["prim_id"].data_ptr(),
                             r["prim_type"].data_ptr() if prim_type else None)
        hs = (ctypes.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        b = ctypes.c_void_p()
        check(lib.p2m_batch_create(hs, ios, len(self.meshes), ctypes.byref(b)), "p2m_batch_create")
        self._b = b

    def run(self, stream=None):
        """One launch over every mesh's queries; returns the per-mesh output
        dicts (CUDA tensors, filled when the stream reaches them)."""
        check(lib.p2m_batch_run(self._b, _stream(stream)), "p2m_batch_run")
        return self.out

    def check(self, stream=None):
        """Synchronise and raise (P2M_ERR_QUEUE_TIMEOUT) if the device error
        word of the last runs reports a malformed work item."""
        check(lib.p2m_batch_check(self._b, _stream(stream)), "p2m_batch_check")

    def autotune(self, reps=3, stream=None):
        """Time the batch launch configurations and keep the fastest;
        returns its time in ms."""
        ms = ctypes.c_float()
        check(lib.p2m_batch_autotune(self._b, reps, _stream(stream), ctypes.byref(ms)),
              "p2m_batch_autotune")
        return ms.value

    @property
    def tuning(self):
        """The batch launch configuration as a dict; assign a dict with some
        of its fields to change those."""
        t = BatchTuning()
        check(lib.p2m_batch_get_tuning(self._b, ctypes.byref(t)), "p2m_batch_get_tuning")
        return {"sort_bits": t.sort_bits, "tile": t.tile, "block_threads": t.block_threads,
                "grid_ctas": t.grid_ctas, "group_by_vertex": t.group_by_vertex,
                "lanes_per_query": t.lanes_per_query}

    @tuning.setter
    def tuning(self, d):
        cur = self.tuning
        cur.update(d)
        t = BatchTuning(cur["sort_bits"], cur["tile"], cur["block_threads"], cur["grid_ctas"],
                        cur["group_by_vertex"], cur["lanes_per_query"])
        check(lib.p2m_batch_set_tuning(self._b, ctypes.byref(t)), "p2m_batch_set_tuning")

    def close(self):
        """Release the batch (idempotent); the meshes stay valid."""
        if getattr(self, "_b", None):
            lib.p2m_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
