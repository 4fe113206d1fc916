// p2m_api.cu -- the extern "C" boundary of libp2m.so (include/p2m.h).
//
// Host glue only: argument checks, device memory of the handle, uploads,
// and launches of the kernels in kernels.cu.  No query arithmetic happens
// here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/p2m.h"
#include "builder.h"
#include "cells.h"
#include "certify.h"
#include "flood.h"
#include "pack.h"
#include "quant.h"
#include "kernels.h"
#include "quant.h"

// seed grid of the Voronoi walk: up to 256 cells per vertex, G <= 512
// (512^3 cells = 512 MiB); measured on the 1.3M-triangle displaced sphere,
// G = 512 walks 5 % faster than G = 256
#ifndef P2M_GRID_PER_VERTEX
#define P2M_GRID_PER_VERTEX 256
#endif
#ifndef P2M_GRID_MAX_BITS
#define P2M_GRID_MAX_BITS 9
#endif

namespace {

using p2m::DevView;
using p2m::Layout;

template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t upload(const T *src, size_t count) {
    reset();
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    n = count;
    return cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
  }
};

p2m_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return P2M_OK;
  if (e == cudaErrorMemoryAllocation) return P2M_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return P2M_ERR_NO_DEVICE;
  return P2M_ERR_CUDA;
}

// concurrent ranges of a split query: at most `streams`, each of at least
// 2^18 queries
int split_count(int64_t n, int streams) {
  const int64_t by_size = n >> 18;
  return (int)std::max<int64_t>(1, std::min<int64_t>(streams, by_size));
}

bool have_device() {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

}  // namespace

struct p2m_handle {
  int device = -1;          // -1: host-only handle (tables built, no queries)
  Layout L;                 // host copy of the layout
  DevBuf<float> kd_nodes, kd_points, edge_rec, face_rec;
  DevBuf<uint32_t> entries;
  DevBuf<uint32_t> row_off, nb_off, nb, chunk_off, seed, sort_seed;
  int grid_bits = 0, sort_grid_bits = 0;
  DevBuf<uint32_t> chunks, super_off, supers;
  DevBuf<float> nbp;
  DevBuf<int32_t> edges, tris;
  DevView view{};
  void *scratch = nullptr;  // query scratch arena
  size_t scratch_bytes = 0;
  p2m::QueryTuning tune;
  size_t device_bytes = 0;
  // timing ring: kEv events per recorded p2m_query
  static constexpr int kRing = 1024;
  static constexpr int kEv = 6;
  std::vector<cudaEvent_t> ring;
  int64_t ring_next = 0, ring_read = 0;
  unsigned long long *counters = nullptr;
  // forked streams of a split p2m_query (tuning field streams): range k > 0
  // of the sorted queries runs on aux[k - 1], which waits on fork (recorded
  // on the caller's stream after the first sort) and is joined back through
  // join[k - 1]
  static constexpr int kMaxStreams = 4;
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;

  ~p2m_handle() {
    for (cudaStream_t st : aux) cudaStreamSynchronize(st);
    if (scratch) cudaFree(scratch);
    if (counters) cudaFree(counters);
    for (auto &e : ring) cudaEventDestroy(e);
    for (cudaEvent_t e : join) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (cudaStream_t st : aux) cudaStreamDestroy(st);
  }

  // streams and events for up to k concurrent ranges (created once;
  // before any capture, by p2m_set_tuning and p2m_reserve)
  p2m_status ensure_aux(int k) {
    if (!fork && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) {
      fork = nullptr;
      return P2M_ERR_CUDA;
    }
    while ((int)aux.size() < k - 1) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return P2M_ERR_CUDA;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(st);
        return P2M_ERR_CUDA;
      }
      aux.push_back(st);
      join.push_back(ev);
    }
    return P2M_OK;
  }

  p2m_status ensure_scratch(size_t bytes) {
    if (bytes <= scratch_bytes) return P2M_OK;
    if (scratch) cudaFree(scratch);
    scratch = nullptr;
    scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&scratch, bytes);
    if (e != cudaSuccess) {
      scratch = nullptr;
      return from_cuda(e);
    }
    scratch_bytes = bytes;
    return P2M_OK;
  }

  void make_view() {
    view.kd_nodes = (const float4 *)kd_nodes.p;
    view.kd_points = (const float4 *)kd_points.p;
    view.row_off = row_off.p;
    view.entries = (const uint4 *)entries.p;
    view.edge_rec = (const float4 *)edge_rec.p;
    view.face_rec = (const float4 *)face_rec.p;
    view.edges = (const int2 *)edges.p;
    view.tris = (const int4 *)tris.p;
    view.nb_off = nb_off.p;
    view.nb = nb.p;
    view.nbp = (const float4 *)nbp.p;
    view.chunk_off = chunk_off.p;
    view.chunks = (const uint4 *)chunks.p;
    view.super_off = super_off.p;
    view.supers = (const uint4 *)supers.p;
    for (int d = 0; d < 3; ++d) {
      view.qlo[d] = L.qframe_lo[d];
      view.qinv[d] = L.qframe_inv[d];
    }
    p2m::q_frame_derive(view.qlo, view.qinv, view.qstep, view.qbase);
    view.seed = seed.p;
    view.grid_bits = seed.p ? grid_bits : 0;
    view.sort_seed = sort_seed.p ? sort_seed.p : seed.p;
    view.sort_grid_bits = sort_seed.p ? sort_grid_bits : view.grid_bits;
    view.nv = L.nv;
    view.depth = L.kd_depth;
    view.L = (int64_t)1 << L.kd_depth;
    for (int d = 0; d < 3; ++d) {
      view.dom_lo[d] = L.dom[d];
      view.dom_hi[d] = L.dom[3 + d];
    }
  }

  cudaError_t upload_tree() {
    cudaError_t e = kd_nodes.upload(L.kd_nodes.data(), L.kd_nodes.size());
    if (e == cudaSuccess) e = kd_points.upload(L.kd_points.data(), L.kd_points.size());
    make_view();
    return e;
  }

  cudaError_t upload_rest() {
    cudaError_t e = row_off.upload(L.row_off.data(), L.row_off.size());
    if (e == cudaSuccess) e = entries.upload(L.entries.data(), L.entries.size());
    if (e == cudaSuccess) e = edge_rec.upload(L.edge_rec.data(), L.edge_rec.size());
    if (e == cudaSuccess) e = face_rec.upload(L.face_rec.data(), L.face_rec.size());
    if (e == cudaSuccess) e = edges.upload(L.edges.data(), L.edges.size());
    if (e == cudaSuccess) e = tris.upload(L.tris.data(), L.tris.size());
    if (e == cudaSuccess && !L.nb_off.empty()) e = nb_off.upload(L.nb_off.data(), L.nb_off.size());
    if (e == cudaSuccess && !L.nb.empty()) e = nb.upload(L.nb.data(), L.nb.size());
    if (e == cudaSuccess && !L.nbp.empty()) e = nbp.upload(L.nbp.data(), L.nbp.size());
    if (e == cudaSuccess && !L.chunk_off.empty())
      e = chunk_off.upload(L.chunk_off.data(), L.chunk_off.size());
    if (e == cudaSuccess && !L.chunks.empty()) e = chunks.upload(L.chunks.data(), L.chunks.size());
    if (e == cudaSuccess && !L.super_off.empty())
      e = super_off.upload(L.super_off.data(), L.super_off.size());
    if (e == cudaSuccess && !L.supers.empty()) e = supers.upload(L.supers.data(), L.supers.size());
    make_view();
    if (e == cudaSuccess) e = make_seed_grid();
    device_bytes = 4 * (kd_nodes.n + kd_points.n + entries.n + edge_rec.n + face_rec.n +
                        row_off.n + edges.n + tris.n + nb_off.n + nb.n + chunk_off.n + chunks.n +
                        seed.n + sort_seed.n + nbp.n + super_off.n + supers.n);
    return e;
  }

  // Seed grid of the Voronoi walk: G^3 cells over D with G = 2^k, up to
  // P2M_GRID_PER_VERTEX cells per vertex (16 <= G <= 2^P2M_GRID_MAX_BITS); each cell holds
  // the nearest vertex of its centre, computed on the device with the exact
  // KD-tree search.
  cudaError_t make_seed_grid() {
    int k = 4;
    while (k < P2M_GRID_MAX_BITS && ((int64_t)1 << (3 * (k + 1))) <= P2M_GRID_PER_VERTEX * L.nv) ++k;
    const size_t cells = (size_t)1 << (3 * k);
    seed.reset();
    cudaError_t e = cudaMalloc((void **)&seed.p, cells * sizeof(uint32_t));
    if (e != cudaSuccess) {
      seed.p = nullptr;
      return e;
    }
    seed.n = cells;
    grid_bits = k;
    make_view();
    e = p2m::launch_seed_grid(view, seed.p, 0);
    // the sort key's grid: the same at 256^3 (64 MiB, small enough for L2)
    // when the walk's grid is finer
    sort_seed.reset();
    if (e == cudaSuccess && k > 8) {
      const size_t c2 = (size_t)1 << 24;
      e = cudaMalloc((void **)&sort_seed.p, c2 * sizeof(uint32_t));
      if (e != cudaSuccess) {
        sort_seed.p = nullptr;
        return e;
      }
      sort_seed.n = c2;
      sort_grid_bits = 8;
      p2m::DevView v2 = view;
      v2.grid_bits = 8;
      e = p2m::launch_seed_grid(v2, sort_seed.p, 0);
    }
    make_view();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
  }
};

namespace {

// Device services of the builder: the exact certification search, the
// Voronoi cells and the flooding, on the handle's device.
struct DeviceNearest : p2m::NearestService {
  p2m_handle *h;
  explicit DeviceNearest(p2m_handle *hh) : h(hh) {}
  bool within(const double *xyz, const double *r2, int64_t n, int64_t *out) override {
    const int64_t chunk = 1 << 22;
    const int64_t m = std::min(n, chunk);
    double *dx = nullptr, *dr = nullptr;
    int64_t *dout = nullptr;
    bool ok = cudaMalloc((void **)&dx, 24 * m) == cudaSuccess &&
              cudaMalloc((void **)&dr, 8 * m) == cudaSuccess &&
              cudaMalloc((void **)&dout, 8 * m) == cudaSuccess;
    for (int64_t s = 0; s < n && ok; s += chunk) {
      const int64_t k = std::min(chunk, n - s);
      ok = cudaMemcpy(dx, xyz + 3 * s, 24 * k, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(dr, r2 + s, 8 * k, cudaMemcpyHostToDevice) == cudaSuccess &&
           p2m::launch_nearest_within_f64(h->view, dx, dr, k, dout, 0) == cudaSuccess &&
           cudaMemcpy(out + s, dout, 8 * k, cudaMemcpyDeviceToHost) == cudaSuccess;
    }
    if (dx) cudaFree(dx);
    if (dr) cudaFree(dr);
    if (dout) cudaFree(dout);
    if (!ok) cudaGetLastError();
    return ok;
  }
  bool flood(const p2m::FloodProblem &pb, std::vector<p2m::FloodRec> &out,
             std::vector<uint8_t> &gave_up, int64_t &inspections) override {
    return p2m::flood_on_device(pb, out, gave_up, inspections);
  }
  bool cells(const p2m::CellProblem &pb, p2m::CellResult &out) override {
    return p2m::cells_on_device(h->view, pb, out);
  }
  bool pack(int64_t nv, const std::vector<p2m::PackPart> &parts, const float qlo[3],
            const float qinv[3], p2m::Layout &out, int64_t &max_list,
            int64_t &bad_boxes) override {
    return p2m::pack_on_device(nv, parts, qlo, qinv, out, max_list, bad_boxes);
  }
};

// the builder fills the handle's own layout; once its KD tree exists the
// tree goes to the device so the certification rounds can search it
bool on_tree_cb(void *ctx, const Layout &) {
  p2m_handle *h = (p2m_handle *)ctx;
  return h->upload_tree() == cudaSuccess;
}

p2m_status check_ready(const p2m_handle *h) {
  if (!h) return P2M_ERR_INVALID_ARG;
  if (h->device < 0) return P2M_ERR_NO_DEVICE;
  return P2M_OK;
}

}  // namespace

extern "C" {

void p2m_default_opts(p2m_build_opts *o) {
  if (!o) return;
  o->domain_scale = 10.f;
  o->domain_margin = 0.f;
  o->delta_rel = 4e-6f;
  o->host_threads = 0;
  o->device_assist = 3;
  o->leaf_size = 8;
}

const char *p2m_status_string(p2m_status s) {
  switch (s) {
    case P2M_OK: return "ok";
    case P2M_ERR_INVALID_ARG: return "invalid argument";
    case P2M_ERR_INVALID_MESH: return "invalid mesh";
    case P2M_ERR_DUPLICATE_VERTEX: return "duplicate vertex position";
    case P2M_ERR_OOM: return "out of memory";
    case P2M_ERR_CUDA: return "CUDA error";
    case P2M_ERR_QUEUE_TIMEOUT: return "work queue error";
    case P2M_ERR_IO: return "I/O error";
    case P2M_ERR_NO_DEVICE: return "no CUDA device";
    case P2M_ERR_TOO_LARGE: return "size exceeds a limit";
  }
  return "unknown status";
}

p2m_status p2m_build(const p2m_mesh *mesh, const p2m_build_opts *opts, p2m_handle **out) {
  if (!mesh || !mesh->tris) return P2M_ERR_INVALID_ARG;
  return p2m_build_mixed(mesh, nullptr, 0, opts, out);
}

p2m_status p2m_build_mixed(const p2m_mesh *mesh, const int32_t *segs, int64_t n_segs,
                           const p2m_build_opts *opts, p2m_handle **out) {
  if (!mesh || !out || !mesh->verts || mesh->n_verts < 0 || mesh->n_tris < 0 || n_segs < 0 ||
      (mesh->n_tris > 0 && !mesh->tris) || (n_segs > 0 && !segs))
    return P2M_ERR_INVALID_ARG;
  *out = nullptr;
  if (mesh->n_verts >= ((int64_t)1 << 30) || mesh->n_tris >= ((int64_t)1 << 29) ||
      n_segs >= ((int64_t)1 << 29))
    return P2M_ERR_TOO_LARGE;
  p2m_build_opts o;
  p2m_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.domain_scale > 0.f) || !(o.domain_margin >= 0.f) || !(o.delta_rel >= 0.f) ||
      o.leaf_size < 2 || o.leaf_size > 32 || o.device_assist < 0 || o.device_assist > 3)
    return P2M_ERR_INVALID_ARG;
  std::unique_ptr<p2m_handle> h(new (std::nothrow) p2m_handle());
  if (!h) return P2M_ERR_OOM;
  if (have_device()) {
    if (cudaGetDevice(&h->device) != cudaSuccess) return P2M_ERR_NO_DEVICE;
  }
  p2m::BuildParams prm;
  prm.domain_scale = o.domain_scale;
  prm.domain_margin = o.domain_margin;
  prm.delta_rel = o.delta_rel;
  prm.threads = o.host_threads;
  prm.leaf_size = o.leaf_size;
  prm.device_flood = o.device_assist >= 2;
  prm.device_cells = o.device_assist == 3;
  prm.device_pack = o.device_assist == 3;
  DeviceNearest dn(h.get());
  const bool assist = o.device_assist && h->device >= 0;
  std::string err;
  int st;
  try {
    st = p2m::build_layout(mesh->verts, mesh->n_verts, mesh->tris, mesh->n_tris, segs, n_segs,
                           prm,
                           assist ? &dn : nullptr, assist ? on_tree_cb : nullptr, h.get(), h->L,
                           err);
  } catch (const std::bad_alloc &) {
    return P2M_ERR_OOM;
  } catch (const std::length_error &) {  // a host array beyond what can be allocated
    return P2M_ERR_OOM;
  }
  if (st) return (p2m_status)st;
  if (h->device >= 0) {
    cudaError_t e = h->upload_tree();
    if (e == cudaSuccess) e = h->upload_rest();
    if (e != cudaSuccess) return from_cuda(e);
  }
  *out = h.release();
  return P2M_OK;
}

void p2m_destroy(p2m_handle *h) { delete h; }

p2m_status p2m_get_tuning(const p2m_handle *h, p2m_tuning *t) {
  if (!h || !t) return P2M_ERR_INVALID_ARG;
  t->sort_bits = h->tune.sort_bits;
  t->block_threads = h->tune.block_threads;
  t->warp_cooperative = h->tune.warp_mode;
  t->nn_walk = h->tune.nn_walk;
  t->chunked = h->tune.chunked;
  t->group_by_vertex = h->tune.group_by_vertex;
  t->sort_key = h->tune.sort_key;
  t->lanes_per_query = h->tune.lanes_per_query;
  t->streams = h->tune.streams;
  return P2M_OK;
}

p2m_status p2m_set_tuning(p2m_handle *h, const p2m_tuning *t) {
  if (!h || !t || t->sort_bits < 0 || t->sort_bits > 24) return P2M_ERR_INVALID_ARG;
  if (t->block_threads != 64 && t->block_threads != 128 && t->block_threads != 256 &&
      t->block_threads != 512)
    return P2M_ERR_INVALID_ARG;
  if (t->warp_cooperative != 0 && t->warp_cooperative != 1) return P2M_ERR_INVALID_ARG;
  if (t->nn_walk < 0 || t->nn_walk > 2) return P2M_ERR_INVALID_ARG;
  if (t->chunked < 0 || t->chunked > 2) return P2M_ERR_INVALID_ARG;
  if (t->group_by_vertex != 0 && t->group_by_vertex != 1) return P2M_ERR_INVALID_ARG;
  if (t->sort_key != 0 && t->sort_key != 1) return P2M_ERR_INVALID_ARG;
  if (t->lanes_per_query != 1 && t->lanes_per_query != 2 && t->lanes_per_query != 4 &&
      t->lanes_per_query != 8)
    return P2M_ERR_INVALID_ARG;
  if (t->streams < 1 || t->streams > p2m_handle::kMaxStreams) return P2M_ERR_INVALID_ARG;
  if (t->streams > 1) {
    p2m_status s = h->ensure_aux(t->streams);
    if (s) return s;
  }
  h->tune.streams = t->streams;
  h->tune.lanes_per_query = t->lanes_per_query;
  h->tune.group_by_vertex = t->group_by_vertex;
  h->tune.sort_key = t->sort_key;
  h->tune.nn_walk = t->nn_walk;
  h->tune.chunked = t->chunked;
  h->tune.sort_bits = t->sort_bits;
  h->tune.block_threads = t->block_threads;
  h->tune.warp_mode = t->warp_cooperative;
  return P2M_OK;
}

p2m_status p2m_reserve(p2m_handle *h, int64_t n) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (n < 0) return P2M_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 31)) return P2M_ERR_TOO_LARGE;
  // one pipeline (plus the staging of p2m_query_host), or the largest split
  const size_t one = p2m::query_scratch_bytes(n, 24, h->L.nv) + 24 * (size_t)n + 4096;
  const size_t split =
      p2m::query_scratch_bytes(n, 24, h->L.nv, split_count(n, p2m_handle::kMaxStreams));
  if ((s = h->ensure_aux(p2m_handle::kMaxStreams))) return s;
  return h->ensure_scratch(std::max(one, split));
}

p2m_status p2m_query(p2m_handle *h, const float *q, int64_t n, float *dist, float *closest,
                     int32_t *prim_id, uint8_t *prim_type, float *save, uint8_t *status,
                     void *stream) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (n < 0) return P2M_ERR_INVALID_ARG;
  if (n == 0) return P2M_OK;
  if (!q || !dist || !prim_id) return P2M_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 31)) return P2M_ERR_TOO_LARGE;
  const int64_t nvk = h->tune.group_by_vertex ? h->L.nv : 0;
  // concurrent ranges after the first sort (tuning field streams); with
  // per-phase timing on, one pipeline on the caller's stream
  const int R = (h->ring.empty() && nvk > 0 && !h->tune.warp_mode)
                    ? split_count(n, h->tune.streams) : 1;
  size_t need = p2m::query_scratch_bytes(n, h->tune.sort_bits, nvk, R);
  if ((s = h->ensure_scratch(need))) return s;
  cudaEvent_t *ev = nullptr;
  if (!h->ring.empty()) {
    ev = &h->ring[p2m_handle::kEv * (h->ring_next % p2m_handle::kRing)];
    ++h->ring_next;
  }
  p2m::SplitStreams split{};
  if (R > 1) {
    if ((s = h->ensure_aux(R))) return s;
    split = {h->aux.data(), h->join.data(), h->fork, R - 1};
  }
  return from_cuda(p2m::launch_query(h->view, q, n, dist, closest, prim_id, prim_type,
                                     (float4 *)save, status, h->scratch, h->scratch_bytes,
                                     h->tune, (cudaStream_t)stream, ev, nullptr,
                                     R > 1 ? &split : nullptr));
}

p2m_status p2m_set_timing(p2m_handle *h, int enable) {
  p2m_status s = check_ready(h);
  if (s) return s;
  for (auto &e : h->ring) cudaEventDestroy(e);
  h->ring.clear();
  h->ring_next = h->ring_read = 0;
  if (enable) {
    h->ring.resize(p2m_handle::kEv * p2m_handle::kRing, nullptr);
    for (auto &e : h->ring)
      if (cudaEventCreate(&e) != cudaSuccess) return P2M_ERR_CUDA;
  }
  return P2M_OK;
}

p2m_status p2m_timing_summary(p2m_handle *h, double out[6]) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (!out || h->ring.empty()) return P2M_ERR_INVALID_ARG;
  constexpr int E = p2m_handle::kEv;
  for (int k = 0; k < E; ++k) out[k] = 0.0;
  int64_t first = std::max(h->ring_read, h->ring_next - (int64_t)p2m_handle::kRing);
  for (int64_t k = first; k < h->ring_next; ++k) {
    cudaEvent_t *ev = &h->ring[E * (k % p2m_handle::kRing)];
    cudaError_t e = cudaEventSynchronize(ev[E - 1]);
    if (e != cudaSuccess) return from_cuda(e);
    out[0] += 1.0;
    for (int p = 0; p < E - 1; ++p) {
      float ms = 0;
      e = cudaEventElapsedTime(&ms, ev[p], ev[p + 1]);
      if (e != cudaSuccess) return from_cuda(e);
      out[1 + p] += ms;
    }
  }
  h->ring_read = h->ring_next;
  return P2M_OK;
}

p2m_status p2m_query_counters(p2m_handle *h, const float *q, int64_t n, int64_t out[6],
                              void *stream) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (!q || !out || n <= 0) return P2M_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 31)) return P2M_ERR_TOO_LARGE;
  if ((s = h->ensure_scratch(p2m::query_scratch_bytes(n, h->tune.sort_bits)))) return s;
  if (!h->counters && cudaMalloc((void **)&h->counters, 64) != cudaSuccess) return P2M_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p2m::launch_query(h->view, q, n, nullptr, nullptr, nullptr, nullptr, nullptr,
                                    nullptr, h->scratch, h->scratch_bytes, h->tune, st, nullptr,
                                    h->counters);
  unsigned long long c[6];
  if (e == cudaSuccess) e = cudaMemcpyAsync(c, h->counters, 48, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  for (int k = 0; k < 6; ++k) out[k] = (int64_t)c[k];
  return P2M_OK;
}

p2m_status p2m_nearest_vertex(p2m_handle *h, const float *q, int64_t n, int32_t *vertex,
                              void *stream) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (n < 0) return P2M_ERR_INVALID_ARG;
  if (n == 0) return P2M_OK;
  if (!q || !vertex) return P2M_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 31)) return P2M_ERR_TOO_LARGE;
  return from_cuda(p2m::launch_nearest(h->view, q, n, vertex, (cudaStream_t)stream, true,
                                       h->view.nb_off ? h->tune.nn_walk : 0));
}

p2m_status p2m_query_host(p2m_handle *h, const float *q, int64_t n, float *dist, float *closest,
                          int32_t *prim_id, uint8_t *prim_type, void *stream) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (n < 0) return P2M_ERR_INVALID_ARG;
  if (n == 0) return P2M_OK;
  if (!q || !dist || !prim_id) return P2M_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 31)) return P2M_ERR_TOO_LARGE;
  // device staging lives in the scratch arena after the query's own part
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t need_q = p2m::query_scratch_bytes(n, h->tune.sort_bits,
                                           h->tune.group_by_vertex ? h->L.nv : 0);
  size_t io = al(12 * (size_t)n) + al(4 * (size_t)n) + al(12 * (size_t)n) + al(4 * (size_t)n) +
              al((size_t)n);
  if ((s = h->ensure_scratch(al(need_q) + io + 256))) return s;
  char *base = (char *)(((uintptr_t)h->scratch + 255) & ~(uintptr_t)255) + al(need_q);
  float *dq = (float *)base;
  base += al(12 * (size_t)n);
  float *dd = (float *)base;
  base += al(4 * (size_t)n);
  float *dc = (float *)base;
  base += al(12 * (size_t)n);
  int32_t *dp = (int32_t *)base;
  base += al(4 * (size_t)n);
  uint8_t *dt = (uint8_t *)base;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(dq, q, 12 * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = p2m::launch_query(h->view, dq, n, dd, closest ? dc : nullptr, dp, prim_type ? dt : nullptr,
                          nullptr, nullptr, h->scratch, al(need_q) + 256, h->tune, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dist, dd, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(prim_id, dp, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && closest)
    e = cudaMemcpyAsync(closest, dc, 12 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && prim_type)
    e = cudaMemcpyAsync(prim_type, dt, (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return from_cuda(e);
}

}  // extern "C"

// A pipeline of host-memory queries: `depth` slots, each with its own
// stream, device scratch and staging buffers, used round robin.  The copies
// of one slot run on the copy engines while another slot's kernels run, so
// a stream of batches costs about max(kernels, copies) per batch instead of
// their sum.
struct p2m_pipe {
  struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t after = nullptr;  // p2m_pipe_submit_device: the caller's stream so far
    void *mem = nullptr;
    size_t bytes = 0;
    bool busy = false;
  };
  p2m_handle *h = nullptr;
  int64_t max_n = 0;
  std::vector<Slot> slots;
  int64_t next = 0;
  ~p2m_pipe() {
    for (auto &s : slots) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      if (s.mem) cudaFree(s.mem);
      if (s.done) cudaEventDestroy(s.done);
      if (s.after) cudaEventDestroy(s.after);
      if (s.stream) cudaStreamDestroy(s.stream);
    }
  }
  // query scratch for any tuning (sort bits up to 24) + staging of q and of
  // the outputs
  size_t query_bytes() const {
    return (p2m::query_scratch_bytes(max_n, 24, h->L.nv) + 255) & ~(size_t)255;
  }
  size_t slot_bytes() const {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t n = (size_t)max_n;
    return query_bytes() + al(12 * n) + al(4 * n) + al(12 * n) + al(4 * n) + al(n) + 256;
  }
};

extern "C" {

p2m_status p2m_pipe_create(p2m_handle *h, int64_t max_n, int depth, p2m_pipe **out) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (!out || max_n <= 0 || depth < 1 || depth > 8) return P2M_ERR_INVALID_ARG;
  if (max_n >= ((int64_t)1 << 31)) return P2M_ERR_TOO_LARGE;
  *out = nullptr;
  std::unique_ptr<p2m_pipe> p(new (std::nothrow) p2m_pipe());
  if (!p) return P2M_ERR_OOM;
  p->h = h;
  p->max_n = max_n;
  p->slots.resize(depth);
  for (auto &sl : p->slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) {
      sl.bytes = p->slot_bytes();
      e = cudaMalloc(&sl.mem, sl.bytes);
      if (e != cudaSuccess) sl.mem = nullptr;
    }
    if (e != cudaSuccess) return from_cuda(e);
  }
  *out = p.release();
  return P2M_OK;
}

p2m_status p2m_pipe_submit(p2m_pipe *p, const float *q, int64_t n, float *dist, float *closest,
                           int32_t *prim_id, uint8_t *prim_type) {
  if (!p) return P2M_ERR_INVALID_ARG;
  p2m_handle *h = p->h;
  p2m_status s = check_ready(h);
  if (s) return s;
  if (n < 0) return P2M_ERR_INVALID_ARG;
  if (n == 0) return P2M_OK;
  if (!q || !dist || !prim_id) return P2M_ERR_INVALID_ARG;
  if (n > p->max_n) return P2M_ERR_TOO_LARGE;
  p2m_pipe::Slot &sl = p->slots[p->next % (int64_t)p->slots.size()];
  // the slot's previous batch must be done before its buffers are reused
  cudaError_t e = sl.busy ? cudaEventSynchronize(sl.done) : cudaSuccess;
  if (e != cudaSuccess) return from_cuda(e);
  sl.busy = false;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nn = (size_t)p->max_n;
  char *base = (char *)(((uintptr_t)sl.mem + 255) & ~(uintptr_t)255) + p->query_bytes();
  float *dq = (float *)base;
  base += al(12 * nn);
  float *dd = (float *)base;
  base += al(4 * nn);
  float *dc = (float *)base;
  base += al(12 * nn);
  int32_t *dp = (int32_t *)base;
  base += al(4 * nn);
  uint8_t *dt = (uint8_t *)base;
  cudaStream_t st = sl.stream;
  e = cudaMemcpyAsync(dq, q, 12 * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = p2m::launch_query(h->view, dq, n, dd, closest ? dc : nullptr, dp,
                          prim_type ? dt : nullptr, nullptr, nullptr, sl.mem, p->query_bytes(),
                          h->tune, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dist, dd, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(prim_id, dp, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && closest)
    e = cudaMemcpyAsync(closest, dc, 12 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && prim_type)
    e = cudaMemcpyAsync(prim_type, dt, (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
  if (e != cudaSuccess) return from_cuda(e);
  sl.busy = true;
  ++p->next;
  return P2M_OK;
}

p2m_status p2m_pipe_submit_device(p2m_pipe *p, const float *q, int64_t n, float *dist,
                                  float *closest, int32_t *prim_id, uint8_t *prim_type,
                                  void *stream) {
  if (!p) return P2M_ERR_INVALID_ARG;
  p2m_handle *h = p->h;
  p2m_status s = check_ready(h);
  if (s) return s;
  if (n < 0) return P2M_ERR_INVALID_ARG;
  if (n == 0) return P2M_OK;
  if (!q || !dist || !prim_id) return P2M_ERR_INVALID_ARG;
  if (n > p->max_n) return P2M_ERR_TOO_LARGE;
  p2m_pipe::Slot &sl = p->slots[p->next % (int64_t)p->slots.size()];
  cudaError_t e = sl.busy ? cudaEventSynchronize(sl.done) : cudaSuccess;
  if (e != cudaSuccess) return from_cuda(e);
  sl.busy = false;
  // the batch starts after the work enqueued so far on `stream`
  if (!sl.after && cudaEventCreateWithFlags(&sl.after, cudaEventDisableTiming) != cudaSuccess) {
    sl.after = nullptr;
    return P2M_ERR_CUDA;
  }
  e = cudaEventRecord(sl.after, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.stream, sl.after, 0);
  if (e == cudaSuccess)
    e = p2m::launch_query(h->view, q, n, dist, closest, prim_id, prim_type, nullptr, nullptr,
                          sl.mem, p->query_bytes(), h->tune, sl.stream);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
  if (e != cudaSuccess) return from_cuda(e);
  sl.busy = true;
  ++p->next;
  return P2M_OK;
}

p2m_status p2m_pipe_join(p2m_pipe *p, void *stream) {
  if (!p) return P2M_ERR_INVALID_ARG;
  for (auto &sl : p->slots) {
    if (!sl.busy) continue;
    cudaError_t e = cudaStreamWaitEvent((cudaStream_t)stream, sl.done, 0);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return P2M_OK;
}

p2m_status p2m_pipe_wait(p2m_pipe *p) {
  if (!p) return P2M_ERR_INVALID_ARG;
  for (auto &sl : p->slots) {
    if (!sl.busy) continue;
    cudaError_t e = cudaEventSynchronize(sl.done);
    if (e != cudaSuccess) return from_cuda(e);
    sl.busy = false;
  }
  return P2M_OK;
}

void p2m_pipe_destroy(p2m_pipe *p) { delete p; }

p2m_status p2m_backward(p2m_handle *h, const float *q, const float *dist, const float *closest,
                        const float *save, const float *grad_dist, int64_t n, float *grad_q,
                        float *grad_verts, void *stream) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (n < 0) return P2M_ERR_INVALID_ARG;
  if (n == 0) return P2M_OK;
  if (!q || !dist || !closest || !save || !grad_dist) return P2M_ERR_INVALID_ARG;
  return from_cuda(p2m::launch_backward(h->view, q, dist, closest, (const float4 *)save,
                                        grad_dist, n, grad_q, grad_verts, (cudaStream_t)stream));
}

p2m_status p2m_update_vertices(p2m_handle *h, const float *verts, int64_t n_verts,
                               int refresh_seed_grid, void *stream) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (!verts || n_verts != h->L.nv) return P2M_ERR_INVALID_ARG;
  if (refresh_seed_grid != 0 && refresh_seed_grid != 1) return P2M_ERR_INVALID_ARG;
  p2m::GeometryRefs g{};
  g.kd_points = (float4 *)h->kd_points.p;
  g.kd_nodes = (float4 *)h->kd_nodes.p;
  g.nbp = (float4 *)h->nbp.p;
  g.nb = h->nb.p;
  g.edge_rec = (float4 *)h->edge_rec.p;
  g.face_rec = (float4 *)h->face_rec.p;
  g.edges = (const int2 *)h->edges.p;
  g.tris = (const int4 *)h->tris.p;
  g.nv = h->L.nv;
  g.n_nb = (int64_t)h->nb.n;
  g.ne = h->L.ne;
  g.nf = h->L.nf;
  g.depth = h->L.kd_depth;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p2m::launch_update_vertices(g, verts, st);
  if (e == cudaSuccess && refresh_seed_grid && h->seed.p) {
    e = p2m::launch_seed_grid(h->view, h->seed.p, st);
    if (e == cudaSuccess && h->sort_seed.p) {
      p2m::DevView v2 = h->view;
      v2.grid_bits = h->sort_grid_bits;
      e = p2m::launch_seed_grid(v2, h->sort_seed.p, st);
    }
  }
  return from_cuda(e);
}

p2m_status p2m_get_edges(const p2m_handle *h, int32_t *edges, int64_t *n_edges) {
  if (!h || !n_edges) return P2M_ERR_INVALID_ARG;
  *n_edges = h->L.ne;
  if (edges) std::memcpy(edges, h->L.edges.data(), sizeof(int32_t) * 2 * h->L.ne);
  return P2M_OK;
}

p2m_status p2m_stats(const p2m_handle *h, int64_t out[16]) {
  if (!h || !out) return P2M_ERR_INVALID_ARG;
  const Layout &L = h->L;
  out[0] = L.nv;
  out[1] = L.nf;
  out[2] = L.ne;
  out[3] = L.n_entries;
  out[4] = L.max_list;
  out[5] = (int64_t)h->device_bytes;
  out[6] = (int64_t)1 << L.kd_depth;
  out[7] = L.kd_depth;
  out[8] = L.neighbour_pairs;
  out[9] = L.inspections;
  out[10] = (int64_t)L.ms_total;
  out[11] = (int64_t)L.ms_cells;
  out[12] = (int64_t)L.ms_inspect;
  out[13] = L.cert_rounds;
  out[14] = L.cert_queries;
  out[15] = L.n_degenerate;
  return P2M_OK;
}

p2m_status p2m_flood_stats(const p2m_handle *h, int64_t out[3]) {
  if (!h || !out) return P2M_ERR_INVALID_ARG;
  out[0] = h->L.flood_device;
  out[1] = h->L.flood_bounded;
  out[2] = h->L.flood_unbounded;
  return P2M_OK;
}

p2m_status p2m_cell_stats(const p2m_handle *h, int64_t out[3]) {
  if (!h || !out) return P2M_ERR_INVALID_ARG;
  out[0] = h->L.cells_device;
  out[1] = h->L.cells_host;
  out[2] = h->L.pack_device;
  return P2M_OK;
}

p2m_status p2m_domain(const p2m_handle *h, float out[7]) {
  if (!h || !out) return P2M_ERR_INVALID_ARG;
  for (int d = 0; d < 6; ++d) out[d] = h->L.dom[d];
  out[6] = h->L.delta;
  return P2M_OK;
}

p2m_status p2m_get_list(const p2m_handle *h, int32_t vertex, int32_t *types, int32_t *ids,
                        float *boxes, int64_t cap, int64_t *len) {
  if (!h || !len || vertex < 0 || vertex >= h->L.nv || cap < 0) return P2M_ERR_INVALID_ARG;
  const Layout &L = h->L;
  const int64_t row = L.pos_of_vertex[vertex];
  const int64_t b = L.row_off[row], e = L.row_off[row + 1];
  *len = e - b;
  for (int64_t j = b; j < e && j - b < cap; ++j) {
    const uint32_t *w = &L.entries[4 * (size_t)j];
    if (types) types[j - b] = (int32_t)(w[0] >> 30);
    if (ids) ids[j - b] = (int32_t)(w[0] & 0x3fffffffu);
    if (boxes) {
      // the set of points the query kernel admits: chunk frame from the
      // chunk's codes, then the entry's codes in it (a hair wider, so that
      // the float rounding of the code computation stays inside)
      const uint32_t *cw = &L.chunks[4 * (size_t)(L.chunk_off[row] + (j - b) / Layout::kChunk)];
      float step[3], base[3];
      p2m::q_frame_derive(L.qframe_lo, L.qframe_inv, step, base);
      uint32_t clc[3], chc[3], elc[3], ehc[3];
      p2m::q_unwords(cw, clc, chc);
      p2m::q_unwords(w + 1, elc, ehc);
      for (int d = 0; d < 3; ++d) {
        const double lo = p2m::q_chunk_lo(clc[d], step[d], base[d]);
        const double inv = p2m::q_chunk_inv(L.qframe_inv[d], cw[3], d);
        boxes[6 * (j - b) + d] = elc[d] == 0 ? -INFINITY : (float)(lo + (elc[d] - 1.01) / inv);
        boxes[6 * (j - b) + 3 + d] =
            ehc[d] == p2m::kQMax ? INFINITY : (float)(lo + (ehc[d] + 0.01) / inv);
      }
    }
  }
  return P2M_OK;
}

// ---------------------------------------------------------------- batched
}  // extern "C"

struct p2m_batch {
  int n = 0;
  int64_t total = 0;
  std::vector<p2m_handle *> meshes;
  std::vector<p2m::BatchIO> io;
  DevBuf<p2m::DevView> views;
  DevBuf<p2m::BatchIO> ios;
  DevBuf<int64_t> qoff;
  DevBuf<int64_t> voff;        // prefix sums of (vertex count + 1) per mesh
  int64_t nv_keys = 0;
  DevBuf<unsigned int> words;  // [0] queue head, [1] error word
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  p2m::BatchTuning tune;
  int sms = 0;
  ~p2m_batch() {
    if (scratch) cudaFree(scratch);
  }
  int grid() const {
    if (tune.grid_ctas > 0) return tune.grid_ctas;
    return sms * p2m::batch_occupancy(tune.block_threads, tune.group_by_vertex);
  }
  p2m_status ensure(int sort_bits, int group) {
    size_t need = p2m::batch_scratch_bytes(total, n, sort_bits, group ? nv_keys : 0);
    if (need <= scratch_bytes) return P2M_OK;
    if (scratch) cudaFree(scratch);
    scratch = nullptr;
    scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&scratch, need);
    if (e != cudaSuccess) {
      scratch = nullptr;
      return from_cuda(e);
    }
    scratch_bytes = need;
    return P2M_OK;
  }
  p2m::BatchDesc desc() const {
    return {views.p, ios.p, qoff.p, voff.p, n, nv_keys};
  }
};

extern "C" {

p2m_status p2m_batch_create(p2m_handle *const *meshes, const p2m_batch_io *io, int n_meshes,
                            p2m_batch **out) {
  if (!meshes || !io || !out || n_meshes <= 0 || n_meshes > 2048) return P2M_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<p2m_batch> b(new (std::nothrow) p2m_batch());
  if (!b) return P2M_ERR_OOM;
  b->n = n_meshes;
  std::vector<p2m::DevView> v(n_meshes);
  std::vector<int64_t> off(n_meshes + 1, 0), vo(n_meshes + 1, 0);
  for (int k = 0; k < n_meshes; ++k) {
    p2m_status s = check_ready(meshes[k]);
    if (s) return s;
    if (io[k].n < 0 || (io[k].n > 0 && (!io[k].q || !io[k].dist || !io[k].prim_id)))
      return P2M_ERR_INVALID_ARG;
    b->meshes.push_back(meshes[k]);
    b->io.push_back({io[k].q, io[k].n, io[k].dist, io[k].closest, io[k].prim_id,
                     io[k].prim_type});
    v[k] = meshes[k]->view;
    off[k + 1] = off[k] + io[k].n;
    vo[k + 1] = vo[k] + meshes[k]->L.nv + 1;
  }
  b->nv_keys = vo[n_meshes];
  if (b->nv_keys > ((int64_t)1 << 24)) b->tune.group_by_vertex = 0;
  b->total = off[n_meshes];
  if (b->total >= ((int64_t)1 << 31)) return P2M_ERR_TOO_LARGE;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = b->views.upload(v.data(), v.size());
  if (e == cudaSuccess) e = b->ios.upload(b->io.data(), b->io.size());
  if (e == cudaSuccess) e = b->qoff.upload(off.data(), off.size());
  if (e == cudaSuccess) e = b->voff.upload(vo.data(), vo.size());
  unsigned int zero[2] = {0, 0};
  if (e == cudaSuccess) e = b->words.upload(zero, 2);
  if (e != cudaSuccess) return from_cuda(e);
  p2m_status s = b->ensure(b->tune.sort_bits, b->tune.group_by_vertex);
  if (s) return s;
  *out = b.release();
  return P2M_OK;
}

p2m_status p2m_batch_run(p2m_batch *b, void *stream) {
  if (!b) return P2M_ERR_INVALID_ARG;
  if (b->scratch_bytes < p2m::batch_scratch_bytes(b->total, b->n, b->tune.sort_bits,
                                                  b->tune.group_by_vertex ? b->nv_keys : 0))
    return P2M_ERR_INVALID_ARG;
  return from_cuda(p2m::launch_batch(b->desc(), b->total, b->scratch, b->scratch_bytes, b->tune,
                                     b->grid(), b->words.p, b->words.p + 1,
                                     (cudaStream_t)stream));
}

p2m_status p2m_batch_get_tuning(const p2m_batch *b, p2m_batch_tuning *t) {
  if (!b || !t) return P2M_ERR_INVALID_ARG;
  t->sort_bits = b->tune.sort_bits;
  t->tile = b->tune.tile;
  t->block_threads = b->tune.block_threads;
  t->grid_ctas = b->tune.grid_ctas;
  t->group_by_vertex = b->tune.group_by_vertex;
  t->lanes_per_query = b->tune.lanes_per_query;
  return P2M_OK;
}

p2m_status p2m_batch_set_tuning(p2m_batch *b, const p2m_batch_tuning *t) {
  if (!b || !t || t->sort_bits < 0 || t->sort_bits > 16 || t->grid_ctas < 0) return P2M_ERR_INVALID_ARG;
  if (t->block_threads != 64 && t->block_threads != 128 && t->block_threads != 256 &&
      t->block_threads != 512)
    return P2M_ERR_INVALID_ARG;
  if (t->tile <= 0 || t->tile % t->block_threads) return P2M_ERR_INVALID_ARG;
  if (t->group_by_vertex != 0 && t->group_by_vertex != 1) return P2M_ERR_INVALID_ARG;
  if (t->lanes_per_query != 1 && t->lanes_per_query != 2 && t->lanes_per_query != 4)
    return P2M_ERR_INVALID_ARG;
  if (((int64_t)b->n << t->sort_bits) > ((int64_t)1 << 24)) return P2M_ERR_TOO_LARGE;
  if (t->group_by_vertex && b->nv_keys > ((int64_t)1 << 24)) return P2M_ERR_TOO_LARGE;
  p2m_status s = b->ensure(t->sort_bits, t->group_by_vertex);
  if (s) return s;
  b->tune.sort_bits = t->sort_bits;
  b->tune.tile = t->tile;
  b->tune.block_threads = t->block_threads;
  b->tune.grid_ctas = t->grid_ctas;
  b->tune.group_by_vertex = t->group_by_vertex;
  b->tune.lanes_per_query = t->lanes_per_query;
  return P2M_OK;
}

p2m_status p2m_batch_check(p2m_batch *b, void *stream) {
  if (!b) return P2M_ERR_INVALID_ARG;
  unsigned int w[2] = {0, 0};
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(w, b->words.p, 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  if (w[1]) {
    unsigned int zero = 0;
    cudaMemcpy(b->words.p + 1, &zero, 4, cudaMemcpyHostToDevice);
    return P2M_ERR_QUEUE_TIMEOUT;
  }
  return P2M_OK;
}

p2m_status p2m_batch_autotune(p2m_batch *b, int reps, void *stream, float *best_ms) {
  if (!b || reps <= 0) return P2M_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return P2M_ERR_CUDA;
  p2m::BatchTuning best = b->tune;
  float bms = 1e30f;
  const int bits_c[] = {8, 10, 12, 14};
  const int tile_c[] = {256, 1024, 4096};
  const int block_c[] = {128, 256};
  p2m_status status = P2M_OK;
  // threads per query (lanes) is tried on the grouped path only
  for (int group = 1; group >= 0; --group)
   for (int lanes = 1; lanes <= (group ? 4 : 1); lanes *= 2)
    for (int bits : bits_c)
      for (int tile : tile_c)
        for (int bt : block_c) {
          if (tile % bt) continue;
          if (((int64_t)b->n << bits) > ((int64_t)1 << 22)) continue;
          if (group && b->nv_keys > ((int64_t)1 << 24)) continue;
          p2m_batch_tuning t{bits, tile, bt, 0, group, lanes};
        if (p2m_batch_set_tuning(b, &t) != P2M_OK) continue;
        if ((status = p2m_batch_run(b, st))) goto done;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r)
          if ((status = p2m_batch_run(b, st))) goto done;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < bms) {
          bms = ms;
          best = b->tune;
        }
      }
done:
  b->ensure(best.sort_bits, best.group_by_vertex);
  b->tune = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_ms) *best_ms = bms;
  return status;
}

void p2m_batch_destroy(p2m_batch *b) { delete b; }

p2m_status p2m_query_batched(p2m_handle *const *meshes, const p2m_batch_io *io, int n_meshes,
                             void *stream) {
  p2m_batch *b = nullptr;
  p2m_status s = p2m_batch_create(meshes, io, n_meshes, &b);
  if (s) return s;
  s = p2m_batch_run(b, stream);
  if (s == P2M_OK) s = p2m_batch_check(b, stream);
  p2m_batch_destroy(b);
  return s;
}

p2m_status p2m_autotune(p2m_handle *h, const float *q, int64_t n, int reps, void *stream,
                        float *best_ms) {
  p2m_status s = check_ready(h);
  if (s) return s;
  if (!q || n <= 0 || reps <= 0) return P2M_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float *dd = nullptr;
  int32_t *dp = nullptr;
  if (cudaMalloc((void **)&dd, 4 * n) != cudaSuccess) return P2M_ERR_OOM;
  if (cudaMalloc((void **)&dp, 4 * n) != cudaSuccess) {
    cudaFree(dd);
    return P2M_ERR_OOM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  p2m::QueryTuning best = h->tune;
  float bms = 1e30f;
  struct Timed {
    float ms;
    p2m::QueryTuning t;
  };
  std::vector<Timed> timed;
  const int bits_c[] = {12, 15, 18, 21, 24};
  const int block_c[] = {128, 256};
  // threads per query: in the one-pass kernel, one thread per query (wm = 0)
  // or a warp answering 32 queries together (wm = 1); in the two-pass path,
  // 1, 2, 4 or 8 lanes splitting each query's list (lanes)
  // list scan: the two-level R-tree (ch = 2) or chunk boxes only (ch = 1)
  for (int gv = 0; gv < 2; ++gv)
  for (int ch = 1; ch < 3; ++ch)
  for (int wm = 0; wm < 2; ++wm)
  for (int lanes = 1; lanes <= 8; lanes *= 2)
  for (int ns = 1; ns <= p2m_handle::kMaxStreams; ++ns)
  for (int key = 0; key < 2; ++key)
  for (int bits : bits_c)
    for (int bt : block_c) {
      if (wm == 1 && gv == 1) continue;
      if (lanes > 1 && gv == 0) continue;
      // concurrent ranges: with one lane and the best-known sorts
      if (ns > 1 && (lanes > 1 || ch != 2 || split_count(n, ns) < ns ||
                     (key != 1 && bits != bits_c[2])))
        continue;
      // sorting by seed vertex ignores sort_bits and needs the regrouping
      if (key == 1 && (gv == 0 || bits != bits_c[0] || !h->seed.p)) continue;
      // the lane split and the one-level scan are tried with the first sort's
      // best-known settings only
      if ((lanes > 1 || ch == 1) && (key != 1 && bits != bits_c[2])) continue;
      p2m_tuning t{bits, bt, wm, 2, ch, gv, key, lanes, ns};
      p2m_set_tuning(h, &t);
      if ((s = p2m_query(h, q, n, dd, nullptr, dp, nullptr, nullptr, nullptr, st))) goto done;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps; ++r)
        if ((s = p2m_query(h, q, n, dd, nullptr, dp, nullptr, nullptr, nullptr, st))) goto done;
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      timed.push_back({ms, h->tune});
    }
  // the fastest few timed again, in turns, three times: the one with the
  // lowest time wins (configurations within a few per cent of each other
  // would otherwise be ranked by the noise of one timing)
  {
    std::sort(timed.begin(), timed.end(),
              [](const Timed &a, const Timed &b) { return a.ms < b.ms; });
    const size_t k = std::min<size_t>(timed.size(), 4);
    std::vector<float> low(k, 1e30f);
    for (int round = 0; round < 3; ++round)
      for (size_t c = 0; c < k; ++c) {
        h->tune = timed[c].t;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r)
          if ((s = p2m_query(h, q, n, dd, nullptr, dp, nullptr, nullptr, nullptr, st)))
            goto done;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        low[c] = std::min(low[c], ms / reps);
      }
    for (size_t c = 0; c < k; ++c)
      if (low[c] < bms) {
        bms = low[c];
        best = timed[c].t;
      }
  }
done:
  h->tune = best;
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(dd);
  cudaFree(dp);
  if (best_ms) *best_ms = bms;
  return s;
}

// ---------------------------------------------------------------- save/load
}  // extern "C"

namespace {
constexpr uint64_t kMagic = 0x314d5032474d5032ull;  // "2PMG2PM1"
constexpr uint32_t kVersion = 7;

uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
  const unsigned char *c = (const unsigned char *)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

template <class T>
bool put_vec(FILE *f, const std::vector<T> &v, uint64_t &ck) {
  uint64_t n = v.size();
  ck = fnv1a(ck, &n, 8);
  ck = fnv1a(ck, v.data(), n * sizeof(T));
  return fwrite(&n, 8, 1, f) == 1 && (n == 0 || fwrite(v.data(), sizeof(T), n, f) == n);
}
template <class T>
bool get_vec(FILE *f, std::vector<T> &v, uint64_t &ck) {
  uint64_t n;
  if (fread(&n, 8, 1, f) != 1 || n > ((uint64_t)1 << 40)) return false;
  v.resize(n);
  if (n && fread(v.data(), sizeof(T), n, f) != n) return false;
  ck = fnv1a(ck, &n, 8);
  ck = fnv1a(ck, v.data(), n * sizeof(T));
  return true;
}
// Every index the query kernels follow, checked against the array it
// indexes: a file whose checksum holds but whose contents do not (written by
// another program, say) is refused instead of sending the kernels out of
// bounds.  Sizes are checked by the caller.
bool layout_consistent(const Layout &L) {
  const int64_t nv = L.nv, nf = L.nf, ne = L.ne;
  const int64_t K = Layout::kChunk;
  if (nv < 1 || nf < 0 || ne < 0 || nv >= ((int64_t)1 << 30) || nf >= ((int64_t)1 << 30) ||
      ne >= ((int64_t)1 << 30) || L.n_entries < 0)
    return false;
  if (L.kd_depth < 0 || L.kd_depth > 30 ||
      (int64_t)L.kd_nodes.size() != 12 * (((int64_t)1 << L.kd_depth) - 1) ||
      (int64_t)L.pos_of_vertex.size() != nv || (int64_t)L.edge_rec.size() != 8 * ne ||
      (int64_t)L.face_rec.size() != 12 * nf || (int64_t)L.tris.size() != 4 * nf)
    return false;
  // tree positions: a permutation of the vertices and its inverse
  for (int64_t p = 0; p < nv; ++p) {
    int32_t v;
    std::memcpy(&v, &L.kd_points[4 * p + 3], 4);
    if (v < 0 || v >= nv || L.pos_of_vertex[v] != p) return false;
  }
  for (int64_t i = 0; i < 2 * ne; ++i)
    if (L.edges[i] < 0 || L.edges[i] >= nv) return false;
  for (int64_t f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k)
      if (L.tris[4 * f + k] < 0 || L.tris[4 * f + k] >= nv) return false;
  // rows, their chunks and super-chunks
  if (L.row_off[0] != 0 || L.chunk_off[0] != 0 || L.super_off[0] != 0 ||
      (int64_t)L.row_off[nv] != L.n_entries)
    return false;
  int64_t maxl = 0;
  for (int64_t p = 0; p < nv; ++p) {
    if (L.row_off[p + 1] < L.row_off[p] || L.chunk_off[p + 1] < L.chunk_off[p] ||
        L.super_off[p + 1] < L.super_off[p])
      return false;
    const int64_t len = L.row_off[p + 1] - L.row_off[p];
    const int64_t nc = L.chunk_off[p + 1] - L.chunk_off[p];
    if (nc != (len + K - 1) / K || L.super_off[p + 1] - L.super_off[p] != (nc + K - 1) / K)
      return false;
    maxl = std::max(maxl, len);
  }
  if (maxl != L.max_list) return false;
  // typed ids of the entries
  for (int64_t j = 0; j < L.n_entries; ++j) {
    const uint32_t w = L.entries[4 * j], type = w >> 30, id = w & ((1u << 30) - 1);
    if (!((type == 1 && id < (uint64_t)ne) || (type == 2 && id < (uint64_t)nf))) return false;
  }
  // Voronoi neighbours and their inline copies
  if (L.nb_off[0] != 0) return false;
  for (int64_t p = 0; p < nv; ++p)
    if (L.nb_off[p + 1] < L.nb_off[p]) return false;
  for (size_t j = 0; j < L.nb.size(); ++j) {
    uint32_t r;
    std::memcpy(&r, &L.nbp[4 * j + 3], 4);
    if (L.nb[j] >= (uint64_t)nv || r != L.nb[j]) return false;
  }
  return true;
}

}  // namespace

extern "C" {

p2m_status p2m_save(const p2m_handle *h, const char *path) {
  if (!h || !path) return P2M_ERR_INVALID_ARG;
  FILE *f = fopen(path, "wb");
  if (!f) return P2M_ERR_IO;
  const Layout &L = h->L;
  uint64_t ck = 1469598103934665603ull;
  int64_t scal[12] = {L.nv, L.nf, L.ne, L.kd_depth, L.n_entries, L.max_list,
                      L.neighbour_pairs, L.inspections, L.cert_rounds, L.cert_queries,
                      L.n_degenerate, 0};
  float fl[19];
  std::memcpy(fl, L.dom, 24);
  fl[6] = L.delta;
  std::memcpy(fl + 7, L.kd_root, 24);
  std::memcpy(fl + 13, L.qframe_lo, 12);
  std::memcpy(fl + 16, L.qframe_inv, 12);
  bool ok = fwrite(&kMagic, 8, 1, f) == 1 && fwrite(&kVersion, 4, 1, f) == 1 &&
            fwrite(scal, 8, 12, f) == 12 && fwrite(fl, 4, 19, f) == 19;
  ck = fnv1a(ck, scal, sizeof(scal));
  ck = fnv1a(ck, fl, sizeof(fl));
  ok = ok && put_vec(f, L.kd_nodes, ck) && put_vec(f, L.kd_points, ck) &&
       put_vec(f, L.pos_of_vertex, ck) && put_vec(f, L.row_off, ck) && put_vec(f, L.entries, ck) &&
       put_vec(f, L.edge_rec, ck) && put_vec(f, L.face_rec, ck) && put_vec(f, L.edges, ck) &&
       put_vec(f, L.tris, ck) && put_vec(f, L.nb_off, ck) && put_vec(f, L.nb, ck) &&
       put_vec(f, L.chunk_off, ck) && put_vec(f, L.chunks, ck) && put_vec(f, L.nbp, ck) &&
       put_vec(f, L.super_off, ck) && put_vec(f, L.supers, ck);
  ok = ok && fwrite(&ck, 8, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  return ok ? P2M_OK : P2M_ERR_IO;
}

p2m_status p2m_load(const char *path, p2m_handle **out) {
  if (!path || !out) return P2M_ERR_INVALID_ARG;
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) return P2M_ERR_IO;
  std::unique_ptr<p2m_handle> h(new (std::nothrow) p2m_handle());
  if (!h) {
    fclose(f);
    return P2M_ERR_OOM;
  }
  Layout &L = h->L;
  uint64_t magic = 0, ck = 1469598103934665603ull, stored = 0;
  uint32_t ver = 0;
  int64_t scal[12];
  float fl[19];
  bool ok = fread(&magic, 8, 1, f) == 1 && magic == kMagic && fread(&ver, 4, 1, f) == 1 &&
            ver == kVersion && fread(scal, 8, 12, f) == 12 && fread(fl, 4, 19, f) == 19;
  if (ok) {
    ck = fnv1a(ck, scal, sizeof(scal));
    ck = fnv1a(ck, fl, sizeof(fl));
    ok = get_vec(f, L.kd_nodes, ck) && get_vec(f, L.kd_points, ck) &&
         get_vec(f, L.pos_of_vertex, ck) && get_vec(f, L.row_off, ck) &&
         get_vec(f, L.entries, ck) && get_vec(f, L.edge_rec, ck) && get_vec(f, L.face_rec, ck) &&
         get_vec(f, L.edges, ck) && get_vec(f, L.tris, ck) && get_vec(f, L.nb_off, ck) &&
         get_vec(f, L.nb, ck) && get_vec(f, L.chunk_off, ck) && get_vec(f, L.chunks, ck) &&
         get_vec(f, L.nbp, ck) && get_vec(f, L.super_off, ck) && get_vec(f, L.supers, ck) &&
         fread(&stored, 8, 1, f) == 1 && stored == ck;
  }
  fclose(f);
  if (!ok) return P2M_ERR_IO;
  L.nv = scal[0];
  L.nf = scal[1];
  L.ne = scal[2];
  L.kd_depth = (int)scal[3];
  L.n_entries = scal[4];
  L.max_list = scal[5];
  L.neighbour_pairs = scal[6];
  L.inspections = scal[7];
  L.cert_rounds = scal[8];
  L.cert_queries = scal[9];
  L.n_degenerate = scal[10];
  std::memcpy(L.dom, fl, 24);
  L.delta = fl[6];
  std::memcpy(L.kd_root, fl + 7, 24);
  std::memcpy(L.qframe_lo, fl + 13, 12);
  std::memcpy(L.qframe_inv, fl + 16, 12);
  if ((int64_t)L.row_off.size() != L.nv + 1 || (int64_t)L.kd_points.size() != 4 * L.nv ||
      (int64_t)L.entries.size() != 4 * L.n_entries || (int64_t)L.edges.size() != 2 * L.ne ||
      (int64_t)L.nb_off.size() != L.nv + 1 || (int64_t)L.nb.size() != (int64_t)L.nb_off.back() ||
      (int64_t)L.chunk_off.size() != L.nv + 1 ||
      (int64_t)L.chunks.size() != 4 * (int64_t)L.chunk_off.back() ||
      L.nbp.size() != 4 * L.nb.size() || (int64_t)L.super_off.size() != L.nv + 1 ||
      L.supers.size() != 4 * (size_t)L.super_off.back() || !layout_consistent(L))
    return P2M_ERR_IO;
  if (have_device() && cudaGetDevice(&h->device) == cudaSuccess) {
    cudaError_t e = h->upload_tree();
    if (e == cudaSuccess) e = h->upload_rest();
    if (e != cudaSuccess) return from_cuda(e);
  } else {
    h->device = -1;
  }
  *out = h.release();
  return P2M_OK;
}

}  // extern "C"

// Read-only access to a handle's device view and tuning for other
// translation units of this library (not part of the C ABI).
namespace p2m {
bool handle_view(const p2m_handle *h, DevView *v, QueryTuning *t) {
  if (!h || h->device < 0) return false;
  *v = h->view;
  *t = h->tune;
  return true;
}
}  // namespace p2m

