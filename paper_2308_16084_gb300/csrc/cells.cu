// cells.cu -- the Voronoi cells of the builder (Alg. A.1's cells, clipped
// to D) on the device, in the host builder's rounds.
//
// The cells are made a chunk at a time; each cell keeps its state in device
// memory (cw::CellSlot).  A seeding kernel makes every cell of the chunk from
// the box and its 32 nearest vertices; then each round a corner kernel lists
// every open cell's far corners not settled in an earlier round in one
// search list (atomic offsets), the
// batched exact search (certify.cu, full occupancy) answers all of them,
// and an apply kernel cuts every cell by the vertices its corners found; a
// widening kernel finally writes the neighbours and the widened cells,
// appended to three arrays through atomic counters, which the host puts in
// row order.  The kernels are persistent (one block of kCellWarps warps per
// SM, rows from an atomic counter) and each warp works on one cell at a time
// with its 32 lanes (cell_warp.h), its polytopes and cut work space in
// shared memory.  This translation unit is compiled with -fmad=false: every
// double operation rounds on its own, as on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <thread>
#include <vector>

#include "cell_core.h"
#include "cell_warp.h"
#include "cells.h"
#include "certify.h"

namespace p2m {
namespace {

constexpr int kCellWarps = 8;          // warps per block, one block per SM
constexpr int64_t kChunk = 1 << 18;    // cells whose state is held at once (2 GB)
constexpr int64_t kCornersPerCell = 64;  // room in a round's search list, on average

// the KD tree as the cell phases read it (float points and boxes, exact in
// double)
struct CellEnv {
  DevView m;
  __device__ int64_t nleaf0() const { return m.L - 1; }
  __device__ int64_t leaf_first(int64_t j) const { return (j * m.nv) >> m.depth; }
  __device__ fc::D3 pos(int64_t p) const {
    const float4 c = __ldg(&m.kd_points[p]);
    return {(double)c.x, (double)c.y, (double)c.z};
  }
  __device__ void child_boxes(int64_t node, double b0[6], double b1[6]) const {
    const float4 A = __ldg(&m.kd_nodes[3 * node + 0]);
    const float4 B = __ldg(&m.kd_nodes[3 * node + 1]);
    const float4 C = __ldg(&m.kd_nodes[3 * node + 2]);
    b0[0] = A.x; b0[1] = A.y; b0[2] = A.z; b0[3] = A.w; b0[4] = B.x; b0[5] = B.y;
    b1[0] = B.z; b1[1] = B.w; b1[2] = C.x; b1[3] = C.y; b1[4] = C.z; b1[5] = C.w;
  }
};

// a chunk of cells: rows c0 .. c0 + n - 1, their slots, the warps' work
// space and the kernel's row counter
struct Chunk {
  int64_t c0, n;
  cw::CellSlot *slots;
  cw::CellExtra *extra;
  unsigned long long *next;
};

// a round's search list: corners xs (3 doubles), bounds rs, answers wres
struct SearchList {
  double *xs, *rs;
  int64_t *wres;
  unsigned long long *used;
  unsigned long long cap;
};

// where the results go: per row info[6p ..] = point offset (-1: handed
// back), point count, loop-start offset, loop-start count (nf + 1),
// neighbour offset, neighbour count; cnt = points, loop starts, neighbours
// used, most rounds of a kept cell, corners searched by kept cells
struct CellSink {
  int64_t *info;
  fc::D3 *pt;
  int32_t *beg;
  int32_t *nb;
  unsigned long long *cnt;
  unsigned long long cap_pt, cap_beg, cap_nb;
};

// the warp's shared work space and its next cell (i: index in the chunk,
// -1 when none is left)
__device__ __forceinline__ int64_t next_cell(fw::WarpWork &S, const Chunk &ch) {
  P2M_LANE0 { S.item = (int64_t)atomicAdd(ch.next, 1ull); }
  P2M_SYNC;
  const int64_t i = S.item;
  P2M_SYNC;
  return i < ch.n ? i : -1;
}

#define CELL_WARP_SETUP                                                        \
  extern __shared__ __align__(16) unsigned char cell_smem[];                  \
  const int wid = threadIdx.x >> 5;                                           \
  fw::WarpWork &S = reinterpret_cast<fw::WarpWork *>(cell_smem)[wid];         \
  cw::CellExtra &X = ch.extra[(int64_t)blockIdx.x * kCellWarps + wid];

__global__ void __launch_bounds__(kCellWarps * 32, 1)
    k_cell_seed(CellEnv env, cc::CellParams cp, Chunk ch) {
  CELL_WARP_SETUP
  for (int64_t i; (i = next_cell(S, ch)) >= 0;)
    cw::cell_seed(S, X, env, ch.c0 + i, cp, ch.slots[i]);
}

// the far corners of every open cell into the round's search list
__global__ void __launch_bounds__(kCellWarps * 32, 1)
    k_cell_corners(CellEnv env, double epsc, Chunk ch, SearchList sl) {
  CELL_WARP_SETUP
  for (int64_t i; (i = next_cell(S, ch)) >= 0;) {
    cw::CellSlot &c = ch.slots[i];
    if (c.status != cw::kOpen) continue;
    const fc::D3 pv = env.pos(ch.c0 + i);
    const int m = cw::round_corners(X, c, pv);
    // the far corners not settled in an earlier round go to the search
    const int ms = m > 0 ? cw::round_unsettled(X, c, m) : 0;
    P2M_LANE0 {
      X.flag = 0;
      c.m = 0;
      if (m > 0) {
        c.rounds += 1;
        c.queries += m;
      }
      if (ms == 0) {
        c.status = cw::kDone;  // no far corner, or every one settled
      } else {
        const unsigned long long at = atomicAdd(sl.used, (unsigned long long)ms);
        X.out_at[0] = at;
        if (at + ms > sl.cap) {
          c.status = cw::kGaveUp;  // no room left: the host makes this cell
          X.flag = at < sl.cap ? 2 : 0;
        } else {
          c.corner_at = (int64_t)at;
          c.m = ms;
          X.flag = 1;
        }
      }
    }
    P2M_SYNC;
    const unsigned long long at = X.out_at[0];
    if (X.flag == 1) {
      P2M_LANES(l)
        for (int j = l; j < ms; j += 32) {
          const fc::D3 x = X.sorted[j];
          sl.xs[3 * (at + j)] = x.x;
          sl.xs[3 * (at + j) + 1] = x.y;
          sl.xs[3 * (at + j) + 2] = x.z;
          sl.rs[at + j] = fc::len2(x - pv) - epsc;
        }
      P2M_END_LANES
    } else if (X.flag == 2) {
      // the part of the list this cell reserved before it ran out: bounds
      // that end its searches at once
      P2M_LANES(l)
        for (unsigned long long j = at + l; j < sl.cap; j += 32) {
          sl.xs[3 * j] = sl.xs[3 * j + 1] = sl.xs[3 * j + 2] = 0.0;
          sl.rs[j] = -1.0;
        }
      P2M_END_LANES
    }
    P2M_SYNC;
  }
}

// every cell with far corners cut by the vertices they found
__global__ void __launch_bounds__(kCellWarps * 32, 1)
    k_cell_apply(CellEnv env, cc::CellParams cp, Chunk ch, const double *__restrict__ xs,
                 const int64_t *__restrict__ wres) {
  CELL_WARP_SETUP
  for (int64_t i; (i = next_cell(S, ch)) >= 0;) {
    cw::CellSlot &c = ch.slots[i];
    if (c.status != cw::kOpen || c.m == 0) continue;
    cw::round_apply(S, X, env, ch.c0 + i, cp, c, xs + 3 * c.corner_at, wres + c.corner_at);
  }
}

// the neighbours and widened cells of the chunk's kept cells
__global__ void __launch_bounds__(kCellWarps * 32, 1)
    k_cell_widen(CellEnv env, cc::CellParams cp, Chunk ch, CellSink o) {
  CELL_WARP_SETUP
  for (int64_t i; (i = next_cell(S, ch)) >= 0;) {
    const cw::CellSlot &c = ch.slots[i];
    const int64_t p = ch.c0 + i;
    int64_t *info = o.info + 6 * p;
    if (c.status == cw::kGaveUp) {
      P2M_LANE0 { info[0] = -1; }
      P2M_SYNC;
      continue;
    }
    const fw::WPoly *w = nullptr;
    const bool ok = cw::cell_widen(S, X, env, p, cp, c, w);
    P2M_LANE0 {
      info[0] = -1;
      X.flag = 0;
      if (ok) {
        const unsigned long long np = (unsigned long long)w->np,
                                 nb = (unsigned long long)(w->nf + 1),
                                 nn = (unsigned long long)X.nb_n;
        X.out_at[0] = atomicAdd(&o.cnt[0], np);
        X.out_at[1] = atomicAdd(&o.cnt[1], nb);
        X.out_at[2] = atomicAdd(&o.cnt[2], nn);
        X.flag = (X.out_at[0] + np <= o.cap_pt && X.out_at[1] + nb <= o.cap_beg &&
                  X.out_at[2] + nn <= o.cap_nb)
                     ? 1
                     : 0;
      }
    }
    P2M_SYNC;
    if (!X.flag) continue;
    const unsigned long long a = X.out_at[0], b = X.out_at[1], cc_ = X.out_at[2];
    P2M_LANES(l)
      for (int k = l; k < w->np; k += 32) o.pt[a + k] = w->pt[k];
      for (int k = l; k <= w->nf; k += 32) o.beg[b + k] = w->beg[k];
      for (int k = l; k < X.nb_n; k += 32) o.nb[cc_ + k] = X.nb[k];
    P2M_END_LANES
    P2M_LANE0 {
      info[1] = (int64_t)w->np;
      info[2] = (int64_t)b;
      info[3] = (int64_t)(w->nf + 1);
      info[4] = (int64_t)cc_;
      info[5] = (int64_t)X.nb_n;
      info[0] = (int64_t)a;
      atomicMax(&o.cnt[3], (unsigned long long)c.rounds);
      atomicAdd(&o.cnt[4], (unsigned long long)c.queries);
    }
    P2M_SYNC;
  }
}

}  // namespace

bool cells_on_device(const DevView &m, const CellProblem &pb, CellResult &out) {
  out = CellResult();
  const int64_t nv = pb.nv;
  if (nv <= 0 || nv != m.nv) return false;
  // optional timing on stderr (P2M_BUILD_TRACE=1)
  const bool trace = std::getenv("P2M_BUILD_TRACE") != nullptr;
  auto ms = [] {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
  };
  const double t0 = ms();
  double t_search = 0;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = kCellWarps * sizeof(fw::WarpWork);
  const cudaFuncAttribute big = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cell_seed, big, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cell_corners, big, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cell_apply, big, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cell_widen, big, (int)smem);
  const int64_t chunk = std::min<int64_t>(nv, kChunk);
  // one block per SM, or fewer when the rows are few
  const int64_t blocks = std::max<int64_t>(
      1, std::min<int64_t>(std::max(sms, 1), (chunk + kCellWarps - 1) / kCellWarps));
  // room for 256 points, 64 loops and 64 neighbours a cell on average (the
  // widened cells of the workload meshes hold 60 to 130 points); a cell past
  // the room is handed back
  const unsigned long long cap_pt = (unsigned long long)std::max<int64_t>(1 << 16, 256 * nv);
  const unsigned long long cap_beg = (unsigned long long)std::max<int64_t>(1 << 14, 64 * nv);
  const unsigned long long cap_nb = cap_beg;
  std::vector<void *> bufs;
  auto get = [&](size_t bytes) -> void * {
    void *q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, std::max<size_t>(bytes, 1));
    if (e != cudaSuccess) return nullptr;
    bufs.push_back(q);
    return q;
  };
  CellSink o;
  o.info = (int64_t *)get(sizeof(int64_t) * 6 * (size_t)nv);
  o.pt = (fc::D3 *)get(sizeof(fc::D3) * cap_pt);
  o.beg = (int32_t *)get(sizeof(int32_t) * cap_beg);
  o.nb = (int32_t *)get(sizeof(int32_t) * cap_nb);
  o.cnt = (unsigned long long *)get(5 * sizeof(unsigned long long));
  o.cap_pt = cap_pt;
  o.cap_beg = cap_beg;
  o.cap_nb = cap_nb;
  Chunk ch;
  ch.slots = (cw::CellSlot *)get(sizeof(cw::CellSlot) * (size_t)chunk);
  ch.extra = (cw::CellExtra *)get(sizeof(cw::CellExtra) * (size_t)(blocks * kCellWarps));
  ch.next = (unsigned long long *)get(2 * sizeof(unsigned long long));
  SearchList sl;
  sl.cap = (unsigned long long)(kCornersPerCell * chunk);
  sl.xs = (double *)get(3 * sizeof(double) * sl.cap);
  sl.rs = (double *)get(sizeof(double) * sl.cap);
  sl.wres = (int64_t *)get(sizeof(int64_t) * sl.cap);
  sl.used = ch.next + 1;
  if (e == cudaSuccess) e = cudaMemset(o.cnt, 0, 5 * sizeof(unsigned long long));
  CellEnv env;
  env.m = m;
  cc::CellParams cp;
  for (int d = 0; d < 3; ++d) {
    cp.lo[d] = pb.lo[d];
    cp.hi[d] = pb.hi[d];
  }
  cp.eps = pb.eps;
  cp.epsc = pb.epsc;
  cp.delta = pb.delta;
  const unsigned grid = (unsigned)blocks, threads = kCellWarps * 32;
  auto reset = [&] {
    if (e == cudaSuccess) e = cudaMemset(ch.next, 0, 2 * sizeof(unsigned long long));
  };
  for (int64_t c0 = 0; c0 < nv && e == cudaSuccess; c0 += chunk) {
    ch.c0 = c0;
    ch.n = std::min(chunk, nv - c0);
    reset();
    if (e == cudaSuccess) k_cell_seed<<<grid, threads, smem>>>(env, cp, ch);
    for (int round = 0; round < cc::kRounds && e == cudaSuccess; ++round) {
      reset();
      if (e == cudaSuccess) k_cell_corners<<<grid, threads, smem>>>(env, cp.epsc, ch, sl);
      unsigned long long used = 0;
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess)
        e = cudaMemcpy(&used, sl.used, sizeof(used), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess || used == 0) break;
      const double ts = ms();
      e = launch_nearest_within_f64(m, sl.xs, sl.rs, (int64_t)std::min(used, sl.cap), sl.wres, 0);
      if (e == cudaSuccess && trace) e = cudaDeviceSynchronize();
      t_search += ms() - ts;
      reset();
      if (e == cudaSuccess) k_cell_apply<<<grid, threads, smem>>>(env, cp, ch, sl.xs, sl.wres);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    reset();
    if (e == cudaSuccess) k_cell_widen<<<grid, threads, smem>>>(env, cp, ch, o);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  const double t2 = ms();
  std::vector<int64_t> info;
  std::vector<fc::D3> pt;
  std::vector<int32_t> beg, nb;
  unsigned long long cnt[5] = {0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(cnt, o.cnt, sizeof(cnt), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    info.resize(6 * (size_t)nv);
    pt.resize((size_t)std::min(cnt[0], cap_pt));
    beg.resize((size_t)std::min(cnt[1], cap_beg));
    nb.resize((size_t)std::min(cnt[2], cap_nb));
    e = cudaMemcpy(info.data(), o.info, sizeof(int64_t) * info.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && !pt.empty())
      e = cudaMemcpy(pt.data(), o.pt, sizeof(fc::D3) * pt.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && !beg.empty())
      e = cudaMemcpy(beg.data(), o.beg, sizeof(int32_t) * beg.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && !nb.empty())
      e = cudaMemcpy(nb.data(), o.nb, sizeof(int32_t) * nb.size(), cudaMemcpyDeviceToHost);
  }
  for (void *q : bufs) cudaFree(q);
  if (e != cudaSuccess) {
    cudaGetLastError();
    out = CellResult();
    return false;
  }
  // row order
  out.gave_up.assign((size_t)nv, 0);
  out.nb_off.assign((size_t)nv + 1, 0);
  out.pt_off.assign((size_t)nv + 1, 0);
  out.beg_off.assign((size_t)nv + 1, 0);
  int64_t handed = 0;
  for (int64_t p = 0; p < nv; ++p) {
    const int64_t *r = &info[6 * (size_t)p];
    const bool ok = r[0] >= 0 && (uint64_t)(r[0] + r[1]) <= pt.size() &&
                    (uint64_t)(r[2] + r[3]) <= beg.size() && (uint64_t)(r[4] + r[5]) <= nb.size();
    out.gave_up[p] = ok ? 0 : 1;
    handed += ok ? 0 : 1;
    out.pt_off[p + 1] = out.pt_off[p] + (ok ? r[1] : 0);
    out.beg_off[p + 1] = out.beg_off[p] + (ok ? r[3] : 0);
    out.nb_off[p + 1] = out.nb_off[p] + (ok ? r[5] : 0);
  }
  out.rounds = (int64_t)cnt[3];
  out.queries = (int64_t)cnt[4];
  out.pt.resize(3 * (size_t)out.pt_off[nv]);
  out.beg.resize((size_t)out.beg_off[nv]);
  out.nb.resize((size_t)out.nb_off[nv]);
  // the rows' copies are independent: spread them over the host's cores
  auto gather = [&](int64_t p0, int64_t p1) {
    for (int64_t p = p0; p < p1; ++p) {
      if (out.gave_up[p]) continue;
      const int64_t *r = &info[6 * (size_t)p];
      for (int64_t i = 0; i < r[1]; ++i) {
        const fc::D3 x = pt[(size_t)(r[0] + i)];
        double *d = &out.pt[3 * (size_t)(out.pt_off[p] + i)];
        d[0] = x.x;
        d[1] = x.y;
        d[2] = x.z;
      }
      std::copy(beg.begin() + r[2], beg.begin() + r[2] + r[3], out.beg.begin() + out.beg_off[p]);
      std::copy(nb.begin() + r[4], nb.begin() + r[4] + r[5], out.nb.begin() + out.nb_off[p]);
    }
  };
  const int64_t nthreads =
      std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(), nv / 4096));
  std::vector<std::thread> pool;
  for (int64_t t = 0; t < nthreads; ++t)
    pool.emplace_back(gather, nv * t / nthreads, nv * (t + 1) / nthreads);
  for (auto &th : pool) th.join();
  if (trace)
    std::fprintf(stderr,
                 "p2m build:   device cells: %.0f ms on the device (searches %.0f ms), gather "
                 "%.0f ms (%lld of %lld cells handed back)\n",
                 t2 - t0, t_search, ms() - t2, (long long)handed, (long long)nv);
  return true;
}

}  // namespace p2m
