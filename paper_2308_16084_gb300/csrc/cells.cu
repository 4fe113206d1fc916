// cells.cu -- the Voronoi cells of the builder (Alg. A.1's cells, clipped
// to D) on the device.
//
// A persistent kernel: one block of kCellWarps warps per SM, each warp
// taking rows from an atomic counter and making their cells with its 32
// lanes (cell_warp.h: the 32-nearest seeding, the certification rounds with
// the exact search inline (within_core.h), one corner per lane, and the
// widened cell; the cuts spread over the lanes as in the flooding).  A
// warp's polytopes and cut work space live in shared memory, the rest of its
// state in a block of device memory of its own.  The neighbours and widened
// cells are appended to three arrays through atomic counters; the host puts
// them in row order.  This translation unit is compiled with -fmad=false:
// every double operation rounds on its own, as on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>

#include "cell_core.h"
#include "cell_warp.h"
#include "cells.h"
#include "within_core.h"

namespace p2m {
namespace {

constexpr int kCellWarps = 8;  // warps per block, one block per SM

// the KD tree as the cell core reads it (float points and boxes, exact in
// double), with the exact search of the certification
struct CellEnv {
  DevView m;
  double s;  // the search's coordinate scale (within_core.h)
  __device__ int64_t nleaf0() const { return m.L - 1; }
  __device__ int64_t leaf_first(int64_t j) const { return wc::leaf_first(m, j); }
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
  __device__ int64_t within(fc::D3 x, double r2) const {
    return wc::nearest_within(m, x.x, x.y, x.z, r2, s);
  }
};

// where the results go: per row info[6p ..] = point offset (-1: handed
// back), point count, loop-start offset, loop-start count (nf + 1),
// neighbour offset, neighbour count; cnt = points, loop starts, neighbours
// used, next row, most rounds of a kept cell, corners searched by kept cells
struct CellSink {
  int64_t *info;
  fc::D3 *pt;
  int32_t *beg;
  int32_t *nb;
  unsigned long long *cnt;
  unsigned long long cap_pt, cap_beg, cap_nb;
};

__global__ void __launch_bounds__(kCellWarps * 32, 1)
    k_cells(CellEnv env, cc::CellParams cp, int64_t nv, cw::CellExtra *extra, CellSink o) {
  extern __shared__ __align__(16) unsigned char cell_smem[];
  const int wid = threadIdx.x >> 5;
  fw::WarpWork &S = reinterpret_cast<fw::WarpWork *>(cell_smem)[wid];
  cw::CellExtra &X = extra[(int64_t)blockIdx.x * kCellWarps + wid];
  for (;;) {
    P2M_LANE0 { S.item = (int64_t)atomicAdd(&o.cnt[3], 1ull); }
    P2M_SYNC;
    const int64_t p = S.item;
    P2M_SYNC;
    if (p >= nv) return;
    int64_t *info = o.info + 6 * p;
    const fw::WPoly *w = nullptr;
    const int r = cw::cell_warp(S, X, env, p, cp, w);
    P2M_LANE0 {
      info[0] = -1;
      X.flag = 0;
      if (r == cc::kCellOk) {
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
    const unsigned long long a = X.out_at[0], b = X.out_at[1], c = X.out_at[2];
    P2M_LANES(l)
      for (int i = l; i < w->np; i += 32) o.pt[a + i] = w->pt[i];
      for (int i = l; i <= w->nf; i += 32) o.beg[b + i] = w->beg[i];
      for (int i = l; i < X.nb_n; i += 32) o.nb[c + i] = X.nb[i];
    P2M_END_LANES
    P2M_LANE0 {
      info[1] = (int64_t)w->np;
      info[2] = (int64_t)b;
      info[3] = (int64_t)(w->nf + 1);
      info[4] = (int64_t)c;
      info[5] = (int64_t)X.nb_n;
      info[0] = (int64_t)a;
      atomicMax(&o.cnt[4], (unsigned long long)X.rounds);
      atomicAdd(&o.cnt[5], (unsigned long long)X.queries);
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
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = kCellWarps * sizeof(fw::WarpWork);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // one block per SM, or fewer when the rows are few
  const int64_t blocks = std::max<int64_t>(
      1, std::min<int64_t>(std::max(sms, 1), (nv + kCellWarps - 1) / kCellWarps));
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
  o.cnt = (unsigned long long *)get(6 * sizeof(unsigned long long));
  o.cap_pt = cap_pt;
  o.cap_beg = cap_beg;
  o.cap_nb = cap_nb;
  cw::CellExtra *extra =
      (cw::CellExtra *)get(sizeof(cw::CellExtra) * (size_t)(blocks * kCellWarps));
  if (e == cudaSuccess) e = cudaMemset(o.cnt, 0, 6 * sizeof(unsigned long long));
  CellEnv env;
  env.m = m;
  env.s = wc::within_scale(m);
  cc::CellParams cp;
  for (int d = 0; d < 3; ++d) {
    cp.lo[d] = pb.lo[d];
    cp.hi[d] = pb.hi[d];
  }
  cp.eps = pb.eps;
  cp.epsc = pb.epsc;
  cp.delta = pb.delta;
  const double t1 = ms();
  if (e == cudaSuccess) {
    k_cells<<<(unsigned)blocks, kCellWarps * 32, smem>>>(env, cp, nv, extra, o);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  const double t2 = ms();
  std::vector<int64_t> info;
  std::vector<fc::D3> pt;
  std::vector<int32_t> beg, nb;
  unsigned long long cnt[6] = {0, 0, 0, 0, 0, 0};
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
  out.rounds = (int64_t)cnt[4];
  out.queries = (int64_t)cnt[5];
  out.pt.resize(3 * (size_t)out.pt_off[nv]);
  out.beg.resize((size_t)out.beg_off[nv]);
  out.nb.resize((size_t)out.nb_off[nv]);
  for (int64_t p = 0; p < nv; ++p) {
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
  if (trace)
    std::fprintf(stderr,
                 "p2m build:   device cells: setup %.0f ms, kernel %.0f ms, gather %.0f ms "
                 "(%lld of %lld cells handed back)\n",
                 t1 - t0, t2 - t1, ms() - t2, (long long)handed, (long long)nv);
  return true;
}

}  // namespace p2m
