// flood.cu -- the builder's flooding inspection (Alg. 1) on the device.
//
// A persistent kernel: one block of kFloodWarps warps per SM, each warp
// taking primitives from an atomic counter and flooding them with its 32
// lanes (flood_warp.h: breadth-first over Voronoi neighbours, the cut of
// each visited cell by the primitive's Space-perp half-spaces, the filter of
// Thm. 5/6 and the Region box of Sec. 4.6, the per-point work spread over
// the lanes).  A warp's work polytopes and queue live in shared memory;
// records are appended to one array through an atomic counter and the host
// sorts them into rows as it does its own.  This translation unit is
// compiled with -fmad=false: every double operation rounds on its own, as
// on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>

#include "flood.h"
#include "flood_core.h"
#include "flood_warp.h"

namespace p2m {
namespace {

constexpr int kFloodWarps = 8;  // warps per block, one block per SM

// the device side of the flat problem: records through an atomic counter
struct DevEnv : fc::Flat {
  FloodRec *rec;
  unsigned long long *count;
  unsigned long long cap;

  __device__ void emit(int32_t row, int32_t typed_id, const float box[6]) {
    const unsigned long long slot = atomicAdd(count, 1ull);
    if (slot < cap) {
      FloodRec r;
      r.row = row;
      r.tid = typed_id;
      for (int d = 0; d < 6; ++d) r.box[d] = box[d];
      rec[slot] = r;
    }
  }
};

__global__ void __launch_bounds__(kFloodWarps * 32, 1)
    k_flood_warp(DevEnv env, int64_t n, double eps, double delta, double eta, uint8_t *gave_up,
                 unsigned long long *insp_total, unsigned long long *next, int32_t *seen,
                 int64_t nv) {
  extern __shared__ __align__(16) unsigned char flood_smem[];
  fw::WarpWork &S = reinterpret_cast<fw::WarpWork *>(flood_smem)[threadIdx.x >> 5];
  // this warp's row stamps (null: the queue is scanned instead)
  int32_t *my_seen =
      seen ? seen + ((int64_t)blockIdx.x * kFloodWarps + (threadIdx.x >> 5)) * nv : nullptr;
  DevEnv e = env;
  for (;;) {
    P2M_LANE0 { S.item = (int64_t)atomicAdd(next, 1ull); }
    P2M_SYNC;
    const int64_t k = S.item;
    P2M_SYNC;
    if (k >= n) return;
    int64_t insp = 0;
    const int r = fw::flood_warp(S, e, k, eps, delta, eta, insp, my_seen);
    P2M_LANE0 {
      gave_up[k] = (uint8_t)(r != 0);
      if (r == 0) atomicAdd(insp_total, (unsigned long long)insp);
    }
  }
}

// device buffers of one call, freed together
struct Bufs {
  std::vector<void *> p;
  ~Bufs() {
    for (void *q : p) cudaFree(q);
  }
  template <class T>
  T *get(size_t count, cudaError_t &e) {
    void *q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return nullptr;
    p.push_back(q);
    return (T *)q;
  }
  template <class T>
  T *put(const T *src, size_t count, cudaError_t &e) {
    T *d = get<T>(count, e);
    if (e == cudaSuccess && count)
      e = cudaMemcpy(d, src, count * sizeof(T), cudaMemcpyHostToDevice);
    return d;
  }
};

}  // namespace

bool flood_on_device(const FloodProblem &pb, std::vector<FloodRec> &out,
                     std::vector<uint8_t> &gave_up, int64_t &inspections) {
  out.clear();
  gave_up.clear();
  inspections = 0;
  if (pb.n <= 0 || pb.nv <= 0) return false;
  const int64_t nv = pb.nv, n = pb.n;
  const int64_t npt = pb.cell_pt_off[nv], nbeg = pb.cell_beg_off[nv];
  const int64_t nnb = pb.nb_off[nv], nperp = pb.perp_off[n];
  // optional timing of the steps on stderr (P2M_BUILD_TRACE=1)
  const bool trace = std::getenv("P2M_BUILD_TRACE") != nullptr;
  auto ms = [] {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
  };
  double t0 = ms(), t1 = t0, t2 = t0;
  const size_t smem = kFloodWarps * sizeof(fw::WarpWork);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flood_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  {
    Bufs B;
    DevEnv env;
    env.pt_off = B.put(pb.cell_pt_off, nv + 1, e);
    env.pt = (const fc::D3 *)B.put(pb.cell_pt, 3 * (size_t)npt, e);
    env.beg_off = B.put(pb.cell_beg_off, nv + 1, e);
    env.beg = B.put(pb.cell_beg, (size_t)nbeg, e);
    env.pos = (const fc::D3 *)B.put(pb.pv, 3 * (size_t)nv, e);
    env.vids = B.put(pb.vid, (size_t)nv, e);
    env.nbo = B.put(pb.nb_off, nv + 1, e);
    env.nbs = B.put(pb.nb, (size_t)nnb, e);
    env.perp_off = B.put(pb.perp_off, n + 1, e);
    env.perp = B.put(pb.perp, 4 * (size_t)nperp, e);
    env.gtype = B.put(pb.gtype, (size_t)n, e);
    env.g = B.put(pb.g, 6 * (size_t)n, e);
    env.seed_row = B.put(pb.seed_row, 3 * (size_t)n, e);
    env.seed_vid = B.put(pb.seed_vid, 3 * (size_t)n, e);
    env.tid = B.put(pb.tid, (size_t)n, e);
    uint8_t *dgave = B.get<uint8_t>((size_t)n, e);
    // records, inspections, work counter
    unsigned long long *cnt = B.get<unsigned long long>(3, e);
    // room for 128 records a primitive (the workload meshes take 15 to 45
    // on average over all primitives, but up to about 100 over their faces
    // alone, and a call may be given faces only), within half the free
    // device memory; a second run with the exact count when that is not
    // enough (the record set of a run is deterministic)
    size_t free_bytes = 0, total_bytes = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_bytes, &total_bytes);
    unsigned long long cap = std::max<unsigned long long>(
        1ull << 20, std::min<unsigned long long>(128ull * (unsigned long long)n,
                                                 free_bytes / 2 / sizeof(FloodRec)));
    int runs = 0;
    unsigned long long h_cnt[2] = {0, 0};
    // one row stamp per warp and row (4 bytes each: 3.2 GB for the 655k rows of
    // the 1.3M-triangle mesh), when that fits in 8 GB; else the warps scan
    // their queues
    int32_t *seen = nullptr;
    const size_t seen_bytes = sizeof(int32_t) * (size_t)sms * kFloodWarps * (size_t)nv;
    if (e == cudaSuccess && seen_bytes <= ((size_t)8 << 30)) {
      if (cudaMalloc((void **)&seen, seen_bytes) == cudaSuccess) {
        B.p.push_back(seen);
      } else {
        cudaGetLastError();
        seen = nullptr;
      }
    }
    for (int attempt = 0; attempt < 2 && e == cudaSuccess; ++attempt) {
      FloodRec *drec = B.get<FloodRec>((size_t)cap, e);
      if (e != cudaSuccess) break;
      e = cudaMemset(cnt, 0, 3 * sizeof(unsigned long long));
      if (e == cudaSuccess && seen) e = cudaMemset(seen, 0, seen_bytes);
      if (e != cudaSuccess) break;
      env.rec = drec;
      env.count = cnt;
      env.cap = cap;
      if (runs++ == 0) t1 = ms();
      k_flood_warp<<<sms, kFloodWarps * 32, smem>>>(env, n, pb.eps, pb.delta, pb.eta, dgave,
                                                     cnt + 1, cnt + 2, seen, nv);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      t2 = ms();
      if (e == cudaSuccess) e = cudaMemcpy(h_cnt, cnt, sizeof(h_cnt), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      if (h_cnt[0] <= cap) {
        out.resize((size_t)h_cnt[0]);
        gave_up.resize((size_t)n);
        e = cudaMemcpy(out.data(), drec, sizeof(FloodRec) * out.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
          e = cudaMemcpy(gave_up.data(), dgave, (size_t)n, cudaMemcpyDeviceToHost);
        break;
      }
      cap = h_cnt[0];
      cudaFree(drec);
      B.p.pop_back();
    }
    if (e == cudaSuccess && gave_up.size() != (size_t)n) e = cudaErrorUnknown;
    inspections = (int64_t)h_cnt[1];
    if (trace)
      std::fprintf(stderr,
                   "p2m build:   device flooding: %lld primitives, upload %.0f ms, kernel %.0f ms, "
                   "download %.0f ms (%llu records, %d run(s))\n",
                   (long long)n, t1 - t0, t2 - t1, ms() - t2, h_cnt[0], runs);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    out.clear();
    gave_up.clear();
    inspections = 0;
    return false;
  }
  return true;
}

}  // namespace p2m
