// flood.cu -- the builder's flooding inspection (Alg. 1) on the device.
//
// One thread per primitive runs the core shared with the host builder
// (flood_core.h): breadth-first over Voronoi neighbours, the cut of each
// visited cell by the primitive's Space-perp half-spaces, the filter of
// Thm. 5/6 and the Region box of Sec. 4.6.  Its work polytopes live in
// local memory; records are appended to one array through an atomic counter
// and the host sorts them into rows as it does its own.  This translation
// unit is compiled with -fmad=false: every double operation rounds on its
// own, as on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "flood.h"
#include "flood_core.h"

namespace p2m {
namespace {

constexpr int kQueue = 1024;  // vertices one primitive may visit on the device

// the device side of the shared core: membership by a scan of the queue
// (every vertex seen so far is in it), records through an atomic counter
struct DevEnv : fc::Flat {
  FloodRec *rec;
  unsigned long long *count;
  unsigned long long cap;

  __device__ void mark_seed(int32_t) {}
  __device__ bool mark(int32_t w, const int32_t *queue, int64_t tail) const {
    for (int64_t k = 0; k < tail; ++k)
      if (queue[k] == w) return false;
    return true;
  }
  __device__ void emit(int32_t row, int32_t tid, const float box[6]) {
    const unsigned long long slot = atomicAdd(count, 1ull);
    if (slot < cap) {
      FloodRec r;
      r.row = row;
      r.tid = tid;
      for (int d = 0; d < 6; ++d) r.box[d] = box[d];
      rec[slot] = r;
    }
  }
};

__global__ void __launch_bounds__(128) k_flood(DevEnv env, int64_t n, double eps, double delta,
                                               double eta, uint8_t *gave_up,
                                               unsigned long long *insp_total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  fc::Prim P;
  fc::Work W;
  int32_t queue[kQueue];
  int64_t insp = 0;
  const int r = env.load(i, P) ? fc::flood_prim(P, eps, delta, eta, env, W, queue, kQueue, insp)
                               : 1;
  gave_up[i] = (uint8_t)(r != 0);
  if (r == 0) atomicAdd(insp_total, (unsigned long long)insp);
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
  // the kernel's work polytopes take ~39 KB of stack a thread; the driver
  // grows the per-thread stack for the launch and keeps it, so the previous
  // limit is put back afterwards to release that reservation
  size_t stack0 = 0;
  cudaError_t e = cudaDeviceGetLimit(&stack0, cudaLimitStackSize);
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
    unsigned long long *cnt = B.get<unsigned long long>(2, e);  // records, inspections
    // room for 16 records a primitive; a second run with the exact count
    // when that is not enough (the run is deterministic in its record set)
    unsigned long long cap = (unsigned long long)std::max<int64_t>(1 << 20, 16 * n);
    unsigned long long h_cnt[2] = {0, 0};
    for (int attempt = 0; attempt < 2 && e == cudaSuccess; ++attempt) {
      FloodRec *drec = B.get<FloodRec>((size_t)cap, e);
      if (e != cudaSuccess) break;
      e = cudaMemset(cnt, 0, 2 * sizeof(unsigned long long));
      if (e != cudaSuccess) break;
      env.rec = drec;
      env.count = cnt;
      env.cap = cap;
      const unsigned blocks = (unsigned)((n + 127) / 128);
      k_flood<<<blocks, 128>>>(env, n, pb.eps, pb.delta, pb.eta, dgave, cnt + 1);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
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
  }
  if (stack0 > 0) {
    const cudaError_t e2 = cudaDeviceSetLimit(cudaLimitStackSize, stack0);
    if (e == cudaSuccess) e = e2;
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
