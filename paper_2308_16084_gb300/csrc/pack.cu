// pack.cu -- the packing of the builder's interception table on the device.
//
// The records are bucketed by row (atomic counts, the row offsets summed on
// the host, atomic placement), each row is put in spatial order by one warp
// (its records' keys sorted in shared memory, bitonic), and one thread per
// row cuts the row into chunks and super-chunks with their codes
// (pack_core.h).  A row's order is a total order of its records, so the
// placement order inside a row does not matter.  This translation unit is
// compiled with -fmad=false: every float and double operation rounds on its
// own, as on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>

#include "pack.h"
#include "pack_core.h"

namespace p2m {
namespace {

constexpr int kSortWarps = 4;    // warps per block of the row sort
constexpr int kSortCap = 4096;   // records a warp sorts (shared memory: 40 KB a warp)

__global__ void k_pack_count(const FloodRec *__restrict__ rec, int64_t n,
                             uint32_t *__restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && rec[i].row >= 0) atomicAdd(&cnt[rec[i].row], 1u);
}

__global__ void k_pack_place(const FloodRec *__restrict__ rec, int64_t n,
                             const uint32_t *__restrict__ row_off, uint32_t *__restrict__ fill,
                             FloodRec *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const FloodRec r = rec[i];
  if (r.row < 0) return;
  out[row_off[r.row] + atomicAdd(&fill[r.row], 1u)] = r;
}

// one warp per row: the row's records (in) in spatial order into out
__global__ void __launch_bounds__(kSortWarps * 32)
    k_pack_sort(const FloodRec *__restrict__ in, const uint32_t *__restrict__ row_off, int64_t nv,
                FloodRec *__restrict__ out, unsigned int *too_long) {
  // per warp: kSortCap keys, then kSortCap indices (dynamic shared memory)
  extern __shared__ __align__(16) unsigned char sort_smem[];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  uint64_t *key = reinterpret_cast<uint64_t *>(sort_smem) + (size_t)w * kSortCap;
  uint16_t *idx = reinterpret_cast<uint16_t *>(reinterpret_cast<uint64_t *>(sort_smem) +
                                               (size_t)kSortWarps * kSortCap) +
                  (size_t)w * kSortCap;
  const unsigned full = 0xffffffffu;
  for (int64_t p = (int64_t)blockIdx.x * kSortWarps + w; p < nv;
       p += (int64_t)gridDim.x * kSortWarps) {
    const uint32_t b = row_off[p], L = row_off[p + 1] - b;
    if (L < 2) {
      if (L == 1 && l == 0) out[b] = in[b];
      continue;
    }
    if (L > (uint32_t)kSortCap) {
      if (l == 0) atomicOr(too_long, 1u);
      continue;
    }
    // the union of the row's centres (a minimum / maximum: any order)
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t j = l; j < L; j += 32) pk::centre_bounds_add(in[b + j], lo, hi);
    for (int o = 16; o > 0; o >>= 1)
      for (int d = 0; d < 3; ++d) {
        lo[d] = pk::fmin_first(lo[d], __shfl_xor_sync(full, lo[d], o));
        hi[d] = pk::fmax_first(hi[d], __shfl_xor_sync(full, hi[d], o));
      }
    uint32_t P = 2;
    while (P < L) P <<= 1;
    for (uint32_t j = l; j < P; j += 32) {
      key[j] = j < L ? pk::row_key(in[b + j], lo, hi) : ~0ull;
      idx[j] = (uint16_t)j;
    }
    __syncwarp();
    // bitonic sort of (key, index) ascending; keys are distinct in a row
    for (uint32_t k = 2; k <= P; k <<= 1)
      for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
        for (uint32_t i = l; i < P; i += 32) {
          const uint32_t x = i ^ jj;
          if (x > i) {
            const bool up = (i & k) == 0;
            const uint64_t a = key[i], c = key[x];
            if ((a > c) == up) {
              key[i] = c;
              key[x] = a;
              const uint16_t t = idx[i];
              idx[i] = idx[x];
              idx[x] = t;
            }
          }
        }
        __syncwarp();
      }
    for (uint32_t j = l; j < L; j += 32) out[b + j] = in[b + idx[j]];
    __syncwarp();
  }
}

// one thread per row: its chunks, entries and super-chunks
__global__ void k_pack_encode(const FloodRec *__restrict__ rec, const uint32_t *__restrict__ row_off,
                              const uint32_t *__restrict__ chunk_off,
                              const uint32_t *__restrict__ super_off, int64_t nv, pk::Frame fr,
                              uint32_t *__restrict__ chunks, uint32_t *__restrict__ entries,
                              uint32_t *__restrict__ supers, unsigned long long *bad) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nv) return;
  int nbad = 0;
  uint32_t c = chunk_off[p];
  for (uint32_t j = row_off[p]; j < row_off[p + 1]; j += pk::kChunk, ++c) {
    const uint32_t cnt = min(pk::kChunk, row_off[p + 1] - j);
    nbad += pk::encode_chunk(rec + j, cnt, fr.lo, fr.inv, fr.step, fr.base,
                             chunks + 4 * (size_t)c, entries + 4 * (size_t)j);
  }
  uint32_t s = super_off[p];
  for (uint32_t k = chunk_off[p]; k < chunk_off[p + 1]; k += pk::kChunk, ++s)
    pk::encode_super(chunks + 4 * (size_t)k, min(pk::kChunk, chunk_off[p + 1] - k),
                     supers + 4 * (size_t)s);
  if (nbad) atomicAdd(bad, (unsigned long long)nbad);
}

inline unsigned blocks_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

bool pack_on_device(int64_t nv, const std::vector<PackPart> &parts, const float qlo[3],
                    const float qinv[3], Layout &out, int64_t &max_list, int64_t &bad_boxes) {
  const bool trace = std::getenv("P2M_BUILD_TRACE") != nullptr;
  auto ms = [] {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
  };
  const double t0 = ms();
  int64_t n = 0;
  for (const PackPart &pp : parts) n += pp.n;
  if (nv <= 0) return false;
  cudaError_t e = cudaSuccess;
  std::vector<void *> bufs;
  auto get = [&](size_t bytes) -> void * {
    void *q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, std::max<size_t>(bytes, 1));
    if (e != cudaSuccess) return nullptr;
    bufs.push_back(q);
    return q;
  };
  auto done = [&](bool ok) {
    for (void *q : bufs) cudaFree(q);
    if (!ok) cudaGetLastError();
    return ok;
  };
  FloodRec *rec = (FloodRec *)get(sizeof(FloodRec) * (size_t)n);
  uint32_t *cnt = (uint32_t *)get(sizeof(uint32_t) * (size_t)nv);
  int64_t at = 0;
  for (const PackPart &pp : parts) {
    if (e == cudaSuccess && pp.n > 0)
      e = cudaMemcpy(rec + at, pp.rec, sizeof(FloodRec) * (size_t)pp.n, cudaMemcpyHostToDevice);
    at += pp.n;
  }
  if (e == cudaSuccess) e = cudaMemset(cnt, 0, sizeof(uint32_t) * (size_t)nv);
  if (e == cudaSuccess && n > 0) k_pack_count<<<blocks_of(n, 256), 256>>>(rec, n, cnt);
  if (e == cudaSuccess) e = cudaGetLastError();
  // the row, chunk and super-chunk offsets, summed here
  std::vector<uint32_t> c(nv);
  if (e == cudaSuccess)
    e = cudaMemcpy(c.data(), cnt, sizeof(uint32_t) * (size_t)nv, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return done(false);
  out.row_off.assign(nv + 1, 0);
  out.chunk_off.assign(nv + 1, 0);
  out.super_off.assign(nv + 1, 0);
  int64_t total = 0;
  max_list = 0;
  for (int64_t p = 0; p < nv; ++p) {
    total += c[p];
    if (total >= ((int64_t)1 << 32)) return done(false);  // the host reports it
    max_list = std::max<int64_t>(max_list, c[p]);
    out.row_off[p + 1] = (uint32_t)total;
    const uint32_t nc = (c[p] + pk::kChunk - 1) / pk::kChunk;
    out.chunk_off[p + 1] = out.chunk_off[p] + nc;
    out.super_off[p + 1] = out.super_off[p] + (nc + pk::kChunk - 1) / pk::kChunk;
  }
  const int64_t nch = out.chunk_off[nv], nsu = out.super_off[nv];
  uint32_t *row_off = (uint32_t *)get(sizeof(uint32_t) * (size_t)(nv + 1));
  uint32_t *chunk_off = (uint32_t *)get(sizeof(uint32_t) * (size_t)(nv + 1));
  uint32_t *super_off = (uint32_t *)get(sizeof(uint32_t) * (size_t)(nv + 1));
  FloodRec *placed = (FloodRec *)get(sizeof(FloodRec) * (size_t)total);
  FloodRec *sorted = (FloodRec *)get(sizeof(FloodRec) * (size_t)total);
  uint32_t *chunks = (uint32_t *)get(4 * sizeof(uint32_t) * (size_t)nch);
  uint32_t *entries = (uint32_t *)get(4 * sizeof(uint32_t) * (size_t)total);
  uint32_t *supers = (uint32_t *)get(4 * sizeof(uint32_t) * (size_t)nsu);
  unsigned long long *flags = (unsigned long long *)get(2 * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(row_off, out.row_off.data(), sizeof(uint32_t) * (size_t)(nv + 1),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(chunk_off, out.chunk_off.data(), sizeof(uint32_t) * (size_t)(nv + 1),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(super_off, out.super_off.data(), sizeof(uint32_t) * (size_t)(nv + 1),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(cnt, 0, sizeof(uint32_t) * (size_t)nv);
  if (e == cudaSuccess) e = cudaMemset(flags, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess && n > 0) k_pack_place<<<blocks_of(n, 256), 256>>>(rec, n, row_off, cnt, placed);
  int dev = 0, sms = 1;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t sort_smem_bytes = (size_t)kSortWarps * kSortCap * (sizeof(uint64_t) + sizeof(uint16_t));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_pack_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sort_smem_bytes);
  if (e == cudaSuccess)
    k_pack_sort<<<(unsigned)std::max(1, sms), kSortWarps * 32, sort_smem_bytes>>>(
        placed, row_off, nv, sorted, (unsigned int *)flags);
  pk::Frame fr;
  for (int d = 0; d < 3; ++d) {
    fr.lo[d] = qlo[d];
    fr.inv[d] = qinv[d];
  }
  q_frame_derive(fr.lo, fr.inv, fr.step, fr.base);
  if (e == cudaSuccess)
    k_pack_encode<<<blocks_of(nv, 128), 128>>>(sorted, row_off, chunk_off, super_off, nv, fr,
                                               chunks, entries, supers, flags + 1);
  if (e == cudaSuccess) e = cudaGetLastError();
  unsigned long long h_flags[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h_flags, flags, sizeof(h_flags), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess || (h_flags[0] & 1ull)) return done(false);  // a row too long to sort
  const double t1 = ms();
  out.entries.resize(4 * (size_t)total);
  out.chunks.resize(4 * (size_t)nch);
  out.supers.resize(4 * (size_t)nsu);
  if (e == cudaSuccess && total)
    e = cudaMemcpy(out.entries.data(), entries, 4 * sizeof(uint32_t) * (size_t)total,
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && nch)
    e = cudaMemcpy(out.chunks.data(), chunks, 4 * sizeof(uint32_t) * (size_t)nch,
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && nsu)
    e = cudaMemcpy(out.supers.data(), supers, 4 * sizeof(uint32_t) * (size_t)nsu,
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return done(false);
  bad_boxes = (int64_t)h_flags[1];
  if (trace)
    std::fprintf(stderr, "p2m build:   device packing: %.0f ms on the device, download %.0f ms "
                 "(%lld entries)\n", t1 - t0, ms() - t1, (long long)total);
  return done(true);
}

}  // namespace p2m
