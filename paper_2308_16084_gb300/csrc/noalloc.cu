// noalloc.cu -- p2m_query_noalloc: the query of p2m_query with its sort
// scratch in a fixed static device array instead of the handle's arena.
//
// Who needs it: code that must not call cudaMalloc while it runs.  Examples
// are hosts whose device memory is owned entirely by another allocator (a
// framework's caching pool that has reserved the GPU), real-time loops that
// cannot afford the device-wide synchronisation cudaMalloc/cudaFree imply,
// and plugins whose host forbids allocations after start-up.  Such callers
// pass their inputs and outputs as usual; the scratch comes from the array
// below, which every GPU that loads this library holds until the process
// exits (kNoallocBytes, about 24.5 MB).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/p2m.h"
#include "kernels.h"

namespace p2m {
bool handle_view(const p2m_handle *h, DevView *v, QueryTuning *t);
}

namespace {

constexpr int64_t kNoallocMaxQueries = (int64_t)1 << 20;
constexpr int kNoallocSortBits = 16;
// layout of launch_query's scratch for kNoallocMaxQueries points and
// 2^kNoallocSortBits buckets: sorted float4 + (bucket, rank) pairs +
// histogram + offsets + 4096 scan-tile sums, each 256-byte aligned, plus the
// alignment slack
constexpr size_t kNoallocBytes = (size_t)16 * kNoallocMaxQueries + (size_t)8 * kNoallocMaxQueries +
                                 2 * ((size_t)4 << kNoallocSortBits) + (size_t)4 * 4096 + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device, looked up once
// per device (with that device current).
p2m_status scratch_address(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return P2M_ERR_NO_DEVICE;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return P2M_ERR_CUDA;
    }
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return P2M_OK;
}

}  // namespace

extern "C" p2m_status p2m_query_noalloc(p2m_handle *h, const float *q, int64_t n, float *dist,
                                        float *closest, int32_t *prim_id, uint8_t *prim_type,
                                        void *stream) {
  p2m::DevView view;
  p2m::QueryTuning tune;
  if (!h) return P2M_ERR_INVALID_ARG;
  if (!p2m::handle_view(h, &view, &tune)) return P2M_ERR_NO_DEVICE;
  if (n < 0) return P2M_ERR_INVALID_ARG;
  if (n > kNoallocMaxQueries) return P2M_ERR_TOO_LARGE;
  if (n == 0) return P2M_OK;
  if (!q || !dist || !prim_id) return P2M_ERR_INVALID_ARG;
  if (tune.sort_bits > kNoallocSortBits) tune.sort_bits = kNoallocSortBits;
  tune.group_by_vertex = 0;  // the static array holds the one-pass scratch only
  if (p2m::query_scratch_bytes(n, tune.sort_bits) > kNoallocBytes) return P2M_ERR_TOO_LARGE;
  void *scratch = nullptr;
  p2m_status s = scratch_address(&scratch);
  if (s) return s;
  // launch_query clears the histogram it counts into on every call, so the
  // previous call's contents of the shared array never leak into this one
  cudaError_t e = p2m::launch_query(view, q, n, dist, closest, prim_id, prim_type, nullptr,
                                    nullptr, scratch, kNoallocBytes, tune, (cudaStream_t)stream);
  if (e == cudaSuccess) return P2M_OK;
  return e == cudaErrorMemoryAllocation ? P2M_ERR_OOM : P2M_ERR_CUDA;
}
