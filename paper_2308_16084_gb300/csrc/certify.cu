// certify.cu -- builder support on the device: the exact certification
// search of the Voronoi cells (Alg. A.1's cells, clipped to D), decided in
// double precision.  Kept apart from the query kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "certify.h"
#include "within_core.h"

namespace p2m {
namespace {

// twelve resident 128-thread blocks per SM: caps the search at 40 registers
// (75 % occupancy instead of 56 % at 52); the builder's certification
// searches of the 1.3M-triangle mesh took 3.42 s against 3.58 s (32
// registers, with spills: 3.96 s)
#ifndef P2M_WITHIN_MIN_BLOCKS
#define P2M_WITHIN_MIN_BLOCKS 12
#endif

__global__ void __launch_bounds__(128, P2M_WITHIN_MIN_BLOCKS) k_nearest_within(DevView m, const double *__restrict__ x,
                                 const double *__restrict__ r2, int64_t n, double s,
                                 int64_t *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = wc::nearest_within(m, x[3 * i], x[3 * i + 1], x[3 * i + 2], r2[i], s);
}

inline unsigned cert_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_nearest_within_f64(const DevView &m, const double *x, const double *r2,
                                      int64_t n, int64_t *out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const double s = wc::within_scale(m);
  k_nearest_within<<<cert_blocks(n, 128), 128, 0, stream>>>(m, x, r2, n, s, out);
  return cudaGetLastError();
}

}  // namespace p2m
