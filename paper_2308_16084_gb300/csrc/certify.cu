// certify.cu -- builder support on the device: the exact certification
// search of the Voronoi cells (Alg. A.1's cells, clipped to D), in double
// precision.  Kept apart from the query kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "certify.h"

namespace p2m {
namespace {

// first KD-tree position of leaf j (leaves split the positions evenly)
__device__ __forceinline__ int64_t cert_leaf_first(const DevView &m, int64_t j) {
  return (j * m.nv) >> m.depth;
}

// Certification search of the builder, in double precision: the nearest
// KD-tree position strictly closer to x than sqrt(r2), or -1; -2 when the
// traversal stack would overflow (the host then searches itself).  Same
// traversal order, pruning and rounded operations (no fused multiply-add) as
// the host search, so the answer is the host's, bit for bit.
__device__ __forceinline__ double box_d2_f64(double qx, double qy, double qz, float lx, float ly,
                                             float lz, float hx, float hy, float hz) {
  const double dx = qx < lx ? __dsub_rn(lx, qx) : (qx > hx ? __dsub_rn(qx, hx) : 0.0);
  const double dy = qy < ly ? __dsub_rn(ly, qy) : (qy > hy ? __dsub_rn(qy, hy) : 0.0);
  const double dz = qz < lz ? __dsub_rn(lz, qz) : (qz > hz ? __dsub_rn(qz, hz) : 0.0);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

constexpr int kWithinStack = 64;

__global__ void k_nearest_within_f64(DevView m, const double *__restrict__ x,
                                     const double *__restrict__ r2, int64_t n,
                                     int64_t *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double qx = x[3 * i], qy = x[3 * i + 1], qz = x[3 * i + 2];
  int node_st[kWithinStack];
  double d2_st[kWithinStack];
  int sp = 0;
  int64_t best = -1;
  double bd = r2[i];
  // the root's own box: every point lies in the union of its children
  node_st[sp] = 0;
  d2_st[sp++] = 0.0;
  const int64_t nleaf0 = m.L - 1;
  while (sp) {
    --sp;
    const int node = node_st[sp];
    const double nd = d2_st[sp];
    if (!(nd < bd)) continue;
    if (node >= nleaf0) {
      const int64_t j = node - nleaf0;
      for (int64_t p = cert_leaf_first(m, j), e = cert_leaf_first(m, j + 1); p < e; ++p) {
        const float4 c = __ldg(&m.kd_points[p]);
        const double dx = __dsub_rn((double)c.x, qx), dy = __dsub_rn((double)c.y, qy),
                     dz = __dsub_rn((double)c.z, qz);
        const double d =
            __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (d < bd) {
          bd = d;
          best = p;
        }
      }
      continue;
    }
    const float4 A = __ldg(&m.kd_nodes[3 * node + 0]);
    const float4 B = __ldg(&m.kd_nodes[3 * node + 1]);
    const float4 C = __ldg(&m.kd_nodes[3 * node + 2]);
    int c0 = 2 * node + 1, c1 = c0 + 1;
    double d0 = box_d2_f64(qx, qy, qz, A.x, A.y, A.z, A.w, B.x, B.y);
    double d1 = box_d2_f64(qx, qy, qz, B.z, B.w, C.x, C.y, C.z, C.w);
    if (d0 > d1) {
      const int tc = c0;
      c0 = c1;
      c1 = tc;
      const double td = d0;
      d0 = d1;
      d1 = td;
    }
    if (sp + 2 > kWithinStack) {
      out[i] = -2;
      return;
    }
    if (d1 < bd) {
      node_st[sp] = c1;
      d2_st[sp++] = d1;
    }
    if (d0 < bd) {
      node_st[sp] = c0;
      d2_st[sp++] = d0;
    }
  }
  out[i] = best;
}

inline unsigned cert_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_nearest_within_f64(const DevView &m, const double *x, const double *r2,
                                      int64_t n, int64_t *out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_nearest_within_f64<<<cert_blocks(n, 128), 128, 0, stream>>>(m, x, r2, n, out);
  return cudaGetLastError();
}

}  // namespace p2m
