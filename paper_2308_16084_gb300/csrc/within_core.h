// within_core.h -- the builder's exact certification search on the device:
// the nearest KD-tree position strictly closer to x than sqrt(r2), decided
// in double precision.  Shared by the batched search (certify.cu) and the
// per-cell Voronoi kernel (cells.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace p2m {
namespace wc {

// first KD-tree position of leaf j (leaves split the positions evenly)
__device__ __forceinline__ int64_t leaf_first(const DevView &m, int64_t j) {
  return (j * m.nv) >> m.depth;
}

// The pruning bound for a double bound bd: float32 distances are compared
// against a bound enlarged past their rounding error.  With e = 2^-23 s the
// float32 error of a coordinate difference (s >= every coordinate
// magnitude), a float32 squared distance differs from the exact one by at
// most 2 sqrt(3) e sqrt(d) + 3 e^2 + 2^-21 d, well inside the margin
// 1e-5 (d + s sqrt(d)) + 1e-9 s^2.
__device__ __forceinline__ float bound_of(double bd, double s) {
  return (float)(bd * (1.0 + 1e-5) + 1e-5 * s * sqrt(bd) + 1e-9 * s * s);
}

__device__ __forceinline__ float box_d2_f32(float qx, float qy, float qz, float lx, float ly,
                                            float lz, float hx, float hy, float hz) {
  const float dx = qx < lx ? lx - qx : (qx > hx ? qx - hx : 0.f);
  const float dy = qy < ly ? ly - qy : (qy > hy ? qy - hy : 0.f);
  const float dz = qz < lz ? lz - qz : (qz > hz ? qz - hz : 0.f);
  return dx * dx + dy * dy + dz * dz;
}

constexpr int kWithinStack = 64;

// s: at least every coordinate magnitude of the points and of the domain
__host__ __device__ inline double within_scale(const DevView &m) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double a = fabs((double)m.dom_lo[d]), b = fabs((double)m.dom_hi[d]);
    s = fmax(s, fmax(a, b));
  }
  return 2.0 * s + 1e-30;
}

// The nearest KD-tree position strictly closer to (qx, qy, qz) than
// sqrt(r2), the lowest among positions at the same double distance, or -1;
// -2 when the traversal stack would overflow (the caller searches another
// way).  The answer is fixed by the point set, so the traversal may differ
// from the host's: it prunes with float32 distances against bound_of, and
// decides every candidate with the double distance computed as the host
// does (each operation rounded on its own).
__device__ __forceinline__ int64_t nearest_within(const DevView &m, double qx, double qy,
                                                  double qz, double r2, double s) {
  const float fx = (float)qx, fy = (float)qy, fz = (float)qz;
  int node_st[kWithinStack];
  float d2_st[kWithinStack];
  int sp = 0;
  int64_t best = -1;
  double bd = r2;
  if (!(bd > 0.0)) return -1;  // no squared distance is below a bound <= 0
  float bf = bound_of(bd, s);
  node_st[sp] = 0;  // the root: every point lies in the union of its children
  d2_st[sp++] = 0.f;
  const int64_t nleaf0 = m.L - 1;
  while (sp) {
    --sp;
    const int node = node_st[sp];
    if (d2_st[sp] > bf) continue;
    if (node >= nleaf0) {
      const int64_t j = node - nleaf0;
      for (int64_t p = leaf_first(m, j), e = leaf_first(m, j + 1); p < e; ++p) {
        const float4 c = __ldg(&m.kd_points[p]);
        const float ex = c.x - fx, ey = c.y - fy, ez = c.z - fz;
        if (ex * ex + ey * ey + ez * ez > bf) continue;
        const double dx = __dsub_rn((double)c.x, qx), dy = __dsub_rn((double)c.y, qy),
                     dz = __dsub_rn((double)c.z, qz);
        const double d =
            __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (d < bd || (best >= 0 && d == bd && p < best)) {
          bd = d;
          best = p;
          bf = bound_of(bd, s);
        }
      }
      continue;
    }
    const float4 A = __ldg(&m.kd_nodes[3 * node + 0]);
    const float4 B = __ldg(&m.kd_nodes[3 * node + 1]);
    const float4 C = __ldg(&m.kd_nodes[3 * node + 2]);
    int c0 = 2 * node + 1, c1 = c0 + 1;
    float d0 = box_d2_f32(fx, fy, fz, A.x, A.y, A.z, A.w, B.x, B.y);
    float d1 = box_d2_f32(fx, fy, fz, B.z, B.w, C.x, C.y, C.z, C.w);
    if (d0 > d1) {
      const int tc = c0;
      c0 = c1;
      c1 = tc;
      const float td = d0;
      d0 = d1;
      d1 = td;
    }
    if (sp + 2 > kWithinStack) return -2;
    if (d1 <= bf) {
      node_st[sp] = c1;
      d2_st[sp++] = d1;
    }
    if (d0 <= bf) {
      node_st[sp] = c0;
      d2_st[sp++] = d0;
    }
  }
  return best;
}

}  // namespace wc
}  // namespace p2m
