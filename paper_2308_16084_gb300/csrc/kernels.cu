// kernels.cu -- sm_103a kernels of the P2M query stage.
//
//   a1  Morton bucket sort of the queries (count with warp-aggregated
//       atomics, exclusive scan, scatter into a float4 stream)
//   a2  nearest vertex: KD tree with the child boxes stored in the parent,
//       nearer child first, far child on a short stack, pruning by box
//       distance; candidate comparisons use the bisector form
//       2 (q-b).(c-b) > |c-b|^2, whose rounding error does not grow with
//       |q-b|^2 / |c-b| the way comparing two squared distances does
//   a3  CSR interception list of that vertex
//   a4  Region-box filter of every entry (Sec. 4.6)
//   a5  d_min = d(q, v) (Alg. A.2)
//   a6  edge: slab test, then the distance to its line
//   a7  face: prism test, then the distance to its plane
//   a8  minimum, written to the caller's order
//   a9  backward scatter
//   a10 batched persistent variant over many meshes
//
// None of this is a dense contraction: the kernels run on the CUDA cores
// and are bound by dependent loads (tree nodes, list entries, records).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "kernels.h"
#include "quant.h"

namespace p2m {
namespace {

constexpr float kPruneSlack = 1.0f + 1.0f / (1 << 20);

// compile-time variants of the query kernel (defaults are the tuned ones)
#ifndef P2M_WALK_BATCH
#define P2M_WALK_BATCH 0
#endif
// resident 512-thread CTAs per SM the query kernel is compiled for (caps
// its registers); 1 leaves the register count to the compiler
#ifndef P2M_QUERY_MIN_BLOCKS
#define P2M_QUERY_MIN_BLOCKS 1
#endif

__device__ __forceinline__ float box_d2(float qx, float qy, float qz, float lx, float ly, float lz,
                                        float hx, float hy, float hz) {
  float dx = fmaxf(fmaxf(lx - qx, qx - hx), 0.f);
  float dy = fmaxf(fmaxf(ly - qy, qy - hy), 0.f);
  float dz = fmaxf(fmaxf(lz - qz, qz - hz), 0.f);
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ int64_t leaf_first(const DevView &m, int64_t j) {
  return (j * m.nv) >> m.depth;
}

// Work counters of one query (counting variant only): internal nodes
// visited, points examined, list entries scanned, edges tested, faces tested.
struct Work {
  int nodes, points, entries, edges, faces, chunks;
};

// Nearest vertex of q: returns the KD-tree position (= table row).
template <bool COUNT = false>
__device__ __forceinline__ int nearest_pos(const DevView &m, float qx, float qy, float qz,
                                           Work *wk = nullptr) {
  int best = -1;
  float bx = 0.f, by = 0.f, bz = 0.f, bd2 = FLT_MAX;
  float wx = 0.f, wy = 0.f, wz = 0.f;  // q - best
  int stk[48];
  float sdd[48];
  int sp = 0;
  int node = 0;
  const int64_t nleaf0 = m.L - 1;
  for (;;) {
    if (node >= nleaf0) {
      const int64_t j = node - nleaf0;
      const int64_t p0 = leaf_first(m, j), p1 = leaf_first(m, j + 1);
      if (COUNT) wk->points += (int)(p1 - p0);
      for (int64_t p = p0; p < p1; ++p) {
        const float4 c = __ldg(&m.kd_points[p]);
        bool take;
        if (best < 0) {
          take = true;
        } else {
          const float ux = c.x - bx, uy = c.y - by, uz = c.z - bz;
          const float lhs = 2.f * (wx * ux + wy * uy + wz * uz) - (ux * ux + uy * uy + uz * uz);
          take = lhs > 0.f || (lhs == 0.f && (int)p < best);
        }
        if (take) {
          best = (int)p;
          bx = c.x;
          by = c.y;
          bz = c.z;
          wx = qx - bx;
          wy = qy - by;
          wz = qz - bz;
          bd2 = wx * wx + wy * wy + wz * wz;
        }
      }
    } else {
      if (COUNT) ++wk->nodes;
      const float4 A = __ldg(&m.kd_nodes[3 * node + 0]);
      const float4 B = __ldg(&m.kd_nodes[3 * node + 1]);
      const float4 C = __ldg(&m.kd_nodes[3 * node + 2]);
      float d0 = box_d2(qx, qy, qz, A.x, A.y, A.z, A.w, B.x, B.y);
      float d1 = box_d2(qx, qy, qz, B.z, B.w, C.x, C.y, C.z, C.w);
      int c0 = 2 * node + 1, c1 = c0 + 1;
      if (d1 < d0) {
        const float t = d0; d0 = d1; d1 = t;
        const int u = c0; c0 = c1; c1 = u;
      }
      const float bound = bd2 * kPruneSlack;
      if (d1 <= bound && sp < 48) {
        stk[sp] = c1;
        sdd[sp] = d1;
        ++sp;
      }
      if (d0 <= bound) {
        node = c0;
        continue;
      }
    }
    bool more = false;
    while (sp > 0) {
      --sp;
      if (sdd[sp] <= bd2 * kPruneSlack) {
        node = stk[sp];
        more = true;
        break;
      }
    }
    if (!more) break;
  }
  return best;
}


// Nearest vertex by KD descent + Voronoi walk.  The descent follows the
// child whose box is nearer to q down to one leaf and keeps its nearest
// vertex.  The walk then moves to any Voronoi neighbour nearer to q (the
// nearest of them), until none is: a vertex nearer to q than every Voronoi
// neighbour is the nearest vertex, because the bisectors of its neighbours
// bound its cell.  The neighbour graph holds inside the domain D only, so
// points outside D, and walks that exceed the step cap, use the full
// backtracking search instead.
constexpr int kWalkCap = 256;

__device__ __forceinline__ int grid_cell(const DevView &m, float v, int a) {
  const int G = 1 << m.grid_bits;
  const float u = (v - m.dom_lo[a]) / (m.dom_hi[a] - m.dom_lo[a]);
  return min(G - 1, max(0, (int)(u * (float)G)));
}

template <bool COUNT = false>
__device__ __forceinline__ int nearest_walk(const DevView &m, float qx, float qy, float qz,
                                            Work *wk = nullptr, bool grid = false) {
  const bool inside = qx >= m.dom_lo[0] && qy >= m.dom_lo[1] && qz >= m.dom_lo[2] &&
                      qx <= m.dom_hi[0] && qy <= m.dom_hi[1] && qz <= m.dom_hi[2];
  if (!inside) return nearest_pos<COUNT>(m, qx, qy, qz, wk);
  const int64_t nleaf0 = m.L - 1;
  int node = 0;
  int seed = -1;
  if (grid && m.seed) {
    const int gb = m.grid_bits;
    const size_t cell = ((size_t)grid_cell(m, qz, 2) << (2 * gb)) |
                        ((size_t)grid_cell(m, qy, 1) << gb) | (size_t)grid_cell(m, qx, 0);
    seed = (int)__ldg(&m.seed[cell]);
    node = (int)nleaf0;  // skip the descent
  }
  while (node < nleaf0) {
    if (COUNT) ++wk->nodes;
    const float4 A = __ldg(&m.kd_nodes[3 * node + 0]);
    const float4 B = __ldg(&m.kd_nodes[3 * node + 1]);
    const float4 C = __ldg(&m.kd_nodes[3 * node + 2]);
    const float d0 = box_d2(qx, qy, qz, A.x, A.y, A.z, A.w, B.x, B.y);
    const float d1 = box_d2(qx, qy, qz, B.z, B.w, C.x, C.y, C.z, C.w);
    node = 2 * node + (d1 < d0 ? 2 : 1);
  }
  int best = -1;
  float bx = 0.f, by = 0.f, bz = 0.f, wx = 0.f, wy = 0.f, wz = 0.f;
  // exact ties go to the lower KD-tree row, as in the backtracking search
  auto offer = [&](int p, float4 c) {
    bool take;
    if (best < 0) {
      take = true;
    } else {
      const float ux = c.x - bx, uy = c.y - by, uz = c.z - bz;
      const float lhs = 2.f * (wx * ux + wy * uy + wz * uz) - (ux * ux + uy * uy + uz * uz);
      take = lhs > 0.f || (lhs == 0.f && p < best);
    }
    if (take) {
      best = p;
      bx = c.x;
      by = c.y;
      bz = c.z;
      wx = qx - bx;
      wy = qy - by;
      wz = qz - bz;
    }
  };
  if (seed >= 0) {
    if (COUNT) ++wk->points;
    offer(seed, __ldg(&m.kd_points[seed]));
  } else {
    const int64_t j = node - nleaf0;
    const int64_t p0 = leaf_first(m, j), p1 = leaf_first(m, j + 1);
    if (COUNT) wk->points += (int)(p1 - p0);
    for (int64_t p = p0; p < p1; ++p) offer((int)p, __ldg(&m.kd_points[p]));
  }
  for (int step = 0; step < kWalkCap; ++step) {
    const int cur = best;
    const uint32_t o0 = __ldg(&m.nb_off[cur]), o1 = __ldg(&m.nb_off[cur + 1]);
    if (COUNT) wk->points += (int)(o1 - o0);
    // the neighbour records carry their positions: one load per neighbour
    for (uint32_t k = o0; k < o1; ++k) {
      const float4 c = __ldg(&m.nbp[k]);
      offer(__float_as_int(c.w), c);
    }
    if (best == cur) return best;
  }
  return nearest_pos<COUNT>(m, qx, qy, qz, wk);
}

// mode 0: backtracking, 1: descent + walk, 2: seed grid + walk
template <bool COUNT = false>
__device__ __forceinline__ int find_nearest(const DevView &m, int mode, float qx, float qy,
                                            float qz, Work *wk = nullptr) {
  return mode ? nearest_walk<COUNT>(m, qx, qy, qz, wk, mode == 2)
              : nearest_pos<COUNT>(m, qx, qy, qz, wk);
}

// ------------------------------------------------------------------ a1
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ff;
  v = (v | (v << 16)) & 0x030000FF;
  v = (v | (v << 8)) & 0x0300F00F;
  v = (v | (v << 4)) & 0x030C30C3;
  v = (v | (v << 2)) & 0x09249249;
  return v;
}

__device__ __forceinline__ uint32_t morton_bucket(float x, float y, float z, const float *lo,
                                                  const float *inv, int shift) {
  float u = fminf(fmaxf((x - lo[0]) * inv[0], 0.f), 0.99999994f);
  float v = fminf(fmaxf((y - lo[1]) * inv[1], 0.f), 0.99999994f);
  float w = fminf(fmaxf((z - lo[2]) * inv[2], 0.f), 0.99999994f);
  if (!(u == u)) u = 0.f;
  if (!(v == v)) v = 0.f;
  if (!(w == w)) w = 0.f;
  uint32_t code = spread10((uint32_t)(u * 1024.f)) | (spread10((uint32_t)(v * 1024.f)) << 1) |
                  (spread10((uint32_t)(w * 1024.f)) << 2);
  return code >> shift;
}

struct SortParams {
  float lo[3];
  float inv[3];
  int shift;
};

// Counting-sort passes over kSortItems queries per thread (item k of a
// block at base + k * blockDim.x, coalesced per item): every thread issues
// all of its atomics (count) or gathers (scatter) before it waits on the
// first, which keeps several in flight per thread.
constexpr int kSortItems = 4;

// sort keys: the Morton bucket of the query, or the seed-grid vertex of its
// cell (nv for a query outside D or not finite): sorted by the latter, the
// lanes of a warp start their Voronoi walks at the same vertex
struct MortonKey {
  SortParams sp;
  __device__ __forceinline__ uint32_t operator()(float x, float y, float z) const {
    return morton_bucket(x, y, z, sp.lo, sp.inv, sp.shift);
  }
};

struct SeedKey {
  DevView m;
  __device__ __forceinline__ int cell(float v, int a) const {
    const int G = 1 << m.sort_grid_bits;
    const float u = (v - m.dom_lo[a]) / (m.dom_hi[a] - m.dom_lo[a]);
    return min(G - 1, max(0, (int)(u * (float)G)));
  }
  __device__ __forceinline__ uint32_t operator()(float x, float y, float z) const {
    const bool in = x >= m.dom_lo[0] && y >= m.dom_lo[1] && z >= m.dom_lo[2] &&
                    x <= m.dom_hi[0] && y <= m.dom_hi[1] && z <= m.dom_hi[2];  // false for NaN
    if (!in) return (uint32_t)m.nv;
    const int gb = m.sort_grid_bits;
    const size_t c = ((size_t)cell(z, 2) << (2 * gb)) | ((size_t)cell(y, 1) << gb) |
                     (size_t)cell(x, 0);
    return __ldg(&m.sort_seed[c]);
  }
};

template <class Key>
__global__ void k_bucket_count(const float *__restrict__ q, int64_t n, Key key,
                               uint32_t *__restrict__ hist, uint2 *__restrict__ key_rank) {
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * kSortItems + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  uint32_t b[kSortItems], got[kSortItems];
  unsigned peers[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t i = base + (int64_t)k * blockDim.x;
    b[k] = i < n ? key(q[3 * i], q[3 * i + 1], q[3 * i + 2])
                 : 0xffffffffu;  // past the end: no bucket has this key
  }
  // warp-aggregated atomics: lanes of one bucket share a single atomicAdd
  // (every lane of the warp stays in the kernel, so the masks are full)
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    peers[k] = __match_any_sync(0xffffffffu, b[k]);
    got[k] = 0;
    if (b[k] != 0xffffffffu && lane == __ffs(peers[k]) - 1)
      got[k] = atomicAdd(&hist[b[k]], (uint32_t)__popc(peers[k]));
  }
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    got[k] = __shfl_sync(0xffffffffu, got[k], __ffs(peers[k]) - 1);
    const int64_t i = base + (int64_t)k * blockDim.x;
    if (i < n) key_rank[i] = make_uint2(b[k], got[k] + __popc(peers[k] & below));
  }
}

// Exclusive scan of hist[0..nb) into off[0..nb) over many CTAs: every CTA
// owns a tile of kScanTile buckets (16 per thread); pass 1 sums tiles, pass
// 2 scans the tile sums in one CTA, pass 3 scans inside every tile and adds
// the tile's offset.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kMaxScanTiles = 4096;  // nb <= 2^24

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < kScanThreads / 32 ? wsum[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) wsum[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1 && total) *total = wi;
  }
  __syncthreads();
  const uint32_t r = inc - v + wsum[wid];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t *__restrict__ hist,
                                                             uint32_t *__restrict__ tile_sum,
                                                             int nb) {
  const int64_t b0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (b0 + k < nb) s += hist[b0 + k];
  __shared__ uint32_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(uint32_t *__restrict__ tile_sum,
                                                                 int ntiles) {
  // exclusive scan in place, one CTA, kScanPer tiles per thread
  const int t0 = threadIdx.x * kScanPer;
  uint32_t v[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = t0 + k < ntiles ? tile_sum[t0 + k] : 0u;
    s += v[k];
  }
  uint32_t run = block_exclusive_scan(s, nullptr);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (t0 + k < ntiles) tile_sum[t0 + k] = run;
    run += v[k];
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *__restrict__ hist,
                                                             const uint32_t *__restrict__ tile_off,
                                                             uint32_t *__restrict__ off, int nb) {
  const int64_t b0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  uint32_t v[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = b0 + k < nb ? hist[b0 + k] : 0u;
    s += v[k];
  }
  uint32_t run = block_exclusive_scan(s, nullptr) + tile_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (b0 + k < nb) off[b0 + k] = run;
    run += v[k];
  }
}

// off = exclusive scan of hist (nb buckets); tiles: kMaxScanTiles u32 scratch
inline void bucket_scan(const uint32_t *hist, uint32_t *off, uint32_t *tiles, int nb,
                        cudaStream_t stream) {
  const int ntiles = (nb + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<ntiles, kScanThreads, 0, stream>>>(hist, tiles, nb);
  k_scan_tile_sums<<<1, kScanThreads, 0, stream>>>(tiles, ntiles);
  k_scan_apply<<<ntiles, kScanThreads, 0, stream>>>(hist, tiles, off, nb);
}

__global__ void k_bucket_scatter(const float *__restrict__ q, int64_t n,
                                 const uint2 *__restrict__ key_rank,
                                 const uint32_t *__restrict__ off, float4 *__restrict__ sorted) {
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * kSortItems + threadIdx.x;
  uint2 kr[kSortItems];
  uint32_t pos[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t i = base + (int64_t)k * blockDim.x;
    kr[k] = i < n ? key_rank[i] : make_uint2(0u, 0u);
  }
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t i = base + (int64_t)k * blockDim.x;
    pos[k] = i < n ? off[kr[k].x] + kr[k].y : 0u;
  }
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t i = base + (int64_t)k * blockDim.x;
    if (i < n)
      sorted[pos[k]] = make_float4(q[3 * i], q[3 * i + 1], q[3 * i + 2], __int_as_float((int)i));
  }
}

__global__ void k_identity(const float *__restrict__ q, int64_t n, float4 *__restrict__ sorted) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  sorted[i] = make_float4(q[3 * i], q[3 * i + 1], q[3 * i + 2], __int_as_float((int)i));
}

// ------------------------------------------------------------ a2..a8
// The running best of a query's scan keeps the squared distance and the
// typed id only (fewer live registers in the latency-bound list scan); the
// winner's closest point and barycentric weights are evaluated once at the
// end (closest_of) with the same arithmetic that tested it.
struct Best {
  float d2;
  uint32_t tid;  // type << 30 | id
};

struct Closest {
  float cx, cy, cz;
  float w1, w2;  // weights of the primitive's 2nd and 3rd vertex; w0 = (1 - w1) - w2
};

// foot of q on the line of edge record {a, 1/|d|^2}, {d = b - a}: returns
// its parameter t (closest point a + t d)
__device__ __forceinline__ float edge_foot(const float4 &a, const float4 &d, float qx, float qy,
                                           float qz, float &cx, float &cy, float &cz) {
  const float wx = qx - a.x, wy = qy - a.y, wz = qz - a.z;
  const float t = (wx * d.x + wy * d.y + wz * d.z) * a.w;
  cx = a.x + t * d.x;
  cy = a.y + t * d.y;
  cz = a.z + t * d.z;
  return t;
}

// foot of q on the plane of face record {a, A}, {e1, B}, {e2, C}: its
// parameters (s, t) (closest point a + s e1 + t e2)
__device__ __forceinline__ void face_foot(const float4 &a, const float4 &e1, const float4 &e2,
                                          float qx, float qy, float qz, float &s, float &t,
                                          float &cx, float &cy, float &cz) {
  const float wx = qx - a.x, wy = qy - a.y, wz = qz - a.z;
  const float p1 = wx * e1.x + wy * e1.y + wz * e1.z;
  const float p2 = wx * e2.x + wy * e2.y + wz * e2.z;
  s = a.w * p1 - e1.w * p2;
  t = e2.w * p2 - e1.w * p1;
  cx = a.x + s * e1.x + t * e2.x;
  cy = a.y + s * e1.y + t * e2.y;
  cz = a.z + s * e1.z + t * e2.z;
}

// the running best of a query whose nearest vertex is row v: that vertex
__device__ __forceinline__ Best best_of_vertex(const DevView &m, float qx, float qy, float qz,
                                               int v) {
  const float4 pv = __ldg(&m.kd_points[v]);
  const float dx = qx - pv.x, dy = qy - pv.y, dz = qz - pv.z;
  Best r;
  r.d2 = dx * dx + dy * dy + dz * dz;
  r.tid = (uint32_t)__float_as_int(pv.w);
  return r;
}

// closest point and weights of the winner tid of a query whose nearest
// vertex is row v (the only vertex the scan can end on: lists hold edges
// and faces)
__device__ __forceinline__ Closest closest_of(const DevView &m, float qx, float qy, float qz,
                                              uint32_t tid, int v) {
  Closest c;
  const uint32_t type = tid >> 30;
  const size_t id = tid & 0x3fffffffu;
  if (type == 0u) {
    const float4 pv = __ldg(&m.kd_points[v]);
    c.cx = pv.x;
    c.cy = pv.y;
    c.cz = pv.z;
    c.w1 = 0.f;
    c.w2 = 0.f;
  } else if (type == 1u) {
    const float4 a = __ldg(&m.edge_rec[2 * id]);
    const float4 d = __ldg(&m.edge_rec[2 * id + 1]);
    c.w1 = edge_foot(a, d, qx, qy, qz, c.cx, c.cy, c.cz);
    c.w2 = 0.f;
  } else {
    const float4 a = __ldg(&m.face_rec[3 * id]);
    const float4 e1 = __ldg(&m.face_rec[3 * id + 1]);
    const float4 e2 = __ldg(&m.face_rec[3 * id + 2]);
    face_foot(a, e1, e2, qx, qy, qz, c.w1, c.w2, c.cx, c.cy, c.cz);
  }
  return c;
}

// a4 + a6/a7 for list entry j: Region-box test (the query's codes qw in its
// chunk's entry frame against the entry's codes, quant.h), then the gated
// distance.  Exact ties keep the lower typed id (vertex < edge < face, then
// lower id), so the result does not depend on the order of the list.
template <bool COUNT>
__device__ __forceinline__ void test_entry(const DevView &m, float qx, float qy, float qz,
                                           uint32_t j, const uint32_t *qw, Best &r, Work *wk) {
  const uint4 e = __ldg(&m.entries[j]);
  if (!q_pass(qw, e.y, e.z, e.w)) return;
  const uint32_t tid = e.x;
  const size_t id = tid & 0x3fffffffu;
  float cx, cy, cz;
  if ((tid >> 30) == 1u) {
    if (COUNT) ++wk->edges;
    const float4 a = __ldg(&m.edge_rec[2 * id]);
    const float4 d = __ldg(&m.edge_rec[2 * id + 1]);
    const float t = edge_foot(a, d, qx, qy, qz, cx, cy, cz);
    if (!(t > 0.f && t < 1.f)) return;
  } else {
    if (COUNT) ++wk->faces;
    const float4 a = __ldg(&m.face_rec[3 * id]);
    const float4 e1 = __ldg(&m.face_rec[3 * id + 1]);
    const float4 e2 = __ldg(&m.face_rec[3 * id + 2]);
    float u, t;
    face_foot(a, e1, e2, qx, qy, qz, u, t, cx, cy, cz);
    if (!(u > 0.f && t > 0.f && u + t < 1.f)) return;
  }
  const float ex = qx - cx, ey = qy - cy, ez = qz - cz;
  const float d2 = ex * ex + ey * ey + ez * ez;
  if (d2 < r.d2 || (d2 == r.d2 && tid < r.tid)) {
    r.d2 = d2;
    r.tid = tid;
  }
}

// entries of chunk c (entries first .. last-1) once its codes admit the
// query (gw: the query's words in the frame of the chunk boxes)
template <bool COUNT>
__device__ __forceinline__ void scan_chunk(const DevView &m, float qx, float qy, float qz,
                                           uint32_t c, uint32_t first, uint32_t last, bool test,
                                           const uint32_t *gw, Best &r, Work *wk) {
  const uint4 cw = __ldg(&m.chunks[c]);
  if (test && !q_pass(gw, cw.x, cw.y, cw.z)) return;
  // the chunk's entry frame: origin from its lower codes, scale inv * 2^e
  float clo[3], cinv[3];
  clo[0] = q_chunk_lo(cw.x & 0xffffu, m.qstep[0], m.qbase[0]);
  clo[1] = q_chunk_lo(cw.x >> 16, m.qstep[1], m.qbase[1]);
  clo[2] = q_chunk_lo(cw.y & 0xffffu, m.qstep[2], m.qbase[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) cinv[d] = q_chunk_inv(m.qinv[d], cw.w, d);
  uint32_t ew[3];
  q_query_words(qx, qy, qz, clo, cinv, ew);
  if (COUNT) wk->entries += (int)(last - first);
  for (uint32_t j = first; j < last; ++j) test_entry<COUNT>(m, qx, qy, qz, j, ew, r, wk);
}

// a3..a8 for a query whose nearest vertex is row v (r already holds v): the
// list as a two-level R-tree (Sec. 4.6).  mode 2: super-chunk boxes, then
// chunk boxes, then entry boxes; mode 1: chunk boxes, then entry boxes;
// mode 0: every entry box.  The three levels test the same query codes
// against nested code boxes (an entry that admits q lies in a chunk and a
// super-chunk that admit q), so every mode finds the same candidates.
// With G lanes per query, lane `sub` takes every G-th super-chunk (mode 2)
// or chunk (modes 0, 1) of the list, starting at its own index.
template <bool COUNT>
__device__ __forceinline__ void scan_list(const DevView &m, float qx, float qy, float qz, int v,
                                          int mode, Best &r, Work *wk, uint32_t sub = 0,
                                          uint32_t G = 1) {
  const uint32_t j0 = __ldg(&m.row_off[v]), j1 = __ldg(&m.row_off[v + 1]);
  const uint32_t c0 = __ldg(&m.chunk_off[v]), c1 = __ldg(&m.chunk_off[v + 1]);
  uint32_t gw[3];
  q_query_words(qx, qy, qz, m.qlo, m.qinv, gw);
  if (mode == 2 && m.supers) {
    const uint32_t s0 = __ldg(&m.super_off[v]), s1 = __ldg(&m.super_off[v + 1]);
    for (uint32_t s = s0 + sub; s < s1; s += G) {
      if (COUNT) ++wk->chunks;
      const uint4 sw = __ldg(&m.supers[s]);
      if (!q_pass(gw, sw.x, sw.y, sw.z)) continue;
      const uint32_t cb = c0 + 8 * (s - s0), ce = min(cb + 8u, c1);
      if (COUNT) wk->chunks += (int)(ce - cb);
      // the boxes of the super-chunk's chunks are all tested first, their
      // loads in flight together, then the admitted chunks are scanned (one
      // chunk box tested and scanned at a time left the list pass 5 % slower
      // on the 1.3M-triangle workload; the order does not change the result)
      uint32_t cpass = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t c = cb + k;
        if (c < ce) {
          const uint4 cw = __ldg(&m.chunks[c]);
          if (q_pass(gw, cw.x, cw.y, cw.z)) cpass |= 1u << k;
        }
      }
      while (cpass) {
        const uint32_t c = cb + (uint32_t)(__ffs(cpass) - 1);
        cpass &= cpass - 1;
        const uint32_t first = j0 + 8 * (c - c0);
        scan_chunk<COUNT>(m, qx, qy, qz, c, first, min(first + 8u, j1), false, gw, r, wk);
      }
    }
    return;
  }
  if (COUNT && mode == 1) wk->chunks += (int)(c1 - c0);
  for (uint32_t c = c0 + sub; c < c1; c += G) {
    const uint32_t first = j0 + 8 * (c - c0);
    scan_chunk<COUNT>(m, qx, qy, qz, c, first, min(first + 8u, j1), mode != 0, gw, r, wk);
  }
}

// The G lanes of one query (G a power of two, adjacent lanes of a warp)
// each hold the best of their slice of the list; the query's best is the
// minimum of (d^2, typed id) over the lanes, the same order test_entry keeps
// (smaller distance, then lower typed id), so the result does not depend on
// G.  Returns true in the one lane whose own best is the query's (the
// lowest such lane), which writes the record.
template <int G>
__device__ __forceinline__ bool group_best(const Best &r) {
  if (G == 1) return true;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
  const unsigned long long key = ((unsigned long long)__float_as_uint(r.d2) << 32) | r.tid;
  unsigned long long best = key;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(gmask, best, o, G);
    best = other < best ? other : best;
  }
  const unsigned hold = __ballot_sync(gmask, key == best) & gmask;
  return (int)lane == __ffs(hold) - 1;
}

// a2..a8 for one query; returns its nearest vertex row (for closest_of)
template <bool COUNT = false>
__device__ __forceinline__ int query_one(const DevView &m, float qx, float qy, float qz, Best &r,
                                         Work *wk = nullptr, int walk = 2, int chunked = 2) {
  const int v = find_nearest<COUNT>(m, walk, qx, qy, qz, wk);
  r = best_of_vertex(m, qx, qy, qz, v);
  scan_list<COUNT>(m, qx, qy, qz, v, chunked, r, wk);
  return v;
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
  return isfinite(x) && isfinite(y) && isfinite(z);
}

// the outputs of query o (the winner r of a query at (qx, qy, qz) whose
// nearest vertex is row v); w0 is saved as (1 - w1) - w2, as k_unpack does
__device__ __forceinline__ void store_result(int64_t o, const DevView &m, float qx, float qy,
                                             float qz, int v, const Best &r, bool ok, uint8_t st,
                                             float *dist, float *closest, int32_t *prim_id,
                                             uint8_t *prim_type, float4 *save, uint8_t *status) {
  if (ok) {
    dist[o] = sqrtf(r.d2);
    if (closest || save) {
      const Closest c = closest_of(m, qx, qy, qz, r.tid, v);
      if (closest) {
        closest[3 * o] = c.cx;
        closest[3 * o + 1] = c.cy;
        closest[3 * o + 2] = c.cz;
      }
      if (save) save[o] = make_float4(__uint_as_float(r.tid), (1.f - c.w1) - c.w2, c.w1, c.w2);
    }
    prim_id[o] = (int32_t)(r.tid & 0x3fffffffu);
    if (prim_type) prim_type[o] = (uint8_t)(r.tid >> 30);
  } else {
    const float nan = __int_as_float(0x7fc00000);
    dist[o] = nan;
    if (closest) closest[3 * o] = closest[3 * o + 1] = closest[3 * o + 2] = nan;
    prim_id[o] = -1;
    if (prim_type) prim_type[o] = 0xff;
    if (save) save[o] = make_float4(__uint_as_float(0xffffffffu), 0.f, 0.f, 0.f);
  }
  if (status) status[o] = st;
}

__global__ void __launch_bounds__(512, P2M_QUERY_MIN_BLOCKS)
k_query(DevView m, const float4 *__restrict__ sq, int64_t n, float *dist,
                        float *closest, int32_t *prim_id, uint8_t *prim_type, float4 *save,
                        uint8_t *status, int walk, int chunked) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 s = sq[i];
  const int64_t o = __float_as_int(s.w);
  Best r;
  int v = 0;
  const bool ok = finite3(s.x, s.y, s.z);
  uint8_t st = ok ? 0 : 2;
  if (ok) {
    if (s.x < m.dom_lo[0] || s.y < m.dom_lo[1] || s.z < m.dom_lo[2] || s.x > m.dom_hi[0] ||
        s.y > m.dom_hi[1] || s.z > m.dom_hi[2])
      st |= 1;
    v = query_one(m, s.x, s.y, s.z, r, nullptr, walk, chunked);
  }
  store_result(o, m, s.x, s.y, s.z, v, r, ok, st, dist, closest, prim_id, prim_type, save,
               status);
}


// ------------------------------------------------ a2..a8, warp-cooperative
// One warp answers 32 Morton-adjacent queries together.  The KD-tree walk is
// shared: a node is entered when any lane's pruning bound admits it
// (ballots), so the warp never diverges on the tree; every lane keeps its own
// best vertex and then scans its own list.
constexpr int kWarpStack = 48;
struct WarpSmem {
  int stack[kWarpStack];
};

template <bool COUNT>
__device__ __forceinline__ int warp_nearest(const DevView &m, float qx, float qy, float qz,
                                            bool active, WarpSmem &ws, Work *wk) {
  const unsigned full = 0xffffffffu;
  int best = -1;
  float bx = 0.f, by = 0.f, bz = 0.f, bd2 = FLT_MAX;
  float wx = 0.f, wy = 0.f, wz = 0.f;
  const int64_t nleaf0 = m.L - 1;
  int sp = 0;
  int node = 0;
  for (;;) {
    if (node >= nleaf0) {
      const int64_t j = node - nleaf0;
      const int64_t p0 = leaf_first(m, j), p1 = leaf_first(m, j + 1);
      if (COUNT && active) wk->points += (int)(p1 - p0);
      for (int64_t p = p0; p < p1; ++p) {
        const float4 c = __ldg(&m.kd_points[p]);
        bool take;
        if (best < 0) {
          take = true;
        } else {
          const float ux = c.x - bx, uy = c.y - by, uz = c.z - bz;
          const float lhs = 2.f * (wx * ux + wy * uy + wz * uz) - (ux * ux + uy * uy + uz * uz);
          take = lhs > 0.f || (lhs == 0.f && (int)p < best);
        }
        if (take && active) {
          best = (int)p;
          bx = c.x;
          by = c.y;
          bz = c.z;
          wx = qx - bx;
          wy = qy - by;
          wz = qz - bz;
          bd2 = wx * wx + wy * wy + wz * wz;
        }
      }
    } else {
      if (COUNT && active) ++wk->nodes;
      const float4 A = __ldg(&m.kd_nodes[3 * node + 0]);
      const float4 B = __ldg(&m.kd_nodes[3 * node + 1]);
      const float4 C = __ldg(&m.kd_nodes[3 * node + 2]);
      const float d0 = box_d2(qx, qy, qz, A.x, A.y, A.z, A.w, B.x, B.y);
      const float d1 = box_d2(qx, qy, qz, B.z, B.w, C.x, C.y, C.z, C.w);
      const float bound = bd2 * kPruneSlack;
      const unsigned m0 = __ballot_sync(full, active && d0 <= bound);
      const unsigned m1 = __ballot_sync(full, active && d1 <= bound);
      if (m0 | m1) {
        const int c0 = 2 * node + 1, c1 = c0 + 1;
        if (m0 && m1) {
          // go first where more lanes find the nearer child
          const unsigned pref0 = __ballot_sync(full, active && d0 <= d1);
          const bool first0 = __popc(pref0) * 2 >= __popc(m0 | m1);
          if (sp < kWarpStack) {
            if ((threadIdx.x & 31) == 0) ws.stack[sp] = first0 ? c1 : c0;
            ++sp;
          }
          node = first0 ? c0 : c1;
        } else {
          node = m0 ? c0 : c1;
        }
        __syncwarp();
        continue;
      }
    }
    // pop the next subtree some lane still needs
    bool more = false;
    while (sp > 0) {
      --sp;
      __syncwarp();
      const int c = ws.stack[sp];
      const int par = (c - 1) >> 1;
      const float4 A = __ldg(&m.kd_nodes[3 * par + 0]);
      const float4 B = __ldg(&m.kd_nodes[3 * par + 1]);
      const float4 C = __ldg(&m.kd_nodes[3 * par + 2]);
      const float d = (c & 1) ? box_d2(qx, qy, qz, A.x, A.y, A.z, A.w, B.x, B.y)
                              : box_d2(qx, qy, qz, B.z, B.w, C.x, C.y, C.z, C.w);
      if (__any_sync(full, active && d <= bd2 * kPruneSlack)) {
        node = c;
        more = true;
        break;
      }
    }
    if (!more) break;
  }
  return best;
}

// returns the lane's nearest vertex row (0 for an inactive lane)
template <bool COUNT>
__device__ __forceinline__ int warp_query(const DevView &m, float qx, float qy, float qz,
                                          bool active, WarpSmem &ws, Best &r, Work *wk,
                                          int walk) {
  int v;
  if (walk) {
    v = active ? nearest_walk<COUNT>(m, qx, qy, qz, wk, walk == 2) : 0;
    __syncwarp();
  } else {
    v = warp_nearest<COUNT>(m, qx, qy, qz, active, ws, wk);
  }
  if (active) {
    r = best_of_vertex(m, qx, qy, qz, v);
    scan_list<COUNT>(m, qx, qy, qz, v, 2, r, wk);
  }
  return v;
}

template <bool COUNT>
__global__ void k_query_warp(DevView m, const float4 *__restrict__ sq, int64_t n, float *dist,
                             float *closest, int32_t *prim_id, uint8_t *prim_type, float4 *save,
                             uint8_t *status, unsigned long long *acc, int walk) {
  extern __shared__ WarpSmem smem_w[];
  WarpSmem &ws = smem_w[threadIdx.x >> 5];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // whole warps stay together; lanes past the end take part inactive
  if (((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >= n) return;
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i < n) s = sq[i];
  const bool ok = i < n && finite3(s.x, s.y, s.z);
  Best r;
  Work w = {0, 0, 0, 0, 0, 0};
  const int v = warp_query<COUNT>(m, s.x, s.y, s.z, ok, ws, r, &w, walk);
  if (COUNT) {
    int v[6] = {w.nodes, w.points, w.entries, w.edges, w.faces, w.chunks};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      unsigned long long x = (unsigned long long)v[k];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], x);
    }
    return;
  }
  if (i >= n) return;
  const int64_t o = __float_as_int(s.w);
  uint8_t st = ok ? 0 : 2;
  if (ok && (s.x < m.dom_lo[0] || s.y < m.dom_lo[1] || s.z < m.dom_lo[2] || s.x > m.dom_hi[0] ||
             s.y > m.dom_hi[1] || s.z > m.dom_hi[2]))
    st |= 1;
  store_result(o, m, s.x, s.y, s.z, v, r, ok, st, dist, closest, prim_id, prim_type, save,
               status);
}


// ------------------------------------------- two-pass query, grouped lists
// Pass 1: nearest vertex of every Morton-sorted query (nv marks a
// non-finite query), counted straight into the per-vertex histogram: the
// lanes that found the same vertex add their count with one atomic, and each
// keeps its rank inside that vertex's bucket.  The queries are then
// regrouped by vertex with a counting sort, so that the lanes of a warp
// mostly share one interception list in pass 2 (uniform loops, broadcast
// loads).
__device__ __forceinline__ uint2 count_key(uint32_t b, uint32_t *__restrict__ hist) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, b);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&hist[b], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return make_uint2(b, base + __popc(peers & ((1u << lane) - 1u)));
}

__global__ void k_nn_pass(DevView m, const float4 *__restrict__ sq, int64_t n, int walk,
                          uint32_t *__restrict__ hist, uint2 *__restrict__ key_rank) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 s = sq[i];
  const uint32_t v = finite3(s.x, s.y, s.z) ? (uint32_t)find_nearest(m, walk, s.x, s.y, s.z)
                                            : (uint32_t)m.nv;
  key_rank[i] = count_key(v, hist);
}

__global__ void k_vertex_scatter(const float4 *__restrict__ sq, int64_t n,
                                 const uint2 *__restrict__ key_rank,
                                 const uint32_t *__restrict__ off, float4 *__restrict__ out,
                                 uint32_t *__restrict__ vout) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 kr = key_rank[i];
  const uint32_t pos = off[kr.x] + kr.y;
  out[pos] = sq[i];
  vout[pos] = kr.x;
}

// four resident 512-thread CTAs per SM: caps k_list_pass at 32 registers
// (full occupancy; the running best is (d^2, typed id) only, and the few
// values that spill stay in L1).  On the 1.3M-triangle workload the list
// pass took 1.105 ms against 1.162 ms at 40 registers (three CTAs) after the
// Morton sort, 1.104 against 1.117 ms after the seed-vertex sort; the
// uncapped 56 registers took 1.40 ms
#ifndef P2M_LIST_MIN_BLOCKS
#define P2M_LIST_MIN_BLOCKS 4
#endif

// Pass 2: the list of each query's nearest vertex (regrouped stream).  The
// result goes out as one 32-byte record in the caller's order, rec[2o] =
// (closest xyz, distance), rec[2o+1] = (type << 30 | id, w1, w2, status):
// a whole sector per query, where separate outputs would each dirty part of
// one.  k_unpack then streams the records into the requested outputs.
// G threads per query (1, 2, 4 or 8): the G adjacent lanes of a query split
// its list (scan_list) and keep the best with one shuffle reduction
// (group_best); whole groups enter and leave together.
template <int G>
__global__ void __launch_bounds__(512, P2M_LIST_MIN_BLOCKS)
k_list_pass(DevView m, const float4 *__restrict__ gq, const uint32_t *__restrict__ gv, int64_t n,
            int chunked, float4 *__restrict__ rec) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / G;
  const uint32_t sub = (uint32_t)(t & (G - 1));
  if (i >= n) return;
  const float4 s = gq[i];
  const int64_t o = __float_as_int(s.w);
  const bool ok = finite3(s.x, s.y, s.z);
  uint32_t st = ok ? 0u : 2u;
  if (!ok) {
    if (sub) return;
    const float nan = __int_as_float(0x7fc00000);
    rec[2 * o] = make_float4(nan, nan, nan, nan);
    rec[2 * o + 1] = make_float4(__uint_as_float(0xffffffffu), 0.f, 0.f, __uint_as_float(st));
    return;
  }
  const int v = (int)gv[i];
  if (s.x < m.dom_lo[0] || s.y < m.dom_lo[1] || s.z < m.dom_lo[2] || s.x > m.dom_hi[0] ||
      s.y > m.dom_hi[1] || s.z > m.dom_hi[2])
    st |= 1u;
  Best r = best_of_vertex(m, s.x, s.y, s.z, v);
  scan_list<false>(m, s.x, s.y, s.z, v, chunked, r, nullptr, sub, G);
  if (!group_best<G>(r)) return;
  const Closest c = closest_of(m, s.x, s.y, s.z, r.tid, v);
  rec[2 * o] = make_float4(c.cx, c.cy, c.cz, sqrtf(r.d2));
  rec[2 * o + 1] = make_float4(__uint_as_float(r.tid), c.w1, c.w2, __uint_as_float(st));
}

// Records (caller order) -> the requested outputs, coalesced.  w0 is rebuilt
// as (1 - w1) - w2, the same operations the list pass evaluated it with
// (face: 1 - s - t; edge: 1 - t with w2 = 0; vertex: 1 with w1 = w2 = 0).
__global__ void k_unpack(const float4 *__restrict__ rec, int64_t n, float *dist, float *closest,
                         int32_t *prim_id, uint8_t *prim_type, float4 *save, uint8_t *status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = __ldcs(&rec[2 * i]);
  const float4 b = __ldcs(&rec[2 * i + 1]);
  const uint32_t tid = __float_as_uint(b.x);
  const bool ok = tid != 0xffffffffu;
  dist[i] = a.w;
  if (closest) {
    closest[3 * i] = a.x;
    closest[3 * i + 1] = a.y;
    closest[3 * i + 2] = a.z;
  }
  prim_id[i] = ok ? (int32_t)(tid & 0x3fffffffu) : -1;
  if (prim_type) prim_type[i] = ok ? (uint8_t)(tid >> 30) : (uint8_t)0xff;
  if (save) save[i] = make_float4(b.x, ok ? (1.f - b.y) - b.z : 0.f, b.y, b.z);
  if (status) status[i] = (uint8_t)__float_as_uint(b.w);
}

// Counting variant of the query (not timed): sums the per-query work.
__global__ void k_query_count(DevView m, const float4 *__restrict__ sq, int64_t n,
                              unsigned long long *__restrict__ acc, int walk, int chunked) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Work w = {0, 0, 0, 0, 0, 0};
  if (i < n) {
    const float4 s = sq[i];
    Best r;
    if (finite3(s.x, s.y, s.z)) query_one<true>(m, s.x, s.y, s.z, r, &w, walk, chunked);
  }
  int v[6] = {w.nodes, w.points, w.entries, w.edges, w.faces, w.chunks};
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    unsigned long long x = (unsigned long long)v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], x);
  }
}

__global__ void k_nearest(DevView m, const float *__restrict__ xyz, int64_t n,
                          int32_t *__restrict__ out, int original_ids, int walk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  int p = finite3(x, y, z) ? find_nearest(m, walk, x, y, z) : -1;
  if (original_ids && p >= 0) p = __float_as_int(__ldg(&m.kd_points[p]).w);
  out[i] = p;
}

__global__ void k_seed_grid(DevView m, uint32_t *__restrict__ seed) {
  const int gb = m.grid_bits;
  const int64_t G = (int64_t)1 << gb;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G * G * G) return;
  const int ix = (int)(i & (G - 1)), iy = (int)((i >> gb) & (G - 1)), iz = (int)(i >> (2 * gb));
  const float x = m.dom_lo[0] + (ix + 0.5f) * (m.dom_hi[0] - m.dom_lo[0]) / (float)G;
  const float y = m.dom_lo[1] + (iy + 0.5f) * (m.dom_hi[1] - m.dom_lo[1]) / (float)G;
  const float z = m.dom_lo[2] + (iz + 0.5f) * (m.dom_hi[2] - m.dom_lo[2]) / (float)G;
  seed[i] = (uint32_t)nearest_pos(m, x, y, z);
}

// --------------------------------------------- moved vertices (a9 support)
// p2m_update_vertices: the vertex-dependent records of the layout from new
// positions, with the builder's arithmetic (float differences; double
// products, sums and quotients rounded one by one, as the host builder
// compiled without contraction), so that unchanged positions give unchanged
// records bit for bit.  The interception lists and Region boxes stay those
// of the build.
__global__ void k_update_points(float4 *__restrict__ kd_points, int64_t nv,
                                const float *__restrict__ verts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nv) return;
  float4 c = kd_points[p];
  const int64_t v = __float_as_int(c.w);
  c.x = verts[3 * v];
  c.y = verts[3 * v + 1];
  c.z = verts[3 * v + 2];
  kd_points[p] = c;
}

__global__ void k_update_neighbours(float4 *__restrict__ nbp, const uint32_t *__restrict__ nb,
                                    int64_t count, const float4 *__restrict__ kd_points) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const float4 c = kd_points[nb[k]];
  float4 o = nbp[k];
  o.x = c.x;
  o.y = c.y;
  o.z = c.z;
  nbp[k] = o;
}

__global__ void k_update_edges(float4 *__restrict__ edge_rec, const int2 *__restrict__ edges,
                               int64_t ne, const float *__restrict__ verts) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int2 ab = edges[e];
  const float *a = verts + 3 * (int64_t)ab.x, *b = verts + 3 * (int64_t)ab.y;
  const float dx = __fsub_rn(b[0], a[0]), dy = __fsub_rn(b[1], a[1]), dz = __fsub_rn(b[2], a[2]);
  const double l2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  edge_rec[2 * e] = make_float4(a[0], a[1], a[2], __double2float_rn(__ddiv_rn(1.0, l2)));
  edge_rec[2 * e + 1] = make_float4(dx, dy, dz, 0.f);
}

__global__ void k_update_faces(float4 *__restrict__ face_rec, const int4 *__restrict__ tris,
                               int64_t nf, const float *__restrict__ verts) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int4 t = tris[f];
  const float *a = verts + 3 * (int64_t)t.x, *b = verts + 3 * (int64_t)t.y,
              *c = verts + 3 * (int64_t)t.z;
  double e1[3], e2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    e1[d] = __dsub_rn((double)b[d], (double)a[d]);
    e2[d] = __dsub_rn((double)c[d], (double)a[d]);
  }
  auto dot = [](const double *x, const double *y) {
    return __dadd_rn(__dadd_rn(__dmul_rn(x[0], y[0]), __dmul_rn(x[1], y[1])),
                     __dmul_rn(x[2], y[2]));
  };
  const double d00 = dot(e1, e1), d01 = dot(e1, e2), d11 = dot(e2, e2);
  const double den = __dsub_rn(__dmul_rn(d00, d11), __dmul_rn(d01, d01));
  // a face the build found degenerate keeps its NaN weights (it is in no list)
  const bool degenerate = isnan(face_rec[3 * f].w);
  const float nan = __int_as_float(0x7fc00000);
  face_rec[3 * f] = make_float4(a[0], a[1], a[2],
                                degenerate ? nan : __double2float_rn(__ddiv_rn(d11, den)));
  face_rec[3 * f + 1] = make_float4(__double2float_rn(e1[0]), __double2float_rn(e1[1]),
                                    __double2float_rn(e1[2]),
                                    degenerate ? nan : __double2float_rn(__ddiv_rn(d01, den)));
  face_rec[3 * f + 2] = make_float4(__double2float_rn(e2[0]), __double2float_rn(e2[1]),
                                    __double2float_rn(e2[2]),
                                    degenerate ? nan : __double2float_rn(__ddiv_rn(d00, den)));
}

// child boxes of the internal nodes first .. first + count - 1 (one level
// of the tree), from their children: the points of a leaf, or the two boxes
// an internal child stores (filled by the previous launch)
__global__ void k_update_kd_level(float4 *__restrict__ kd_nodes,
                                  const float4 *__restrict__ kd_points, int64_t nv, int depth,
                                  int64_t first, int64_t count) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t i = first + t;
  const int64_t nleaf0 = ((int64_t)1 << depth) - 1;
  float lo[2][3], hi[2][3];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int64_t c = 2 * i + 1 + k;
    for (int d = 0; d < 3; ++d) {  // an empty leaf keeps the builder's (+inf, -inf)
      lo[k][d] = __int_as_float(0x7f800000);
      hi[k][d] = __int_as_float(0xff800000);
    }
    if (c >= nleaf0) {
      const int64_t j = c - nleaf0;
      const int64_t p0 = (j * nv) >> depth, p1 = ((j + 1) * nv) >> depth;
      for (int64_t p = p0; p < p1; ++p) {
        const float4 q = kd_points[p];
        lo[k][0] = fminf(lo[k][0], q.x);
        lo[k][1] = fminf(lo[k][1], q.y);
        lo[k][2] = fminf(lo[k][2], q.z);
        hi[k][0] = fmaxf(hi[k][0], q.x);
        hi[k][1] = fmaxf(hi[k][1], q.y);
        hi[k][2] = fmaxf(hi[k][2], q.z);
      }
    } else {
      const float4 A = kd_nodes[3 * c], B = kd_nodes[3 * c + 1], C = kd_nodes[3 * c + 2];
      lo[k][0] = fminf(A.x, B.z);
      lo[k][1] = fminf(A.y, B.w);
      lo[k][2] = fminf(A.z, C.x);
      hi[k][0] = fmaxf(A.w, C.y);
      hi[k][1] = fmaxf(B.x, C.z);
      hi[k][2] = fmaxf(B.y, C.w);
    }
  }
  kd_nodes[3 * i] = make_float4(lo[0][0], lo[0][1], lo[0][2], hi[0][0]);
  kd_nodes[3 * i + 1] = make_float4(hi[0][1], hi[0][2], lo[1][0], lo[1][1]);
  kd_nodes[3 * i + 2] = make_float4(lo[1][2], hi[1][0], hi[1][1], hi[1][2]);
}

// ------------------------------------------------------------------ a9
__global__ void k_backward(DevView m, const float *__restrict__ q, const float *__restrict__ dist,
                           const float *__restrict__ closest, const float4 *__restrict__ save,
                           const float *__restrict__ gd, int64_t n, float *grad_q,
                           float *grad_v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float d = dist[i], g = gd[i];
  float ux = 0.f, uy = 0.f, uz = 0.f;
  const bool live = d > 0.f && isfinite(d);
  if (live) {
    const float inv = 1.f / d;
    ux = (q[3 * i] - closest[3 * i]) * inv;
    uy = (q[3 * i + 1] - closest[3 * i + 1]) * inv;
    uz = (q[3 * i + 2] - closest[3 * i + 2]) * inv;
  }
  if (grad_q) {
    grad_q[3 * i] = g * ux;
    grad_q[3 * i + 1] = g * uy;
    grad_q[3 * i + 2] = g * uz;
  }
  if (!grad_v || !live || g == 0.f) return;
  const float4 s = save[i];
  const uint32_t tid = __float_as_uint(s.x);
  const uint32_t typ = tid >> 30, id = tid & 0x3fffffffu;
  int vid[3] = {-1, -1, -1};
  const float w[3] = {s.y, s.z, s.w};
  if (typ == 0) {
    vid[0] = (int)id;
  } else if (typ == 1) {
    const int2 e = __ldg(&m.edges[id]);
    vid[0] = e.x;
    vid[1] = e.y;
  } else if (typ == 2) {
    const int4 t = __ldg(&m.tris[id]);
    vid[0] = t.x;
    vid[1] = t.y;
    vid[2] = t.z;
  } else {
    return;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (vid[k] < 0 || w[k] == 0.f) continue;
    const float c = -g * w[k];
    atomicAdd(&grad_v[3 * (size_t)vid[k]], c * ux);
    atomicAdd(&grad_v[3 * (size_t)vid[k] + 1], c * uy);
    atomicAdd(&grad_v[3 * (size_t)vid[k] + 2], c * uz);
  }
}

// ----------------------------------------------------------------- a10
// The mesh of a global query index: binary search of the query-count
// prefix sums, kept in shared memory.
__device__ __forceinline__ int mesh_of(const int64_t *qoff, int n_meshes, int64_t i) {
  int lo = 0, hi = n_meshes;  // qoff[lo] <= i < qoff[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (qoff[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr int kMaxBatchMeshes = 2048;

__global__ void k_batch_count(BatchDesc d, int64_t total, int bits, uint32_t *__restrict__ hist,
                              uint2 *__restrict__ key_rank) {
  __shared__ int64_t s_off[kMaxBatchMeshes + 1];
  for (int k = threadIdx.x; k <= d.n_meshes; k += blockDim.x) s_off[k] = d.qoff[k];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = mesh_of(s_off, d.n_meshes, i);
  const int64_t l = i - s_off[k];
  const float *q = d.ios[k].q;
  const DevView &m = d.views[k];
  float inv[3];
  for (int a = 0; a < 3; ++a) {
    const float ext = m.dom_hi[a] - m.dom_lo[a];
    inv[a] = ext > 0.f ? 1.f / ext : 0.f;
  }
  const uint32_t b = ((uint32_t)k << bits) |
                     (bits ? morton_bucket(q[3 * l], q[3 * l + 1], q[3 * l + 2], m.dom_lo, inv,
                                           30 - bits)
                           : 0u);
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, b);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&hist[b], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  key_rank[i] = make_uint2(b, base + __popc(peers & ((1u << lane) - 1u)));
}

__global__ void k_batch_scatter(BatchDesc d, int64_t total, const uint2 *__restrict__ key_rank,
                                const uint32_t *__restrict__ off, float4 *__restrict__ sorted) {
  __shared__ int64_t s_off[kMaxBatchMeshes + 1];
  for (int k = threadIdx.x; k <= d.n_meshes; k += blockDim.x) s_off[k] = d.qoff[k];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = mesh_of(s_off, d.n_meshes, i);
  const int64_t l = i - s_off[k];
  const float *q = d.ios[k].q;
  const uint2 kr = key_rank[i];
  sorted[off[kr.x] + kr.y] = make_float4(q[3 * l], q[3 * l + 1], q[3 * l + 2],
                                         __int_as_float((int)i));
}

// Persistent CTAs drain the work queue: item t = sorted queries
// [t*tile, (t+1)*tile).  The queue is one atomic counter, so no CTA ever
// waits for another.
__global__ void k_batch_query(BatchDesc d, const float4 *__restrict__ sorted, int64_t total,
                              int tile, unsigned int *queue_head, unsigned int *error_word) {
  __shared__ int64_t s_off[kMaxBatchMeshes + 1];
  __shared__ unsigned int s_item;
  for (int k = threadIdx.x; k <= d.n_meshes; k += blockDim.x) s_off[k] = d.qoff[k];
  const int64_t n_items = (total + tile - 1) / tile;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(queue_head, 1u);
    __syncthreads();
    const int64_t it = s_item;
    if (it >= n_items) break;
    const int64_t base = it * (int64_t)tile;
    for (int t = threadIdx.x; t < tile; t += blockDim.x) {
      const int64_t pos = base + t;
      if (pos >= total) break;
      const float4 s = sorted[pos];
      const int64_t gi = __float_as_int(s.w);
      if (gi < 0 || gi >= total) {
        atomicOr(error_word, 1u);
        continue;
      }
      const int k = mesh_of(s_off, d.n_meshes, gi);
      const int64_t l = gi - s_off[k];
      const BatchIO &io = d.ios[k];
      Best r;
      int v = 0;
      const bool ok = finite3(s.x, s.y, s.z);
      if (ok) v = query_one(d.views[k], s.x, s.y, s.z, r);
      store_result(l, d.views[k], s.x, s.y, s.z, v, r, ok, 0, io.dist, io.closest, io.prim_id,
                   io.prim_type, nullptr, nullptr);
    }
  }
}

// Two-pass batch, as in the single-mesh path: nearest vertex of every sorted
// query, counted into one histogram over all meshes' vertices (key =
// voff[mesh] + vertex, nv of a mesh marks its non-finite queries); the
// queries are regrouped by that key, the persistent list pass drains tiles
// of the regrouped stream and writes one 32-byte record per query in the
// concatenated caller order, and k_batch_unpack scatters the records into
// each mesh's outputs.
__global__ void k_batch_nn(BatchDesc d, const float4 *__restrict__ sorted, int64_t total,
                           uint32_t *__restrict__ vhist, uint2 *__restrict__ key_rank) {
  __shared__ int64_t s_off[kMaxBatchMeshes + 1];
  for (int k = threadIdx.x; k <= d.n_meshes; k += blockDim.x) s_off[k] = d.qoff[k];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const float4 s = sorted[i];
  const int64_t gi = __float_as_int(s.w);
  const int k = mesh_of(s_off, d.n_meshes, gi);
  const DevView &m = d.views[k];
  const int walk = !m.nb_off ? 0 : (m.seed ? 2 : 1);
  const uint32_t v = finite3(s.x, s.y, s.z) ? (uint32_t)find_nearest(m, walk, s.x, s.y, s.z)
                                            : (uint32_t)m.nv;
  key_rank[i] = count_key((uint32_t)d.voff[k] + v, vhist);
}

// resident 512-thread CTAs per SM the persistent batch list kernel is
// compiled for (its register cap, 40 registers): its mesh descriptor is
// indexed by a run-time mesh number, so its fields take registers that
// k_list_pass reads from its parameters, and a 32-register cap would spill
// more than it does now
#ifndef P2M_BATCH_LIST_MIN_BLOCKS
#define P2M_BATCH_LIST_MIN_BLOCKS 3
#endif

template <int G>
__global__ void __launch_bounds__(512, P2M_BATCH_LIST_MIN_BLOCKS)
k_batch_list(BatchDesc d, const float4 *__restrict__ grouped, const uint32_t *__restrict__ gv,
             int64_t total, int tile, float4 *__restrict__ rec, unsigned int *queue_head,
             unsigned int *error_word) {
  __shared__ int64_t s_off[kMaxBatchMeshes + 1];
  __shared__ unsigned int s_item;
  for (int k = threadIdx.x; k <= d.n_meshes; k += blockDim.x) s_off[k] = d.qoff[k];
  const int64_t n_items = (total + tile - 1) / tile;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(queue_head, 1u);
    __syncthreads();
    const int64_t it = s_item;
    if (it >= n_items) break;
    const int64_t base = it * (int64_t)tile;
    // G adjacent threads per query: the G lanes of a query share its
    // position, so they take every branch below together
    for (int u = threadIdx.x; u < tile * G; u += blockDim.x) {
      const int64_t pos = base + u / G;
      const uint32_t sub = (uint32_t)(u & (G - 1));
      if (pos >= total) break;
      const float4 s = grouped[pos];
      const int64_t gi = __float_as_int(s.w);
      if (gi < 0 || gi >= total) {
        if (!sub) atomicOr(error_word, 1u);
        continue;
      }
      const int k = mesh_of(s_off, d.n_meshes, gi);
      const DevView &m = d.views[k];
      const int64_t v = (int64_t)gv[pos] - d.voff[k];
      const bool ok = finite3(s.x, s.y, s.z);
      if (!ok || v < 0 || v >= m.nv) {
        if (sub) continue;
        if (ok) atomicOr(error_word, 2u);
        const float nan = __int_as_float(0x7fc00000);
        rec[2 * gi] = make_float4(nan, nan, nan, nan);
        rec[2 * gi + 1] = make_float4(__uint_as_float(0xffffffffu), 0.f, 0.f, __uint_as_float(2u));
        continue;
      }
      Best r = best_of_vertex(m, s.x, s.y, s.z, (int)v);
      scan_list<false>(m, s.x, s.y, s.z, (int)v, 2, r, nullptr, sub, G);
      if (!group_best<G>(r)) continue;
      const Closest c = closest_of(m, s.x, s.y, s.z, r.tid, (int)v);
      rec[2 * gi] = make_float4(c.cx, c.cy, c.cz, sqrtf(r.d2));
      rec[2 * gi + 1] = make_float4(__uint_as_float(r.tid), c.w1, c.w2, __uint_as_float(0u));
    }
  }
}

__global__ void k_batch_unpack(BatchDesc d, const float4 *__restrict__ rec, int64_t total) {
  __shared__ int64_t s_off[kMaxBatchMeshes + 1];
  for (int k = threadIdx.x; k <= d.n_meshes; k += blockDim.x) s_off[k] = d.qoff[k];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = mesh_of(s_off, d.n_meshes, i);
  const int64_t l = i - s_off[k];
  const BatchIO &io = d.ios[k];
  const float4 a = __ldcs(&rec[2 * i]);
  const float4 b = __ldcs(&rec[2 * i + 1]);
  const uint32_t tid = __float_as_uint(b.x);
  const bool ok = tid != 0xffffffffu;
  io.dist[l] = a.w;
  if (io.closest) {
    io.closest[3 * l] = a.x;
    io.closest[3 * l + 1] = a.y;
    io.closest[3 * l + 2] = a.z;
  }
  io.prim_id[l] = ok ? (int32_t)(tid & 0x3fffffffu) : -1;
  if (io.prim_type) io.prim_type[l] = ok ? (uint8_t)(tid >> 30) : (uint8_t)0xff;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t query_scratch_bytes(int64_t n, int sort_bits, int64_t nv, int ranges) {
  size_t nb = sort_bits > 0 ? ((size_t)1 << sort_bits) : 0;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t base = al(16 * (size_t)n) + al(8 * (size_t)n) + 2 * al(4 * nb) + al(4 * kMaxScanTiles);
  if (nv > 0)  // regrouping: vertex per query, second float4 stream, 32-byte result
               // records, vertex histogram and offsets
    base += al(4 * (size_t)n) + al(16 * (size_t)n) + al(32 * (size_t)n) +
            2 * al(4 * (size_t)(nv + 1));
  if (nv > 0 && ranges > 1)  // every further range: its histogram, offsets, scan tiles
    base += (size_t)(ranges - 1) * (2 * al(4 * (size_t)(nv + 1)) + al(4 * kMaxScanTiles));
  return base + 256;
}

cudaError_t launch_query(const DevView &m, const float *q, int64_t n, float *dist,
                         float *closest, int32_t *prim_id, uint8_t *prim_type, float4 *save,
                         uint8_t *status, void *scratch, size_t scratch_bytes,
                         const QueryTuning &tune, cudaStream_t stream, cudaEvent_t *ev,
                         unsigned long long *counters, const SplitStreams *split) {
  if (n <= 0) return cudaSuccess;
  if (scratch_bytes < query_scratch_bytes(n, tune.sort_bits)) return cudaErrorInvalidValue;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char *base = (char *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  float4 *sorted = (float4 *)base;
  base += al(16 * (size_t)n);
  uint2 *key_rank = (uint2 *)base;
  base += al(8 * (size_t)n);
  const int T = 256;
  if (ev) cudaEventRecord(ev[0], stream);
  const bool grouped = tune.group_by_vertex && !counters && !tune.warp_mode &&
                       m.nv + 1 <= (int64_t)kScanTile * kMaxScanTiles;
  const size_t nbm = tune.sort_bits > 0 ? ((size_t)1 << tune.sort_bits) : 0;
  // regrouping buffers, after the sort's own scratch
  char *b2 = (char *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255) + al(16 * (size_t)n) +
             al(8 * (size_t)n) + 2 * al(4 * nbm) + al(4 * kMaxScanTiles);
  uint32_t *gv = (uint32_t *)b2;
  b2 += al(4 * (size_t)n);
  float4 *grouped_q = (float4 *)b2;
  b2 += al(16 * (size_t)n);
  float4 *rec = (float4 *)b2;
  b2 += al(32 * (size_t)n);
  uint32_t *vhist = (uint32_t *)b2;
  b2 += al(4 * (size_t)(m.nv + 1));
  uint32_t *voff = (uint32_t *)b2;
  uint32_t *tiles2 = (uint32_t *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255) +
                     (al(16 * (size_t)n) + al(8 * (size_t)n) + 2 * al(4 * nbm)) / 4;
  if (grouped && scratch_bytes < query_scratch_bytes(n, tune.sort_bits, m.nv))
    return cudaErrorInvalidValue;
  if (grouped && tune.sort_key == 1 && m.sort_seed) {
    // counting sort by seed-grid vertex, in the regrouping's vertex buffers
    cudaMemsetAsync(vhist, 0, 4 * (size_t)(m.nv + 1), stream);
    k_bucket_count<SeedKey><<<blocks_for(n, T * kSortItems), T, 0, stream>>>(
        q, n, SeedKey{m}, vhist, key_rank);
    bucket_scan(vhist, voff, tiles2, (int)(m.nv + 1), stream);
    k_bucket_scatter<<<blocks_for(n, T * kSortItems), T, 0, stream>>>(q, n, key_rank, voff,
                                                                      sorted);
  } else if (tune.sort_bits > 0) {
    const size_t nb = nbm;
    uint32_t *hist = (uint32_t *)base;
    base += al(4 * nb);
    uint32_t *off = (uint32_t *)base;
    base += al(4 * nb);
    uint32_t *tiles = (uint32_t *)base;
    SortParams sp;
    for (int d = 0; d < 3; ++d) {
      sp.lo[d] = m.dom_lo[d];
      float ext = m.dom_hi[d] - m.dom_lo[d];
      sp.inv[d] = ext > 0 ? 1.f / ext : 0.f;
    }
    sp.shift = 30 - tune.sort_bits;
    cudaMemsetAsync(hist, 0, 4 * nb, stream);
    k_bucket_count<MortonKey><<<blocks_for(n, T * kSortItems), T, 0, stream>>>(
        q, n, MortonKey{sp}, hist, key_rank);
    bucket_scan(hist, off, tiles, (int)nb, stream);
    k_bucket_scatter<<<blocks_for(n, T * kSortItems), T, 0, stream>>>(q, n, key_rank, off,
                                                                      sorted);
  } else {
    k_identity<<<blocks_for(n, T), T, 0, stream>>>(q, n, sorted);
  }
  const int bt = tune.block_threads;
  if (ev) cudaEventRecord(ev[1], stream);
  const int ranges = (grouped && split && !ev) ? 1 + split->n_aux : 1;
  if (ranges > 1) {
    // The passes after the first sort as `ranges` contiguous ranges of the
    // sorted stream, concurrently: a range of queries sorted by seed vertex
    // is a compact region, so its lanes still share lists, while the ranges'
    // kernels fill the SM time one pipeline leaves idle (small scans,
    // kernel tails).  Each range has its own vertex histogram, offsets and
    // scan tiles (after the single-range scratch); the records land in the
    // caller's order, so one k_unpack on the launching stream follows the
    // join.  Results do not depend on the split.
    if (scratch_bytes < query_scratch_bytes(n, tune.sort_bits, m.nv, ranges))
      return cudaErrorInvalidValue;
    const int walk = !m.nb_off ? 0 : (tune.nn_walk == 2 && !m.seed ? 1 : tune.nn_walk);
    char *extra = (char *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255) +
                  (query_scratch_bytes(n, tune.sort_bits, m.nv) - 256);
    const size_t ext = 2 * al(4 * (size_t)(m.nv + 1)) + al(4 * kMaxScanTiles);
    const int64_t cn = (n + ranges - 1) / ranges;
    cudaError_t e = cudaEventRecord(split->fork, stream);
    for (int r = 0; r < ranges && e == cudaSuccess; ++r) {
      const int64_t a = r * cn, b = min(n, a + cn);
      if (a >= b) break;
      const int64_t nr = b - a;
      cudaStream_t sr = r == 0 ? stream : split->aux[r - 1];
      uint32_t *vh = vhist, *vo = voff, *tl = tiles2;
      if (r > 0) {
        char *x = extra + (size_t)(r - 1) * ext;
        vh = (uint32_t *)x;
        vo = (uint32_t *)(x + al(4 * (size_t)(m.nv + 1)));
        tl = (uint32_t *)(x + 2 * al(4 * (size_t)(m.nv + 1)));
        e = cudaStreamWaitEvent(sr, split->fork, 0);
      }
      cudaMemsetAsync(vh, 0, 4 * (size_t)(m.nv + 1), sr);
      k_nn_pass<<<blocks_for(nr, bt), bt, 0, sr>>>(m, sorted + a, nr, walk, vh, key_rank + a);
      bucket_scan(vh, vo, tl, (int)(m.nv + 1), sr);
      k_vertex_scatter<<<blocks_for(nr, T), T, 0, sr>>>(sorted + a, nr, key_rank + a, vo,
                                                         grouped_q + a, gv + a);
      const int G = tune.lanes_per_query;
      const unsigned lb = blocks_for(nr * G, bt);
      if (G == 8)
        k_list_pass<8><<<lb, bt, 0, sr>>>(m, grouped_q + a, gv + a, nr, tune.chunked, rec);
      else if (G == 4)
        k_list_pass<4><<<lb, bt, 0, sr>>>(m, grouped_q + a, gv + a, nr, tune.chunked, rec);
      else if (G == 2)
        k_list_pass<2><<<lb, bt, 0, sr>>>(m, grouped_q + a, gv + a, nr, tune.chunked, rec);
      else
        k_list_pass<1><<<lb, bt, 0, sr>>>(m, grouped_q + a, gv + a, nr, tune.chunked, rec);
      if (r > 0 && e == cudaSuccess) e = cudaEventRecord(split->join[r - 1], sr);
      if (r > 0 && e == cudaSuccess) e = cudaStreamWaitEvent(stream, split->join[r - 1], 0);
    }
    if (e != cudaSuccess) return e;
    k_unpack<<<blocks_for(n, T), T, 0, stream>>>(rec, n, dist, closest, prim_id, prim_type, save,
                                                 status);
    return cudaGetLastError();
  }
  if (grouped) {
    const int walk = !m.nb_off ? 0 : (tune.nn_walk == 2 && !m.seed ? 1 : tune.nn_walk);
    cudaMemsetAsync(vhist, 0, 4 * (size_t)(m.nv + 1), stream);
    k_nn_pass<<<blocks_for(n, bt), bt, 0, stream>>>(m, sorted, n, walk, vhist, key_rank);
    if (ev) cudaEventRecord(ev[2], stream);
    bucket_scan(vhist, voff, tiles2, (int)(m.nv + 1), stream);
    k_vertex_scatter<<<blocks_for(n, T), T, 0, stream>>>(sorted, n, key_rank, voff, grouped_q,
                                                         gv);
    if (ev) cudaEventRecord(ev[3], stream);
    const int G = tune.lanes_per_query;
    const unsigned lb = blocks_for(n * G, bt);
    if (G == 8)
      k_list_pass<8><<<lb, bt, 0, stream>>>(m, grouped_q, gv, n, tune.chunked, rec);
    else if (G == 4)
      k_list_pass<4><<<lb, bt, 0, stream>>>(m, grouped_q, gv, n, tune.chunked, rec);
    else if (G == 2)
      k_list_pass<2><<<lb, bt, 0, stream>>>(m, grouped_q, gv, n, tune.chunked, rec);
    else
      k_list_pass<1><<<lb, bt, 0, stream>>>(m, grouped_q, gv, n, tune.chunked, rec);
    if (ev) cudaEventRecord(ev[4], stream);
    k_unpack<<<blocks_for(n, T), T, 0, stream>>>(rec, n, dist, closest, prim_id, prim_type, save,
                                                 status);
    if (ev) cudaEventRecord(ev[5], stream);
    return cudaGetLastError();
  }
  const size_t wsm = (size_t)(bt / 32) * sizeof(WarpSmem);
  const int walk = !m.nb_off ? 0 : (tune.nn_walk == 2 && !m.seed ? 1 : tune.nn_walk);
  const int chunked = tune.chunked;
  if (ev) {
    cudaEventRecord(ev[2], stream);
    cudaEventRecord(ev[3], stream);
  }
  if (counters) {
    cudaMemsetAsync(counters, 0, 6 * sizeof(unsigned long long), stream);
    if (tune.warp_mode)
      k_query_warp<true><<<blocks_for(n, bt), bt, wsm, stream>>>(m, sorted, n, nullptr, nullptr,
                                                                 nullptr, nullptr, nullptr,
                                                                 nullptr, counters, walk);
    else
      k_query_count<<<blocks_for(n, bt), bt, 0, stream>>>(m, sorted, n, counters, walk, chunked);
  } else if (tune.warp_mode) {
    k_query_warp<false><<<blocks_for(n, bt), bt, wsm, stream>>>(m, sorted, n, dist, closest,
                                                                prim_id, prim_type, save, status,
                                                                nullptr, walk);
  } else {
    k_query<<<blocks_for(n, bt), bt, 0, stream>>>(m, sorted, n, dist, closest, prim_id,
                                                  prim_type, save, status, walk, chunked);
  }
  if (ev) {
    cudaEventRecord(ev[4], stream);
    cudaEventRecord(ev[5], stream);
  }
  return cudaGetLastError();
}

cudaError_t launch_nearest(const DevView &m, const float *xyz, int64_t n, int32_t *out_pos,
                           cudaStream_t stream, bool original_ids, int nn_walk) {
  if (n <= 0) return cudaSuccess;
  if (nn_walk && !m.nb_off) return cudaErrorInvalidValue;
  if (nn_walk == 2 && !m.seed) nn_walk = 1;
  k_nearest<<<blocks_for(n, 128), 128, 0, stream>>>(m, xyz, n, out_pos, original_ids ? 1 : 0,
                                                    nn_walk);
  return cudaGetLastError();
}

cudaError_t launch_seed_grid(const DevView &m, uint32_t *seed, cudaStream_t stream) {
  if (m.grid_bits <= 0) return cudaSuccess;
  const int64_t cells = (int64_t)1 << (3 * m.grid_bits);
  k_seed_grid<<<blocks_for(cells, 128), 128, 0, stream>>>(m, seed);
  return cudaGetLastError();
}

cudaError_t launch_backward(const DevView &m, const float *q, const float *dist,
                            const float *closest, const float4 *save, const float *grad_dist,
                            int64_t n, float *grad_q, float *grad_verts, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_backward<<<blocks_for(n, 256), 256, 0, stream>>>(m, q, dist, closest, save, grad_dist, n,
                                                     grad_q, grad_verts);
  return cudaGetLastError();
}

cudaError_t launch_update_vertices(const GeometryRefs &g, const float *verts,
                                   cudaStream_t stream) {
  const int T = 256;
  if (g.nv <= 0) return cudaSuccess;
  k_update_points<<<blocks_for(g.nv, T), T, 0, stream>>>(g.kd_points, g.nv, verts);
  if (g.n_nb > 0 && g.nbp && g.nb)
    k_update_neighbours<<<blocks_for(g.n_nb, T), T, 0, stream>>>(g.nbp, g.nb, g.n_nb,
                                                                  g.kd_points);
  if (g.ne > 0)
    k_update_edges<<<blocks_for(g.ne, T), T, 0, stream>>>(g.edge_rec, g.edges, g.ne, verts);
  if (g.nf > 0)
    k_update_faces<<<blocks_for(g.nf, T), T, 0, stream>>>(g.face_rec, g.tris, g.nf, verts);
  for (int l = g.depth - 1; l >= 0; --l) {
    const int64_t first = ((int64_t)1 << l) - 1, count = (int64_t)1 << l;
    k_update_kd_level<<<blocks_for(count, T), T, 0, stream>>>(g.kd_nodes, g.kd_points, g.nv,
                                                              g.depth, first, count);
  }
  return cudaGetLastError();
}

size_t batch_scratch_bytes(int64_t total, int n_meshes, int sort_bits, int64_t nv_keys) {
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nb = (size_t)n_meshes << sort_bits;
  size_t b = al(16 * (size_t)total) + al(8 * (size_t)total) + 2 * al(4 * nb) +
             al(4 * kMaxScanTiles) + 256;
  if (nv_keys > 0)  // regrouping: vertex key per query, second float4 stream, records,
                    // vertex histogram and offsets
    b += al(4 * (size_t)total) + al(16 * (size_t)total) + al(32 * (size_t)total) +
         2 * al(4 * (size_t)nv_keys);
  return b;
}

int batch_occupancy(int block_threads, int group_by_vertex) {
  int blocks = 0;
  if (group_by_vertex)  // the G variants differ only in index arithmetic
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_batch_list<1>, block_threads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_batch_query, block_threads, 0);
  return blocks > 0 ? blocks : 1;
}

cudaError_t launch_batch(const BatchDesc &d, int64_t total, void *scratch, size_t scratch_bytes,
                         const BatchTuning &t, int grid, unsigned int *queue_head,
                         unsigned int *error_word, cudaStream_t stream) {
  if (total <= 0) return cudaSuccess;
  if (d.n_meshes > kMaxBatchMeshes || t.tile <= 0) return cudaErrorInvalidValue;
  const int64_t nv_keys = t.group_by_vertex ? d.nv_keys : 0;
  if (nv_keys > (int64_t)kScanTile * kMaxScanTiles) return cudaErrorInvalidValue;
  if (scratch_bytes < batch_scratch_bytes(total, d.n_meshes, t.sort_bits, nv_keys))
    return cudaErrorInvalidValue;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char *base = (char *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  float4 *sorted = (float4 *)base;
  base += al(16 * (size_t)total);
  uint2 *key_rank = (uint2 *)base;
  base += al(8 * (size_t)total);
  const size_t nb = (size_t)d.n_meshes << t.sort_bits;
  uint32_t *hist = (uint32_t *)base;
  base += al(4 * nb);
  uint32_t *off = (uint32_t *)base;
  base += al(4 * nb);
  uint32_t *tiles = (uint32_t *)base;
  const int T = 256;
  cudaMemsetAsync(hist, 0, 4 * nb, stream);
  k_batch_count<<<blocks_for(total, T), T, 0, stream>>>(d, total, t.sort_bits, hist, key_rank);
  bucket_scan(hist, off, tiles, (int)nb, stream);
  k_batch_scatter<<<blocks_for(total, T), T, 0, stream>>>(d, total, key_rank, off, sorted);
  cudaMemsetAsync(queue_head, 0, sizeof(unsigned int), stream);
  if (nv_keys > 0) {
    base = (char *)tiles + al(4 * kMaxScanTiles);
    uint32_t *gv = (uint32_t *)base;
    base += al(4 * (size_t)total);
    float4 *grouped = (float4 *)base;
    base += al(16 * (size_t)total);
    float4 *rec = (float4 *)base;
    base += al(32 * (size_t)total);
    uint32_t *vhist = (uint32_t *)base;
    base += al(4 * (size_t)nv_keys);
    uint32_t *voff = (uint32_t *)base;
    cudaMemsetAsync(vhist, 0, 4 * (size_t)nv_keys, stream);
    k_batch_nn<<<blocks_for(total, t.block_threads), t.block_threads, 0, stream>>>(
        d, sorted, total, vhist, key_rank);
    bucket_scan(vhist, voff, tiles, (int)nv_keys, stream);
    k_vertex_scatter<<<blocks_for(total, T), T, 0, stream>>>(sorted, total, key_rank, voff,
                                                             grouped, gv);
    if (t.lanes_per_query == 4)
      k_batch_list<4><<<grid, t.block_threads, 0, stream>>>(d, grouped, gv, total, t.tile, rec,
                                                            queue_head, error_word);
    else if (t.lanes_per_query == 2)
      k_batch_list<2><<<grid, t.block_threads, 0, stream>>>(d, grouped, gv, total, t.tile, rec,
                                                            queue_head, error_word);
    else
      k_batch_list<1><<<grid, t.block_threads, 0, stream>>>(d, grouped, gv, total, t.tile, rec,
                                                            queue_head, error_word);
    k_batch_unpack<<<blocks_for(total, T), T, 0, stream>>>(d, rec, total);
    return cudaGetLastError();
  }
  k_batch_query<<<grid, t.block_threads, 0, stream>>>(d, sorted, total, t.tile, queue_head,
                                                      error_word);
  return cudaGetLastError();
}

}  // namespace p2m
