// kernels.h -- device layout view and the host-side launchers of the query
// kernels (implemented in kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace p2m {

// Read-only view of one mesh's device layout (see builder.h for formats).
struct DevView {
  const float4 *kd_nodes;   // (L-1) * 3: child boxes of every internal node
  const float4 *kd_points;  // nv: x, y, z, original vertex id bits
  const uint32_t *row_off;  // nv + 1
  const uint4 *entries;     // per entry: typed id + 15-bit box codes in its chunk's frame
  const float4 *edge_rec;   // 2 per edge
  const float4 *face_rec;   // 3 per face
  const int2 *edges;        // canonical edges
  const int4 *tris;         // faces (a, b, c, 0)
  const uint32_t *nb_off;   // nv + 1: Voronoi neighbours of each row (CSR)
  const uint32_t *nb;       // neighbour rows
  const float4 *nbp;        // neighbour positions, parallel to nb: x, y, z, row bits
  const uint32_t *chunk_off;  // nv + 1: chunks of each row (CSR)
  const uint4 *chunks;        // per chunk: box codes in the frame below + entry-frame exponents
  const uint32_t *super_off;  // nv + 1: super-chunks (8 chunks each) of each row
  const uint4 *supers;        // per super-chunk: box codes in the same frame
  float qlo[3], qinv[3];      // frame of the chunk boxes (quant.h)
  float qstep[3], qbase[3];   // 1 / qinv and qlo - qstep (float ops, quant.h)
  const uint32_t *seed;       // G^3 rows: nearest vertex of every seed-grid cell centre
  int grid_bits;              // G = 2^grid_bits cells per axis over D (0 = no grid)
  const uint32_t *sort_seed;  // the same at 2^sort_grid_bits <= 256 cells per axis (small
  int sort_grid_bits;         // enough for L2): the key of the seed-vertex sort
  int64_t nv;
  int64_t L;                // KD-tree leaves (2^depth)
  int depth;
  float dom_lo[3], dom_hi[3];
};

// Launch configuration of the query path.
struct QueryTuning {
  int sort_bits = 18;
  int block_threads = 256;
  int warp_mode = 0;  // 0: one thread per query, 1: warp-cooperative KD walk
  int nn_walk = 2;    // 0: KD-tree backtracking, 1: KD descent + Voronoi walk,
                      // 2: seed-grid lookup + Voronoi walk
  int chunked = 2;    // 0: scan every list entry, 1: chunk boxes first,
                      // 2: super-chunk boxes, then chunk boxes
  int group_by_vertex = 1;  // 1: nearest-vertex pass, regroup queries by
                            // vertex, then the list pass (two kernels)
  int sort_key = 0;  // 0: Morton buckets (2^sort_bits); 1: the seed-grid vertex of
                     // the query's cell (with group_by_vertex and a seed grid)
  int lanes_per_query = 1;  // threads per query in the list pass (1, 2, 4, 8)
  int streams = 1;  // after the first sort, the passes of the two-pass path run as up to
                    // this many contiguous ranges of the sorted queries on forked streams
};

// Scratch needed by launch_query for n points, in bytes (nv: vertices of
// the mesh, for the regrouping by nearest vertex; 0 = no regrouping; ranges:
// concurrent ranges of the sorted stream, each with its own vertex histogram).
size_t query_scratch_bytes(int64_t n, int sort_bits, int64_t nv = 0, int ranges = 1);

// Streams for the concurrent ranges of a split query: range r > 0 runs on
// aux[r - 1], which waits on `fork` (recorded on the launching stream after
// the first sort) and is joined back through join[r - 1]; n_aux + 1 ranges.
struct SplitStreams {
  const cudaStream_t *aux;
  const cudaEvent_t *join;
  cudaEvent_t fork;
  int n_aux;
};

// Morton bucket sort (a1) + query (a2..a8).  All pointers device.
// ev (6 events or NULL) marks: start, sorted, nearest vertices found,
// regrouped by vertex, list pass done, outputs written (the one-pass kernel
// records events 2 and 3 where it starts and 4 and 5 where it ends); with
// `counters` (6 device u64) the counting variant runs instead of the query
// and sums internal nodes, points, entries, edges, faces and chunk boxes.
cudaError_t launch_query(const DevView &m, const float *q, int64_t n, float *dist,
                         float *closest, int32_t *prim_id, uint8_t *prim_type, float4 *save,
                         uint8_t *status, void *scratch, size_t scratch_bytes,
                         const QueryTuning &tune, cudaStream_t stream,
                         cudaEvent_t *ev = nullptr, unsigned long long *counters = nullptr,
                         const SplitStreams *split = nullptr);

// Nearest vertex (KD-tree position) of each point: used by the builder to
// certify Voronoi cells.
cudaError_t launch_nearest(const DevView &m, const float *xyz, int64_t n, int32_t *out_pos,
                           cudaStream_t stream, bool original_ids = false, int nn_walk = 0);

// Fill the seed grid: nearest vertex (row) of every cell centre of the
// G^3 grid over D (G = 2^view.grid_bits), by KD-tree backtracking.
cudaError_t launch_seed_grid(const DevView &m, uint32_t *seed, cudaStream_t stream);

// Mutable device arrays of the vertex-dependent geometry (p2m_update_vertices).
struct GeometryRefs {
  float4 *kd_points;   // nv
  float4 *kd_nodes;    // (2^depth - 1) * 3
  float4 *nbp;         // n_nb
  const uint32_t *nb;  // n_nb
  float4 *edge_rec;    // 2 * ne
  float4 *face_rec;    // 3 * nf
  const int2 *edges;   // ne
  const int4 *tris;    // nf
  int64_t nv, n_nb, ne, nf;
  int depth;
};

// New vertex positions (original order, nv x 3 float, device): KD points and
// child boxes, neighbour positions, edge and face records.
cudaError_t launch_update_vertices(const GeometryRefs &g, const float *verts,
                                   cudaStream_t stream);

// Backward scatter (a9).
cudaError_t launch_backward(const DevView &m, const float *q, const float *dist,
                            const float *closest, const float4 *save, const float *grad_dist,
                            int64_t n, float *grad_q, float *grad_verts, cudaStream_t stream);

// Batched persistent query (a10): every mesh's queries in one Morton sort
// keyed by (mesh, bucket), then one persistent kernel whose CTAs take tiles
// of the sorted stream from an atomic counter.
struct BatchIO {
  const float *q;
  int64_t n;
  float *dist;
  float *closest;
  int32_t *prim_id;
  uint8_t *prim_type;
};
struct BatchDesc {           // device pointers
  const DevView *views;      // n_meshes
  const BatchIO *ios;        // n_meshes
  const int64_t *qoff;       // n_meshes + 1 prefix sums of the query counts
  const int64_t *voff;       // n_meshes + 1 prefix sums of (vertex count + 1)
  int n_meshes;
  int64_t nv_keys;           // voff[n_meshes] (host copy)
};
struct BatchTuning {
  int sort_bits = 12;
  int tile = 1024;
  int block_threads = 256;
  int grid_ctas = 0;
  int group_by_vertex = 1;  // two-pass: nearest vertex, regroup, persistent list pass
  int lanes_per_query = 1;  // threads per query in the persistent list pass (1, 2, 4)
};
size_t batch_scratch_bytes(int64_t total, int n_meshes, int sort_bits, int64_t nv_keys = 0);
cudaError_t launch_batch(const BatchDesc &d, int64_t total, void *scratch, size_t scratch_bytes,
                         const BatchTuning &t, int grid, unsigned int *queue_head,
                         unsigned int *error_word, cudaStream_t stream);
// resident CTAs per SM of the persistent kernel for a block size
int batch_occupancy(int block_threads, int group_by_vertex);

}  // namespace p2m
