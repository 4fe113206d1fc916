/*
 * p2m.h -- C ABI of the GB300 point-to-mesh query library (libp2m.so).
 *
 * The library answers, for every query point q, the closest point on a
 * triangle mesh, the distance to it and the closest primitive (vertex, open
 * edge or open face), following the query stage of P2M (Zong et al., "P2M:
 * A Fast Solver for Querying Distance from Point to Mesh Surface", ACM TOG
 * 2023; query = Alg. A.2, preprocessing = Alg. A.1).
 *
 * Conventions shared by every entry point
 *   - Plain pointers and sizes only.  "host" pointers are CPU memory,
 *     "device" pointers are CUDA global memory on the current device.
 *   - The caller owns every buffer it passes; the library never frees or
 *     keeps a caller pointer beyond the call.  A handle owns its device
 *     layout and a scratch arena, both released by p2m_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it and the call returns without
 *     synchronising, unless stated otherwise.
 *   - Coordinates are float32, xyz interleaved; triangle indices int32.
 *   - Every call returns a p2m_status.  Per-query conditions (non-finite
 *     input, point outside the domain) are reported in the optional status
 *     array, never through the return code.  No call traps the GPU.
 *   - Edge ids follow the canonical order: unique (min,max) vertex pairs
 *     sorted lexicographically (p2m_get_edges exports them).
 */
#ifndef P2M_H
#define P2M_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  P2M_OK = 0,
  P2M_ERR_INVALID_ARG = 1,      /* NULL pointer, negative size, unknown option        */
  P2M_ERR_INVALID_MESH = 2,     /* index out of range, repeated index in a triangle,
                                   unreferenced vertex, non-finite coordinate, no faces */
  P2M_ERR_DUPLICATE_VERTEX = 3, /* two vertices at one position (Voronoi cells would
                                   be undefined; the paper assumes one copy per vertex,
                                   Sec. 4.1)                                            */
  P2M_ERR_OOM = 4,              /* host or device allocation failed                    */
  P2M_ERR_CUDA = 5,             /* a CUDA runtime call failed                          */
  P2M_ERR_QUEUE_TIMEOUT = 6,    /* the batched work queue gave up after its bounded wait */
  P2M_ERR_IO = 7,               /* file missing, short, corrupt or wrong version       */
  P2M_ERR_NO_DEVICE = 8,        /* no usable CUDA device                               */
  P2M_ERR_TOO_LARGE = 9         /* a size exceeds a documented limit                   */
} p2m_status;

/* primitive types; distance ties go to the lower value, then the lower id */
typedef enum { P2M_PRIM_VERTEX = 0, P2M_PRIM_EDGE = 1, P2M_PRIM_FACE = 2 } p2m_prim_type;

/* per-query status bits written to the optional status array */
enum {
  P2M_Q_OUTSIDE_DOMAIN = 1, /* q outside the domain D: answered, exactness not guaranteed */
  P2M_Q_NONFINITE = 2       /* q has a NaN/inf coordinate: outputs are NaN / -1       */
};

/* A triangle mesh with one shared copy per vertex (Sec. 4.1).  Host memory. */
typedef struct {
  const float *verts;   /* n_verts * 3 */
  int64_t n_verts;
  const int32_t *tris;  /* n_tris * 3 */
  int64_t n_tris;
} p2m_mesh;

/* Build options.  Pass NULL to p2m_build for the defaults. */
typedef struct {
  float domain_scale;  /* query domain D = bbox scaled about its centre by this factor
                          (default 10: the paper samples queries in 10x the bbox, Sec. 5) */
  float domain_margin; /* plus this fraction of the bbox diagonal on every side (default 0) */
  float delta_rel;     /* conservative widening of cells, Space-perp half-spaces, filter
                          and Region boxes, as a fraction of diag(D) (default 4e-6)        */
  int host_threads;    /* preprocessing threads, 0 = all cores (default 0)                 */
  int device_assist;   /* 1 = the exact searches that certify the corners of the Voronoi
                          cells on the GPU (double-precision decisions),
                          2 = that and the flooding (Alg. 1, one warp per primitive) on
                          the GPU, the host threads flooding a share of the primitives
                          beside it, 3 = that, the whole cell stage (one warp per cell)
                          and the packing of the table on the GPU too, 0 = CPU only.  The GPU steps are the host's
                          double-precision steps without fused multiply-adds; what
                          their buffers cannot hold is handed back to the host.
                          Every setting gives the same layout bit for bit (default 3,
                          the fastest build on a GB300; without a GPU every setting
                          builds on the host)                                          */
  int leaf_size;       /* KD-tree bucket size, 2..32 (default 8)                            */
} p2m_build_opts;

/* Fill *opts with the defaults. */
void p2m_default_opts(p2m_build_opts *opts);

typedef struct p2m_handle p2m_handle;

/*
 * Preprocess a mesh (Alg. A.1) and upload the query layout to the current
 * CUDA device: KD tree of V, Voronoi cells of V clipped to D, flooding
 * interception inspection (Alg. 1) with the convexity filter (Thm. 5/6),
 * Region bounding boxes (Sec. 4.6), packed as a CSR interception table.
 * The mesh is copied; `mesh` may be freed after the call.  Synchronous.
 * Errors: INVALID_ARG, INVALID_MESH, DUPLICATE_VERTEX, OOM, CUDA, NO_DEVICE,
 * TOO_LARGE (2^30 vertices or 2^29 triangles or segments and beyond, a table
 * of 2^32 entries, or a domain D reaching beyond +-1e18, where float32
 * squared distances would overflow).
 */
p2m_status p2m_build(const p2m_mesh *mesh, const p2m_build_opts *opts, p2m_handle **out);

/*
 * Environment variables p2m_build reads (diagnostics and tests; none
 * changes the tables it builds):
 *   P2M_BUILD_TRACE        set: time every build stage on stderr.
 *   P2M_FLOOD_UNBOUNDED=1  flood every primitive with the unbounded host code.
 *   P2M_FLOOD_LANES=1      flood on the host with the device kernel's warp
 *                          algorithm, its 32 lanes run one after another.
 *   P2M_INJECT_BAD_ALLOC=<stage>  host fault injection: a worker thread of
 *                          the "cells", "flooding" or "packing" stage throws
 *                          std::bad_alloc; p2m_build returns P2M_ERR_OOM.
 */

/*
 * Mixed primitives (Sec. 5, mixed segments and triangles): p2m_build with,
 * besides the mesh's triangles (n_tris may be 0, tris then NULL), n_segs
 * segments `segs` (2 vertex indices each, host memory) that are edges of no
 * face, e.g. a wireframe beside a surface.  Segments join the canonical edge
 * list (a segment that repeats a face side is that edge) and are reported
 * as P2M_PRIM_EDGE; the Space-perp of a segment is the slab between the
 * planes through its endpoints.  Every vertex must be used by a triangle or
 * a segment.  Errors as p2m_build.
 */
p2m_status p2m_build_mixed(const p2m_mesh *mesh, const int32_t *segs, int64_t n_segs,
                           const p2m_build_opts *opts, p2m_handle **out);

/* Release the handle and all device memory it owns (NULL is a no-op). */
void p2m_destroy(p2m_handle *h);

/*
 * Closest point query (Alg. A.2) for n points, on `stream`.
 *   q            device, n*3 float   query points
 *   dist         device, n float     distance to the mesh
 *   closest      device, n*3 float   closest point (may be NULL)
 *   prim_id      device, n int32     vertex / edge / face id of the closest primitive
 *   prim_type    device, n uint8     p2m_prim_type (may be NULL)
 *   save         device, n*4 float   what p2m_backward needs: {typed id bits, w0, w1, w2}
 *                                    (barycentric weights of the closest point), or NULL
 *   status       device, n uint8     P2M_Q_* bits, or NULL
 * Outputs are in the caller's order.  Queries are Morton-sorted internally
 * (scratch owned by the handle; grown on demand, see p2m_reserve).
 * n == 0 is a no-op.  Errors: INVALID_ARG, OOM, CUDA, TOO_LARGE (n >= 2^31).
 */
p2m_status p2m_query(p2m_handle *h, const float *q, int64_t n, float *dist, float *closest,
                     int32_t *prim_id, uint8_t *prim_type, float *save, uint8_t *status,
                     void *stream);

/* Nearest mesh vertex of each of n device points (the KD-tree search of
 * Alg. A.2, first line): vertex[i] = original vertex id, -1 for a
 * non-finite point.  Ties between equidistant vertices may go either way
 * within float32 rounding.  Errors: INVALID_ARG, CUDA, TOO_LARGE. */
p2m_status p2m_nearest_vertex(p2m_handle *h, const float *q, int64_t n, int32_t *vertex,
                              void *stream);

/* Same as p2m_query with HOST buffers: copies q in, runs, copies results out,
 * synchronises `stream` before returning (dist/prim_id required, others may
 * be NULL). */
p2m_status p2m_query_host(p2m_handle *h, const float *q, int64_t n, float *dist, float *closest,
                          int32_t *prim_id, uint8_t *prim_type, void *stream);

/* Pipelined host-buffer queries (the paper queries one point at a time and
 * has no counterpart; this is p2m_query_host for a stream of batches).  A
 * pipe holds `depth` (1..8) slots, each with its own CUDA stream and device
 * scratch sized for batches of up to max_n queries (about 110 B per query
 * plus the handle's per-vertex histogram); p2m_pipe_create allocates them
 * (synchronous).  p2m_pipe_submit enqueues one batch on the next slot:
 * copy q (n x 3 host floats) in, run the query with the handle's current
 * tuning, copy dist and prim_id (and closest, prim_type when not NULL) out
 * to the given host buffers, and returns without waiting, except for the
 * slot's previous batch.  The host buffers must stay untouched until
 * p2m_pipe_wait returns (or the slot comes round again); they should be
 * pinned (cudaHostAlloc / torch pin_memory) for the copies to overlap the
 * kernels of the other slots.  The handle must outlive the pipe.
 * Errors: INVALID_ARG, OOM, CUDA, TOO_LARGE (n > max_n, max_n >= 2^31). */
typedef struct p2m_pipe p2m_pipe;
p2m_status p2m_pipe_create(p2m_handle *h, int64_t max_n, int depth, p2m_pipe **out);
p2m_status p2m_pipe_submit(p2m_pipe *p, const float *q, int64_t n, float *dist, float *closest,
                           int32_t *prim_id, uint8_t *prim_type);
/* A batch on DEVICE buffers on the pipe's next slot: the query of the n
 * device points q runs on the slot's stream with the slot's scratch (no
 * copies), after the work enqueued so far on `stream`, writing the device
 * outputs (dist and prim_id required; closest, prim_type may be NULL).  It
 * returns without waiting, except for the slot's previous batch.  Batches on
 * different slots may run concurrently, which keeps the SMs busier than one
 * batch at a time; the outputs are complete after p2m_pipe_wait, or on a
 * stream after p2m_pipe_join.  Errors as p2m_pipe_submit. */
p2m_status p2m_pipe_submit_device(p2m_pipe *p, const float *q, int64_t n, float *dist,
                                  float *closest, int32_t *prim_id, uint8_t *prim_type,
                                  void *stream);
/* Makes `stream` wait for every batch submitted so far (no host wait). */
p2m_status p2m_pipe_join(p2m_pipe *p, void *stream);
/* Waits for every submitted batch; their host outputs are then complete. */
p2m_status p2m_pipe_wait(p2m_pipe *p);
void p2m_pipe_destroy(p2m_pipe *p);

/*
 * p2m_query without any device allocation (the paper has no counterpart;
 * this is a deployment variant of p2m_query).  For callers that must not
 * call cudaMalloc while they run: processes whose GPU memory belongs to
 * another allocator, real-time loops that cannot take the device-wide
 * synchronisation of cudaMalloc/cudaFree, plugin hosts that forbid
 * allocation after start-up.  The sort scratch is a static device array of
 * about 24.5 MB that every GPU loading this library keeps until the process
 * exits.  Arguments and outputs as in p2m_query (device pointers; closest
 * and prim_type may be NULL; no save or status outputs).
 *   - n may be at most 1,048,576 (2^20); larger n returns P2M_ERR_TOO_LARGE.
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - Every call on a device shares the one array, and each call clears the
 *     part that must start at zero.  Calls whose GPU work overlaps (different
 *     streams, or different host threads, without ordering between them)
 *     race on the array and may return wrong results: order them.
 * Allocates nothing (no cudaMalloc/cudaFree, no allocating library call).
 * Errors: INVALID_ARG, NO_DEVICE, TOO_LARGE, CUDA.
 */
p2m_status p2m_query_noalloc(p2m_handle *h, const float *q, int64_t n, float *dist,
                             float *closest, int32_t *prim_id, uint8_t *prim_type, void *stream);

/* Launch tuning of the query path (chosen by the autotuner or by hand).
 *   sort_bits      Morton bucket bits of the query sort, 0..24 (0 = no sort);
 *                  queries are grouped into 2^sort_bits spatial buckets
 *   block_threads  threads per CTA of the query kernel: 64, 128, 256 or 512
 *   warp_cooperative  0: one thread per query; 1: a warp answers 32 sorted
 *                  queries together (shared KD-tree walk decided by ballots,
 *                  each distinct interception list staged once through
 *                  shared memory).  Results are identical.
 *   nn_walk        nearest-vertex search: 0 = KD-tree descent with
 *                  backtracking (Sec. 2.1); 1 = KD-tree descent to one leaf,
 *                  then a walk over Voronoi neighbours to the nearest vertex
 *                  (exact: a vertex nearer than all its Voronoi neighbours is
 *                  the nearest; points outside D use backtracking); 2 = the
 *                  walk starts from a seed grid over D whose cells hold the
 *                  nearest vertex of their centres (default).
 *   chunked        list scan: 0 = test the Region box of every entry; 1 =
 *                  test the box of each chunk of 8 spatially ordered
 *                  entries first; 2 = test the box of each group of 8
 *                  chunks first, then chunk boxes (a two-level R-tree per
 *                  list, Sec. 4.6; default).
 *   group_by_vertex  1 = two passes: nearest vertex of every query, a
 *                  counting sort of the queries by that vertex, then the
 *                  list scans, so the lanes of a warp share interception
 *                  lists (default); 0 = one fused kernel.
 *   sort_key       0 = the first sort orders the queries by Morton bucket
 *                  (2^sort_bits buckets, default); 1 = by the vertex a seed
 *                  grid gives their cell (a 256^3 copy of the walk's grid
 *                  when that is finer), so the lanes of a warp start their
 *                  Voronoi walks near the same vertex (needs
 *                  group_by_vertex = 1; otherwise the Morton sort runs;
 *                  sort_bits unused).  Results do not depend on it.
 *   lanes_per_query  threads per query in the list pass of the two-pass
 *                  path: 1, 2, 4 or 8 adjacent lanes split a query's
 *                  interception list (every G-th group of 64 entries) and
 *                  keep the best with a warp shuffle.  Results do not
 *                  depend on it.
 *   streams        1..4 (two-pass path): after the first sort, the
 *                  nearest-vertex pass, the regrouping and the list pass run
 *                  as up to this many contiguous ranges of the sorted
 *                  queries (each at least 2^18), the first on the caller's
 *                  stream and the others on streams the handle forks from it
 *                  with an event and joins back to it, so that the ranges'
 *                  kernels run concurrently; the output write follows the
 *                  join.  The call still ends on the caller's stream (graph
 *                  capture works as for one stream, after p2m_reserve);
 *                  results do not depend on it.  While per-phase timing is
 *                  on (p2m_set_timing) a call runs as one pipeline. */
typedef struct {
  int sort_bits;
  int block_threads;
  int warp_cooperative;
  int nn_walk;
  int chunked;
  int group_by_vertex;
  int sort_key;
  int lanes_per_query;
  int streams;
} p2m_tuning;
p2m_status p2m_get_tuning(const p2m_handle *h, p2m_tuning *t);
p2m_status p2m_set_tuning(p2m_handle *h, const p2m_tuning *t);

/* Instrumentation.  While timing is enabled, every p2m_query records CUDA
 * events on the caller's stream between its phases (a ring of the last 1024
 * calls; no host synchronisation).  p2m_timing_summary waits for the calls
 * recorded since its previous call and returns {calls, total ms of the
 * Morton sort, of the nearest-vertex pass, of the regrouping by vertex, of
 * the list pass, of the output write} (the one-pass kernel counts entirely
 * as list pass; its output write is part of it and counts 0).  Enabling (or
 * disabling) clears the ring. */
p2m_status p2m_set_timing(p2m_handle *h, int enable);
p2m_status p2m_timing_summary(p2m_handle *h, double out[6]);

/* Work counters of a query batch (device q, n points): runs a counting
 * variant of the query kernel (outputs are not written) and returns the
 * totals of KD-tree internal nodes visited, vertices examined, list entries
 * scanned, edges tested, faces tested and chunk boxes tested in out[0..5].
 * Synchronous. */
p2m_status p2m_query_counters(p2m_handle *h, const float *q, int64_t n, int64_t out[6],
                              void *stream);

/* Pre-size the handle's scratch arena for queries of up to n points, so that
 * later p2m_query calls with n or fewer points allocate nothing (needed
 * before capturing p2m_query into a CUDA graph); it also creates the forked
 * streams of split calls (tuning field streams). */
p2m_status p2m_reserve(p2m_handle *h, int64_t n);

/*
 * Backward pass of d(q) = |q - c(q)| for n queries, on `stream`.  With
 * u = (q - c)/d: grad_q = grad_dist * u, and for the vertices v_k of the
 * closest primitive with barycentric weights w_k (from `save`):
 * grad_verts[v_k] -= grad_dist * w_k * u  (accumulated with atomics, so the
 * caller zeroes grad_verts first if it wants a fresh gradient).  Queries
 * with d == 0 contribute nothing.
 *   q, dist, closest, save: device, as produced by p2m_query
 *   grad_dist    device, n float
 *   grad_q       device, n*3 float or NULL
 *   grad_verts   device, n_verts*3 float or NULL
 * Errors: INVALID_ARG, CUDA.
 */
p2m_status p2m_backward(p2m_handle *h, const float *q, const float *dist, const float *closest,
                        const float *save, const float *grad_dist, int64_t n, float *grad_q,
                        float *grad_verts, void *stream);

/*
 * Move the mesh's vertices (the differentiable path's geometry refresh):
 * the vertex-dependent parts of the device layout are recomputed from new
 * positions on `stream` -- the KD-tree points and child boxes, the Voronoi
 * neighbours' positions and the edge and face records -- while the
 * interception lists and Region boxes (Alg. A.1, Sec. 4.6) stay those of
 * the build.  The distance a later query returns is then the exact distance
 * to the best primitive among its nearest vertex and that vertex's list
 * (Alg. A.2 on the moved geometry), an upper bound of the true distance that
 * equals it wherever the build's list and box still cover the moved closest
 * primitive, which small moves keep for nearly every query; rebuild the
 * handle after large moves.  Positions equal to the build's leave every
 * record unchanged bit for bit.
 *   verts        device, n_verts*3 float, original vertex order (read during
 *                the call's kernels only; the caller keeps ownership)
 *   n_verts      must equal the mesh's vertex count
 *   refresh_seed_grid  1: also recompute the seed grids of the nearest-vertex
 *                walk (one exact search per grid cell, slower); 0: keep them
 *                (the walk then starts from the build's seeds)
 * The host copy of the layout (p2m_save, p2m_get_list) and the domain D are
 * not changed.  Asynchronous on `stream`; no allocation.
 * Errors: INVALID_ARG (NULL verts, wrong count, refresh flag not 0/1),
 * NO_DEVICE, CUDA.
 */
p2m_status p2m_update_vertices(p2m_handle *h, const float *verts, int64_t n_verts,
                               int refresh_seed_grid, void *stream);

/* One mesh's slice of a batched query (device pointers, n points). */
typedef struct {
  const float *q;     /* n*3 */
  int64_t n;
  float *dist;        /* n */
  float *closest;     /* n*3, may be NULL */
  int32_t *prim_id;   /* n */
  uint8_t *prim_type; /* n, may be NULL */
} p2m_batch_io;

/* Tuning of a batched run.
 *   sort_bits  Morton bucket bits per mesh, 0..16 (all meshes share one sort
 *              keyed by (mesh, bucket))
 *   tile       queries per work-queue item, a multiple of block_threads
 *   block_threads, grid_ctas  persistent launch shape (grid_ctas 0 = one
 *              wave: SM count x resident CTAs per SM)
 *   group_by_vertex  1: nearest-vertex pass over all meshes, regroup the
 *              queries by (mesh, nearest vertex), then the persistent list
 *              pass (needs sum of (vertex count + 1) <= 2^24); 0: one
 *              persistent pass per query
 *   lanes_per_query  threads per query in the persistent list pass (1, 2
 *              or 4; with group_by_vertex = 1), as in p2m_tuning */
typedef struct {
  int sort_bits;
  int tile;
  int block_threads;
  int grid_ctas;
  int group_by_vertex;
  int lanes_per_query;
} p2m_batch_tuning;

typedef struct p2m_batch p2m_batch;

/*
 * Many meshes in one persistent launch (the paper has no batched mode).
 * p2m_batch_create checks the slices, allocates the batch's scratch and
 * uploads the mesh descriptors (synchronous; allocates).  p2m_batch_run then
 * enqueues, on `stream`: one Morton sort of all queries keyed by (mesh,
 * bucket), the nearest-vertex pass and the regrouping by (mesh, vertex),
 * one persistent list kernel whose CTAs take tiles of the regrouped queries
 * from a device work queue (a single atomic counter, so no CTA ever waits
 * on another), then the output write.  p2m_batch_run allocates nothing and does not
 * synchronise, so it can be captured into a CUDA graph.  The handles and
 * the io buffers must stay alive while the batch is used.
 * Errors: INVALID_ARG, OOM, CUDA, TOO_LARGE (total queries >= 2^31),
 * QUEUE_TIMEOUT (p2m_batch_check: the device reported a malformed item).
 */
p2m_status p2m_batch_create(p2m_handle *const *meshes, const p2m_batch_io *io, int n_meshes,
                            p2m_batch **out);
p2m_status p2m_batch_run(p2m_batch *b, void *stream);
p2m_status p2m_batch_get_tuning(const p2m_batch *b, p2m_batch_tuning *t);
p2m_status p2m_batch_set_tuning(p2m_batch *b, const p2m_batch_tuning *t);
/* Times every candidate tuning on `stream` (each run `reps` times after one
 * warm-up) and keeps the fastest; *best_ms receives its time. */
p2m_status p2m_batch_autotune(p2m_batch *b, int reps, void *stream, float *best_ms);
/* Synchronises `stream` and reads the device error word of the last runs. */
p2m_status p2m_batch_check(p2m_batch *b, void *stream);
void p2m_batch_destroy(p2m_batch *b);

/* Convenience: create, run, check and destroy (synchronous). */
p2m_status p2m_query_batched(p2m_handle *const *meshes, const p2m_batch_io *io, int n_meshes,
                             void *stream);

/* Times the single-mesh query for every candidate p2m_tuning on the given
 * device queries (reps runs each after a warm-up) and keeps the fastest. */
p2m_status p2m_autotune(p2m_handle *h, const float *q, int64_t n, int reps, void *stream,
                        float *best_ms);

/* Export the canonical edge list (host, n_edges*2).  *n_edges receives the
 * count; pass edges == NULL to query the count only. */
p2m_status p2m_get_edges(const p2m_handle *h, int32_t *edges, int64_t *n_edges);

/* Statistics of the built layout: out[0..15] = n_verts, n_tris, n_edges,
 * table entries, max list length, device bytes, KD-tree leaves, KD-tree
 * depth, voronoi neighbour pairs, flooding inspections, build ms total,
 * cells ms, inspection ms, certification rounds, certification queries,
 * degenerate faces. */
p2m_status p2m_stats(const p2m_handle *h, int64_t out[16]);

/* How the flooding of a handle's build was split: out[0] = primitives
 * flooded on the device (device_assist 2 or 3; how many depends on how fast
 * the host threads flooding beside it are), out[1] = flooded on the host by
 * the bounded core shared with the device, out[2] = flooded on the host by
 * the unbounded code (primitives whose polytopes exceed the core's fixed
 * buffers, or whose cap loop needs the angular ordering).  All zero for a
 * handle made by p2m_load. */
p2m_status p2m_flood_stats(const p2m_handle *h, int64_t out[3]);

/* How the Voronoi cells of a handle's build were split: out[0] = cells
 * made on the device (device_assist = 3), out[1] = made on the host (every
 * cell with device_assist 0 to 2; with 3 the ones whose work overflowed the
 * device's fixed buffers, whose cap loop needs the angular ordering or
 * whose exact search gave up); out[2] = 1 if the table was packed on the
 * device (device_assist = 3; the host packs when a row is longer than the
 * device's sort holds), else 0.  All zero for a handle made by p2m_load. */
p2m_status p2m_cell_stats(const p2m_handle *h, int64_t out[3]);

/* The domain D (lo xyz, hi xyz) and delta of a handle. */
p2m_status p2m_domain(const p2m_handle *h, float out[7]);

/* Interception list of a vertex (original id), host output: types[] and
 * ids[] of up to cap entries, Region boxes box[6*] (lo, hi) or NULL.
 * Returns the list length in *len. */
p2m_status p2m_get_list(const p2m_handle *h, int32_t vertex, int32_t *types, int32_t *ids,
                        float *boxes, int64_t cap, int64_t *len);

/* Serialise the built layout to a file (versioned header + checksum) and
 * load it back onto the current device.  p2m_load checks, besides the
 * checksum, every index the query kernels follow against the array it
 * indexes (tree positions, rows, chunks, typed ids, neighbours), so a file
 * whose contents do not fit is refused before anything reaches the device.
 * Errors: IO (missing, short, corrupt, wrong version or inconsistent
 * contents), OOM, CUDA. */
p2m_status p2m_save(const p2m_handle *h, const char *path);
p2m_status p2m_load(const char *path, p2m_handle **out);

/* Human-readable name of a status code (static string). */
const char *p2m_status_string(p2m_status s);

#ifdef __cplusplus
}
#endif
#endif /* P2M_H */
