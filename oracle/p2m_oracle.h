/*
 * p2m_oracle.h -- plain FP64 CPU reference of the P2M point-to-mesh method
 * (Zong et al., "P2M: A Fast Solver for Querying Distance from Point to Mesh
 * Surface", ACM TOG 2023).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA product
 * path shares no code, header, table or helper with it.
 *
 * Two oracles live here:
 *   - the plain definition (orc_bruteforce): the distance from a point to
 *     the mesh is the minimum over all vertices, open edges and open faces of
 *     the distance to that primitive, where an open edge (face) only counts
 *     when the orthogonal projection falls strictly inside it (Sec. 4.1,
 *     open point sets; Alg. A.2 gating);
 *   - the paper's method: preprocessing of Alg. A.1 (Space-perp half-spaces,
 *     Voronoi cells of V, KD tree, flooding interception inspection of
 *     Alg. 1 with the convexity filter of Thm. 5/6, Region bounding boxes of
 *     Sec. 4.6) and the query of Alg. A.2.
 *
 * All arithmetic is double precision (Sec. 5.4 states the paper's code uses
 * double-precision variables).  Inputs are float32 coordinates widened
 * exactly to double by the caller.
 */
#ifndef P2M_ORACLE_H
#define P2M_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (0 = ok) */
enum {
  ORC_OK = 0,
  ORC_BAD_ARG = 1,
  ORC_BAD_INDEX = 2,        /* vertex index out of range                */
  ORC_REPEATED_INDEX = 3,   /* a triangle or segment names a vertex twice */
  ORC_DUPLICATE_VERTEX = 4, /* two vertices share a position            */
  ORC_UNREFERENCED = 5,     /* a vertex used by no triangle or segment  */
  ORC_NONFINITE = 6,        /* NaN / inf coordinate                      */
  ORC_NOMEM = 7,
  ORC_EMPTY = 8             /* no triangles and no segments              */
};

/* primitive types, ordered for tie breaks: vertex < edge < face */
enum { ORC_VERTEX = 0, ORC_EDGE = 1, ORC_FACE = 2 };

typedef struct orc_mesh orc_mesh;

/* Build topology, the KD tree of V and (if build_tables) the Voronoi cells,
 * the interception table and the Region boxes.  The query domain D is the
 * bbox of V scaled by domain_scale about its centre plus domain_margin *
 * bbox diagonal on every side.  delta_rel * diag(D) is the conservative
 * margin delta (cells, Space-perp half-spaces and the filter are widened by
 * it, so the table can only grow).  n_threads <= 0 uses 1 thread. */
orc_mesh *orc_create(const double *V, int64_t nv, const int32_t *F, int64_t nf,
                     double domain_scale, double domain_margin, double delta_rel,
                     int build_tables, int n_threads, int *status);
/* Mixed primitives (Sec. 5, mixed segments and triangles): S holds ns
 * segments (vertex index pairs) that are edges of no face; the segments'
 * Space-perp is the slab between their endpoint planes (reading of Eq. 5
 * with no adjacent face).  nf may be 0 (a wireframe).  orc_create is this
 * with ns = 0. */
orc_mesh *orc_create_mixed(const double *V, int64_t nv, const int32_t *F, int64_t nf,
                           const int32_t *S, int64_t ns, double domain_scale,
                           double domain_margin, double delta_rel, int build_tables,
                           int n_threads, int *status);
/* orc_create_mixed with the Voronoi neighbours given (off in orc_create
 * and orc_create_mixed): cand_off[nv+1], cand[] hold the Delaunay
 * neighbours of every vertex (CSR, no self entries), e.g. from a library
 * triangulation.  The Voronoi cell of v is then D clipped by the bisectors of
 * exactly these vertices, with no k-nearest seeding and no corner
 * certification.  The arrays are read during the call only.  NULL, NULL:
 * the certified construction. */
orc_mesh *orc_create_ex(const double *V, int64_t nv, const int32_t *F, int64_t nf,
                        const int32_t *S, int64_t ns, double domain_scale, double domain_margin,
                        double delta_rel, int build_tables, int n_threads,
                        const int64_t *cand_off, const int32_t *cand, int *status);
void orc_destroy(orc_mesh *m);

/* info[0..15]: nv, nf, ne, n_table_entries, n_degenerate_faces,
 * n_voronoi_neighbour_pairs, n_inspections (flooding visits),
 * t_topology_ms, t_kdt_ms, t_voronoi_ms, t_inspection_ms, 0...
 * dom[0..6]: D lo xyz, D hi xyz, delta */
void orc_info(const orc_mesh *m, int64_t info[16], double dom[7]);

/* canonical edge list: unique (min,max) pairs sorted lexicographically */
void orc_edges(const orc_mesh *m, int32_t *E /* ne*2 */);

/* Per-query results shared by the brute force and the P2M query:
 *   dist[n], cp[n*3] closest point, ptype[n], pid[n] primitive id,
 *   bv[n*3] vertex ids of the primitive (-1 padded), bw[n*3] barycentric
 *   weights of the closest point with respect to bv.
 * second[n] (brute force only, may be NULL): the smallest distance over the
 * primitives other than the reported one (gated like the best). */
int orc_bruteforce(const orc_mesh *m, const double *q, int64_t n, int n_threads,
                   double *dist, double *cp, int32_t *ptype, int64_t *pid,
                   int32_t *bv, double *bw, double *second);

/* Alg. A.2.  use_boxes != 0 applies the Region bounding-box filter (the
 * paper searches an R-tree of these boxes; a linear scan of the same boxes
 * selects the same primitives).  nn[n] nearest vertex; cnt[n*4] per query:
 * KD-tree nodes visited, list entries scanned, edges tested, faces tested
 * (any of the optional outputs may be NULL). */
int orc_query(const orc_mesh *m, const double *q, int64_t n, int n_threads, int use_boxes,
              double *dist, double *cp, int32_t *ptype, int64_t *pid,
              int32_t *bv, double *bw, int32_t *nn, int64_t *cnt);

/* KD tree nearest vertex (ties -> lowest index) and nodes visited */
int orc_kdt_nn(const orc_mesh *m, const double *q, int64_t n, int32_t *nn, int64_t *visits);

/* interception table as CSR: off[nv+1], type[], id[], box[6*] (lo xyz, hi xyz) */
void orc_table(const orc_mesh *m, int64_t *off, int32_t *type, int32_t *id, double *box);

/* Voronoi neighbours of v (exact cell): returns count, writes up to cap ids */
int orc_cell_neighbors(const orc_mesh *m, int32_t v, int32_t *out, int cap);
/* corners of the (widened) Voronoi cell of v; returns count */
int orc_cell_corners(const orc_mesh *m, int32_t v, double *out, int cap);
/* volume of the exact (unwidened) Voronoi cell of v clipped to D */
double orc_cell_volume(const orc_mesh *m, int32_t v);

/* Single interception test of Thm. 5/6 on ConvexPoly(v,p); returns 1 if v
 * may intercept p, 0 if not, and writes the Region box (lo, hi) when 1.
 * ncorner receives the corner count of ConvexPoly(v,p) (0 = empty). */
int orc_intercepts(const orc_mesh *m, int32_t v, int32_t ptype, int32_t pid,
                   double box[6], int32_t *ncorner);

/* corners of ConvexPoly(v,p) = widened Cell(v) cut by the widened
 * Space-perp half-spaces of p; returns the corner count (0 = empty) */
int orc_convexpoly(const orc_mesh *m, int32_t v, int32_t ptype, int32_t pid, double *out, int cap);

/* Generic convex clipping used by the tests: clip the box [lo,hi] by the
 * half-spaces n.x <= c (planes: k*4 doubles) and return the corners. */
int orc_clip_box(const double lo[3], const double hi[3], const double *planes, int k,
                 double *out, int cap);

#ifdef __cplusplus
}
#endif
#endif
