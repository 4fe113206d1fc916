/*
 * p2m_oracle.c -- plain FP64 reference of the P2M method (see p2m_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg.  Nothing in the product links it.
 *
 * Layout of this file, in the order of the paper:
 *   1. mesh topology: V, E (derived, canonical order), F  (Sec. 4.1)
 *   2. gated primitive distances shared by both oracles     (Alg. A.2)
 *   3. brute force over all primitives = the plain definition
 *   4. KD tree: median split on cycled axes, NN with backtracking (Sec. 2.1)
 *   5. convex polytope cutting                               (Sec. 4.4 "Implementation")
 *   6. Voronoi cells of V clipped to the query domain D      (Sec. 4.3 Remark)
 *   7. Space-perp half-spaces of edges and faces             (Eq. 4/5, Alg. A.1)
 *   8. interception test of Thm. 5/6 + Region bounding box   (Sec. 4.4, 4.6)
 *   9. flooding inspection                                   (Alg. 1)
 *  10. query                                                 (Alg. A.2)
 *
 * Where the paper is silent the following readings are used:
 *   - the bounded domain is an explicit box D instead of the 8 virtual
 *     points of the Sec. 4.3 Remark (the virtual points can tie with a real
 *     vertex at a corner of [-M,M]^3);
 *   - every inequality errs toward keeping more: cells, Space-perp
 *     half-spaces and the Region boxes are widened by delta, and the
 *     filter of Thm. 5/6 is relaxed to |x-v|^2 - Dist^2 + eta > 0 with
 *     eta = 2*delta*diag(D) + delta^2, so a float32 query that lands a
 *     rounding error away from a cell still finds its primitive;
 *   - ties between primitives at exactly equal distance go to the lower
 *     dimension (vertex < edge < face), then to the lower id.
 */
#define _GNU_SOURCE
#include "p2m_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */

static inline double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static inline void sub3(double *r, const double *a, const double *b) {
  r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static inline void cross3(double *r, const double *a, const double *b) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double dist2(const double *a, const double *b) {
  double d[3];
  sub3(d, a, b);
  return dot3(d, d);
}
static double now_ms(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec * 1e3 + ts.tv_nsec * 1e-6;
}

/* a simple parallel-for: workers take chunks from a shared counter */
typedef struct {
  int64_t n, chunk, next;
  void (*body)(void *ctx, int64_t i, int tid);
  void *ctx;
} pfor_t;
typedef struct { pfor_t *p; int tid; } pfor_arg;

static void *pfor_worker(void *arg) {
  pfor_arg *a = (pfor_arg *)arg;
  pfor_t *p = a->p;
  for (;;) {
    int64_t s = __atomic_fetch_add(&p->next, p->chunk, __ATOMIC_RELAXED);
    if (s >= p->n) break;
    int64_t e = s + p->chunk < p->n ? s + p->chunk : p->n;
    for (int64_t i = s; i < e; ++i) p->body(p->ctx, i, a->tid);
  }
  return NULL;
}
static void parallel_for(int64_t n, int nt, int64_t chunk,
                         void (*body)(void *, int64_t, int), void *ctx) {
  pfor_t p = {n, chunk, 0, body, ctx};
  if (nt <= 1 || n < 2 * chunk) {
    for (int64_t i = 0; i < n; ++i) body(ctx, i, 0);
    return;
  }
  pthread_t th[256];
  pfor_arg args[256];
  if (nt > 256) nt = 256;
  for (int t = 0; t < nt; ++t) {
    args[t].p = &p;
    args[t].tid = t;
    pthread_create(&th[t], NULL, pfor_worker, &args[t]);
  }
  for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------ */
/* convex polytope: a list of faces, each a plane n.x <= c and a convex */
/* polygon of its corners in cyclic order (Sec. 4.4 "Implementation":   */
/* repeated cutting by half-spaces; here faces keep their polygons, so  */
/* corners and polytope edges are read off the polygons).               */
/* ------------------------------------------------------------------ */

typedef struct {
  int nf, np, fcap, pcap;
  double *pl;   /* 4 per face */
  int32_t *src; /* generator of the face: >= 0 vertex id, < 0 other */
  int32_t *fb;  /* first point of the face */
  int32_t *fc;  /* point count of the face */
  double *pt;   /* 3 per point */
} opoly;

static void poly_free(opoly *p) {
  free(p->pl); free(p->src); free(p->fb); free(p->fc); free(p->pt);
  memset(p, 0, sizeof(*p));
}
static int poly_reserve(opoly *p, int nf, int np) {
  if (nf > p->fcap) {
    int c = nf * 2 + 8;
    p->pl = (double *)realloc(p->pl, sizeof(double) * 4 * c);
    p->src = (int32_t *)realloc(p->src, sizeof(int32_t) * c);
    p->fb = (int32_t *)realloc(p->fb, sizeof(int32_t) * c);
    p->fc = (int32_t *)realloc(p->fc, sizeof(int32_t) * c);
    if (!p->pl || !p->src || !p->fb || !p->fc) return -1;
    p->fcap = c;
  }
  if (np > p->pcap) {
    int c = np * 2 + 32;
    p->pt = (double *)realloc(p->pt, sizeof(double) * 3 * c);
    if (!p->pt) return -1;
    p->pcap = c;
  }
  return 0;
}
static void poly_copy(opoly *dst, const opoly *s) {
  poly_reserve(dst, s->nf, s->np);
  dst->nf = s->nf;
  dst->np = s->np;
  memcpy(dst->pl, s->pl, sizeof(double) * 4 * s->nf);
  memcpy(dst->src, s->src, sizeof(int32_t) * s->nf);
  memcpy(dst->fb, s->fb, sizeof(int32_t) * s->nf);
  memcpy(dst->fc, s->fc, sizeof(int32_t) * s->nf);
  memcpy(dst->pt, s->pt, sizeof(double) * 3 * s->np);
}

/* axis-aligned box lo..hi as 6 faces (src -1..-6) */
static void poly_box(opoly *p, const double *lo, const double *hi) {
  poly_reserve(p, 6, 24);
  p->nf = 0;
  p->np = 0;
  for (int ax = 0; ax < 3; ++ax) {
    for (int s = 0; s < 2; ++s) {
      int f = p->nf++;
      double *pl = p->pl + 4 * f;
      pl[0] = pl[1] = pl[2] = 0.0;
      pl[ax] = s ? 1.0 : -1.0;
      pl[3] = s ? hi[ax] : -lo[ax];
      p->src[f] = -1 - f;
      p->fb[f] = p->np;
      p->fc[f] = 4;
      int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
      double u[4] = {lo[a1], hi[a1], hi[a1], lo[a1]};
      double w[4] = {lo[a2], lo[a2], hi[a2], hi[a2]};
      for (int k = 0; k < 4; ++k) {
        double *x = p->pt + 3 * p->np++;
        x[ax] = s ? hi[ax] : lo[ax];
        x[a1] = u[k];
        x[a2] = w[k];
      }
    }
  }
}

/* Cut polytope `in` by the half-space pl[0..2].x <= pl[3]; the new face
 * (if any) gets generator `src`.  Points within eps of the plane count as
 * on it.  Writes `out` (never aliasing `in`).  Returns 1 if the plane cut
 * something off, 0 if `in` was entirely inside (out = copy). */
static int poly_clip(const opoly *in, const double *pl, int src, opoly *out, double eps) {
  int any_out = 0, any_in = 0;
  for (int i = 0; i < in->np; ++i) {
    double s = dot3(pl, in->pt + 3 * i) - pl[3];
    if (s > eps) any_out = 1;
    if (s < -eps) any_in = 1;
  }
  if (!any_out) {
    poly_copy(out, in);
    return 0;
  }
  out->nf = 0;
  out->np = 0;
  if (!any_in) return 1; /* everything cut away (or flat) -> empty */

  /* cap points collected on the cutting plane */
  int ncap = 0, capcap = 64;
  double *cap = (double *)malloc(sizeof(double) * 3 * capcap);
  for (int f = 0; f < in->nf; ++f) {
    int k = in->fc[f];
    const double *P = in->pt + 3 * in->fb[f];
    poly_reserve(out, out->nf + 1, out->np + 2 * k + 2);
    int start = out->np, cnt = 0;
    for (int i = 0; i < k; ++i) {
      const double *a = P + 3 * i, *b = P + 3 * ((i + 1) % k);
      double sa = dot3(pl, a) - pl[3], sb = dot3(pl, b) - pl[3];
      if (sa <= eps) {
        memcpy(out->pt + 3 * out->np++, a, sizeof(double) * 3);
        ++cnt;
        if (sa >= -eps) {
          if (ncap + 1 > capcap) { capcap *= 2; cap = (double *)realloc(cap, sizeof(double) * 3 * capcap); }
          memcpy(cap + 3 * ncap++, a, sizeof(double) * 3);
        }
      }
      if ((sa < -eps && sb > eps) || (sa > eps && sb < -eps)) {
        double t = sa / (sa - sb), x[3];
        for (int d = 0; d < 3; ++d) x[d] = a[d] + t * (b[d] - a[d]);
        memcpy(out->pt + 3 * out->np++, x, sizeof(double) * 3);
        ++cnt;
        if (ncap + 1 > capcap) { capcap *= 2; cap = (double *)realloc(cap, sizeof(double) * 3 * capcap); }
        memcpy(cap + 3 * ncap++, x, sizeof(double) * 3);
      }
    }
    if (cnt >= 3) {
      int g = out->nf++;
      memcpy(out->pl + 4 * g, in->pl + 4 * f, sizeof(double) * 4);
      out->src[g] = in->src[f];
      out->fb[g] = start;
      out->fc[g] = cnt;
    } else {
      out->np = start;
    }
  }
  /* de-duplicate the cap points */
  int m = 0;
  double tol2 = 100.0 * eps * eps;
  for (int i = 0; i < ncap; ++i) {
    int dup = 0;
    for (int j = 0; j < m; ++j)
      if (dist2(cap + 3 * i, cap + 3 * j) <= tol2) { dup = 1; break; }
    if (!dup) {
      if (m != i) memcpy(cap + 3 * m, cap + 3 * i, sizeof(double) * 3);
      ++m;
    }
  }
  if (m >= 3) {
    /* a kept face lying in the cutting plane already closes the polytope */
    int coplanar = 0;
    for (int g = 0; g < out->nf; ++g) {
      const double *q = out->pl + 4 * g;
      if (dot3(q, pl) > 1.0 - 1e-12 && fabs(q[3] - pl[3]) <= eps) { coplanar = 1; break; }
    }
    if (!coplanar) {
      /* order the cap polygon by angle about its centroid */
      double c[3] = {0, 0, 0}, u[3], w[3], t[3] = {1, 0, 0};
      for (int i = 0; i < m; ++i)
        for (int d = 0; d < 3; ++d) c[d] += cap[3 * i + d] / m;
      if (fabs(pl[0]) > 0.6) { t[0] = 0; t[1] = 1; }
      cross3(u, pl, t);
      double un = sqrt(dot3(u, u));
      for (int d = 0; d < 3; ++d) u[d] /= un;
      cross3(w, pl, u);
      double *ang = (double *)malloc(sizeof(double) * m);
      int *ord = (int *)malloc(sizeof(int) * m);
      for (int i = 0; i < m; ++i) {
        double r[3];
        sub3(r, cap + 3 * i, c);
        ang[i] = atan2(dot3(r, w), dot3(r, u));
        ord[i] = i;
      }
      for (int i = 1; i < m; ++i) { /* insertion sort: m is small */
        int o = ord[i];
        int j = i - 1;
        while (j >= 0 && ang[ord[j]] > ang[o]) { ord[j + 1] = ord[j]; --j; }
        ord[j + 1] = o;
      }
      poly_reserve(out, out->nf + 1, out->np + m);
      int g = out->nf++;
      memcpy(out->pl + 4 * g, pl, sizeof(double) * 4);
      out->src[g] = src;
      out->fb[g] = out->np;
      out->fc[g] = m;
      for (int i = 0; i < m; ++i)
        memcpy(out->pt + 3 * out->np++, cap + 3 * ord[i], sizeof(double) * 3);
      free(ang);
      free(ord);
    }
  }
  free(cap);
  if (out->nf < 4) { out->nf = 0; out->np = 0; } /* a closed polytope has >= 4 faces */
  return 1;
}

/* volume by fanning every face polygon from the first corner */
static double poly_volume(const opoly *p) {
  if (p->nf == 0) return 0.0;
  const double *o = p->pt;
  double vol = 0.0;
  for (int f = 0; f < p->nf; ++f) {
    const double *P = p->pt + 3 * p->fb[f];
    for (int i = 1; i + 1 < p->fc[f]; ++i) {
      double a[3], b[3], c[3], x[3];
      sub3(a, P, o);
      sub3(b, P + 3 * i, o);
      sub3(c, P + 3 * (i + 1), o);
      cross3(x, b, c);
      vol += fabs(dot3(a, x)) / 6.0;
    }
  }
  return vol;
}

/* ------------------------------------------------------------------ */
/* the mesh object                                                     */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t v, type, id;
  double box[6];
} orc_rec;

struct orc_mesh {
  int64_t nv, nf, ne, ns;
  double *V;
  int32_t *F;
  int32_t *S;        /* ns*2 segments (edges of no face), may be NULL */
  int32_t *E;        /* ne*2 canonical edges */
  int32_t *fe;       /* nf*3 edge id of (F[k], F[k+1]) */
  int64_t *efo;      /* edge -> faces CSR (a segment entry holds -1) */
  int32_t *ef;
  uint8_t *fdeg;     /* 1 = zero-area face (excluded from F, edges kept) */
  int64_t ndeg;
  /* KD tree */
  int32_t *kpt, *klo, *khi;
  int8_t *kax;
  double *kbox;      /* bounding box of each subtree's points (lo xyz, hi xyz) */
  int32_t kroot;
  /* domain D and margins */
  double dlo[3], dhi[3], diag, delta, eta, eps;
  /* cells */
  opoly *cell;       /* widened cells */
  double *cvol;      /* exact cell volume */
  int64_t *nbo;
  int32_t *nb;       /* Voronoi neighbours */
  /* table */
  int64_t nt;
  int64_t *to;
  int32_t *tt, *ti;
  double *tb;
  int64_t ninspect;
  double tms[4];
  /* optional inputs of orc_create_ex */
  const int64_t *cand_off; /* nv+1: Delaunay neighbours of each vertex (CSR) */
  const int32_t *cand;     /* or NULL: k-nearest seeding + corner certification */
};

/* ------------------------------------------------------------------ */
/* 1. topology                                                          */
/* ------------------------------------------------------------------ */

typedef struct { int32_t a, b, f, k; } half_t;
static int cmp_half(const void *x, const void *y) {
  const half_t *p = (const half_t *)x, *q = (const half_t *)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  if (p->f != q->f) return p->f < q->f ? -1 : 1;
  return p->k - q->k;
}

static int cmp_vpos(const void *x, const void *y, void *ctx) {
  const double *V = (const double *)ctx;
  int32_t i = *(const int32_t *)x, j = *(const int32_t *)y;
  for (int d = 0; d < 3; ++d) {
    if (V[3 * i + d] != V[3 * j + d]) return V[3 * i + d] < V[3 * j + d] ? -1 : 1;
  }
  return i < j ? -1 : (i > j);
}

/* The edges are the unique (min, max) vertex pairs of the faces' sides and
 * of the segments; a segment that repeats a face side is that edge. */
static int build_topology(orc_mesh *m) {
  int64_t nf = m->nf, nh = 3 * m->nf + m->ns;
  half_t *h = (half_t *)malloc(sizeof(half_t) * (nh > 0 ? nh : 1));
  if (!h) return ORC_NOMEM;
  for (int64_t f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k) {
      int32_t u = m->F[3 * f + k], w = m->F[3 * f + (k + 1) % 3];
      half_t *e = h + 3 * f + k;
      e->a = u < w ? u : w;
      e->b = u < w ? w : u;
      e->f = (int32_t)f;
      e->k = k;
    }
  for (int64_t s = 0; s < m->ns; ++s) {
    int32_t u = m->S[2 * s], w = m->S[2 * s + 1];
    half_t *e = h + 3 * nf + s;
    e->a = u < w ? u : w;
    e->b = u < w ? w : u;
    e->f = -1;
    e->k = 0;
  }
  qsort(h, nh, sizeof(half_t), cmp_half);
  int64_t ne = 0;
  for (int64_t i = 0; i < nh; ++i)
    if (i == 0 || h[i].a != h[i - 1].a || h[i].b != h[i - 1].b) ++ne;
  m->ne = ne;
  m->E = (int32_t *)malloc(sizeof(int32_t) * 2 * (ne > 0 ? ne : 1));
  m->fe = (int32_t *)malloc(sizeof(int32_t) * 3 * (nf > 0 ? nf : 1));
  m->efo = (int64_t *)calloc(ne + 1, sizeof(int64_t));
  m->ef = (int32_t *)malloc(sizeof(int32_t) * (nh > 0 ? nh : 1));
  if (!m->E || !m->fe || !m->efo || !m->ef) { free(h); return ORC_NOMEM; }
  int64_t e = -1;
  for (int64_t i = 0; i < nh; ++i) {
    if (i == 0 || h[i].a != h[i - 1].a || h[i].b != h[i - 1].b) {
      ++e;
      m->E[2 * e] = h[i].a;
      m->E[2 * e + 1] = h[i].b;
    }
    if (h[i].f >= 0) m->fe[3 * h[i].f + h[i].k] = (int32_t)e;
    m->ef[i] = h[i].f;
    m->efo[e + 1] = i + 1;
  }
  free(h);
  /* zero-area faces */
  m->fdeg = (uint8_t *)calloc(nf > 0 ? nf : 1, 1);
  m->ndeg = 0;
  for (int64_t f = 0; f < nf; ++f) {
    const double *a = m->V + 3 * m->F[3 * f], *b = m->V + 3 * m->F[3 * f + 1],
                 *c = m->V + 3 * m->F[3 * f + 2];
    double e1[3], e2[3], n[3];
    sub3(e1, b, a);
    sub3(e2, c, a);
    cross3(n, e1, e2);
    double nn = dot3(n, n), s = dot3(e1, e1) * dot3(e2, e2);
    if (!(nn > 1e-24 * s) || s == 0.0) { m->fdeg[f] = 1; ++m->ndeg; }
  }
  return ORC_OK;
}

static int validate(const double *V, int64_t nv, const int32_t *F, int64_t nf,
                    const int32_t *S, int64_t ns) {
  if (nf < 0 || ns < 0 || nf + ns <= 0) return ORC_EMPTY;
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!isfinite(V[i])) return ORC_NONFINITE;
  uint8_t *used = (uint8_t *)calloc(nv > 0 ? nv : 1, 1);
  if (!used) return ORC_NOMEM;
  for (int64_t f = 0; f < nf; ++f) {
    int32_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) { free(used); return ORC_BAD_INDEX; }
    if (a == b || b == c || a == c) { free(used); return ORC_REPEATED_INDEX; }
    used[a] = used[b] = used[c] = 1;
  }
  for (int64_t s = 0; s < ns; ++s) {
    int32_t a = S[2 * s], b = S[2 * s + 1];
    if (a < 0 || b < 0 || a >= nv || b >= nv) { free(used); return ORC_BAD_INDEX; }
    if (a == b) { free(used); return ORC_REPEATED_INDEX; }
    used[a] = used[b] = 1;
  }
  for (int64_t i = 0; i < nv; ++i)
    if (!used[i]) { free(used); return ORC_UNREFERENCED; }
  free(used);
  int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * nv);
  if (!ord) return ORC_NOMEM;
  for (int64_t i = 0; i < nv; ++i) ord[i] = (int32_t)i;
  qsort_r(ord, nv, sizeof(int32_t), cmp_vpos, (void *)V);
  for (int64_t i = 1; i < nv; ++i) {
    const double *p = V + 3 * ord[i], *q = V + 3 * ord[i - 1];
    if (p[0] == q[0] && p[1] == q[1] && p[2] == q[2]) { free(ord); return ORC_DUPLICATE_VERTEX; }
  }
  free(ord);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* 2. gated primitive distances (Alg. A.2): an edge counts only if the  */
/* projection onto its line falls strictly between the endpoints, a face */
/* only if the projection onto its plane falls strictly inside it.       */
/* Both oracles call exactly these functions.                           */
/* ------------------------------------------------------------------ */

typedef struct {
  double d2;
  int32_t type;
  int64_t id;
  double cp[3];
  int32_t bv[3];
  double bw[3];
} cand_t;

static inline int cand_better(const cand_t *a, const cand_t *b) {
  if (a->d2 != b->d2) return a->d2 < b->d2;
  if (a->type != b->type) return a->type < b->type;
  return a->id < b->id;
}

static inline void cand_vertex(const orc_mesh *m, int32_t v, const double *q, cand_t *c) {
  const double *p = m->V + 3 * v;
  c->d2 = dist2(q, p);
  c->type = ORC_VERTEX;
  c->id = v;
  memcpy(c->cp, p, sizeof(double) * 3);
  c->bv[0] = v; c->bv[1] = -1; c->bv[2] = -1;
  c->bw[0] = 1.0; c->bw[1] = 0.0; c->bw[2] = 0.0;
}

/* returns 1 if the slab test passes (0 < t < 1) */
static inline int cand_edge(const orc_mesh *m, int64_t e, const double *q, cand_t *c) {
  const double *a = m->V + 3 * m->E[2 * e], *b = m->V + 3 * m->E[2 * e + 1];
  double d[3], w[3];
  sub3(d, b, a);
  sub3(w, q, a);
  double t = dot3(w, d) / dot3(d, d);
  if (!(t > 0.0 && t < 1.0)) return 0;
  for (int k = 0; k < 3; ++k) c->cp[k] = a[k] + t * d[k];
  c->d2 = dist2(q, c->cp);
  c->type = ORC_EDGE;
  c->id = e;
  c->bv[0] = m->E[2 * e]; c->bv[1] = m->E[2 * e + 1]; c->bv[2] = -1;
  c->bw[0] = 1.0 - t; c->bw[1] = t; c->bw[2] = 0.0;
  return 1;
}

/* returns 1 if the prism test passes (projection strictly inside) */
static inline int cand_face(const orc_mesh *m, int64_t f, const double *q, cand_t *c) {
  if (m->fdeg[f]) return 0;
  const int32_t *t3 = m->F + 3 * f;
  const double *a = m->V + 3 * t3[0], *b = m->V + 3 * t3[1], *cc = m->V + 3 * t3[2];
  double e1[3], e2[3], w[3];
  sub3(e1, b, a);
  sub3(e2, cc, a);
  sub3(w, q, a);
  double d00 = dot3(e1, e1), d01 = dot3(e1, e2), d11 = dot3(e2, e2);
  double d20 = dot3(w, e1), d21 = dot3(w, e2);
  double den = d00 * d11 - d01 * d01;
  double s = (d11 * d20 - d01 * d21) / den;
  double t = (d00 * d21 - d01 * d20) / den;
  if (!(s > 0.0 && t > 0.0 && s + t < 1.0)) return 0;
  for (int k = 0; k < 3; ++k) c->cp[k] = a[k] + s * e1[k] + t * e2[k];
  c->d2 = dist2(q, c->cp);
  c->type = ORC_FACE;
  c->id = f;
  c->bv[0] = t3[0]; c->bv[1] = t3[1]; c->bv[2] = t3[2];
  c->bw[0] = 1.0 - s - t; c->bw[1] = s; c->bw[2] = t;
  return 1;
}

static void cand_store(const cand_t *c, int64_t i, double *dist, double *cp, int32_t *ptype,
                       int64_t *pid, int32_t *bv, double *bw) {
  if (dist) dist[i] = sqrt(c->d2);
  if (cp) memcpy(cp + 3 * i, c->cp, sizeof(double) * 3);
  if (ptype) ptype[i] = c->type;
  if (pid) pid[i] = c->id;
  if (bv) memcpy(bv + 3 * i, c->bv, sizeof(int32_t) * 3);
  if (bw) memcpy(bw + 3 * i, c->bw, sizeof(double) * 3);
}

/* ------------------------------------------------------------------ */
/* 3. brute force: minimum over every vertex, open edge and open face   */
/* ------------------------------------------------------------------ */

typedef struct {
  const orc_mesh *m;
  const double *q;
  double *dist, *cp, *bw, *second;
  int32_t *ptype, *bv;
  int64_t *pid;
} bf_ctx;

static void bf_body(void *vctx, int64_t i, int tid) {
  (void)tid;
  bf_ctx *x = (bf_ctx *)vctx;
  const orc_mesh *m = x->m;
  const double *q = x->q + 3 * i;
  cand_t best, sec, c;
  best.d2 = sec.d2 = INFINITY;
  best.type = sec.type = 3;
  best.id = sec.id = INT64_MAX;
#define BF_OFFER()                                   \
  do {                                               \
    if (cand_better(&c, &best)) { sec = best; best = c; } \
    else if (cand_better(&c, &sec)) sec = c;         \
  } while (0)
  for (int64_t v = 0; v < m->nv; ++v) { cand_vertex(m, (int32_t)v, q, &c); BF_OFFER(); }
  for (int64_t e = 0; e < m->ne; ++e) if (cand_edge(m, e, q, &c)) BF_OFFER();
  for (int64_t f = 0; f < m->nf; ++f) if (cand_face(m, f, q, &c)) BF_OFFER();
#undef BF_OFFER
  cand_store(&best, i, x->dist, x->cp, x->ptype, x->pid, x->bv, x->bw);
  if (x->second) x->second[i] = sqrt(sec.d2);
}

int orc_bruteforce(const orc_mesh *m, const double *q, int64_t n, int n_threads,
                   double *dist, double *cp, int32_t *ptype, int64_t *pid,
                   int32_t *bv, double *bw, double *second) {
  if (!m || (!q && n)) return ORC_BAD_ARG;
  bf_ctx x = {m, q, dist, cp, bw, second, ptype, bv, pid};
  parallel_for(n, n_threads, 16, bf_body, &x);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* 4. KD tree of V: median split, split dimension cycled with depth     */
/* (Sec. 2.1); nearest neighbour by descent then unwinding.  A subtree  */
/* is skipped when the bounding box of its points is farther than the   */
/* best so far (a valid lower bound, tighter than the splitting plane   */
/* alone for queries inside closed surfaces).                           */
/* ------------------------------------------------------------------ */

typedef struct { const double *V; int axis; } kd_sort_ctx;
static int cmp_kd(const void *x, const void *y, void *ctx) {
  const kd_sort_ctx *c = (const kd_sort_ctx *)ctx;
  int32_t i = *(const int32_t *)x, j = *(const int32_t *)y;
  double a = c->V[3 * i + c->axis], b = c->V[3 * j + c->axis];
  if (a != b) return a < b ? -1 : 1;
  return i < j ? -1 : (i > j);
}

static int32_t kd_build(orc_mesh *m, int32_t *idx, int64_t n, int depth, int32_t *next) {
  if (n <= 0) return -1;
  kd_sort_ctx c = {m->V, depth % 3};
  qsort_r(idx, n, sizeof(int32_t), cmp_kd, &c);
  int64_t mid = n / 2;
  int32_t node = (*next)++;
  m->kpt[node] = idx[mid];
  m->kax[node] = (int8_t)(depth % 3);
  int32_t lo = kd_build(m, idx, mid, depth + 1, next);
  int32_t hi = kd_build(m, idx + mid + 1, n - mid - 1, depth + 1, next);
  m->klo[node] = lo;
  m->khi[node] = hi;
  double *b = m->kbox + 6 * node;
  const double *p = m->V + 3 * m->kpt[node];
  for (int d = 0; d < 3; ++d) { b[d] = p[d]; b[3 + d] = p[d]; }
  for (int c = 0; c < 2; ++c) {
    int32_t ch = c ? hi : lo;
    if (ch < 0) continue;
    const double *cb = m->kbox + 6 * ch;
    for (int d = 0; d < 3; ++d) {
      if (cb[d] < b[d]) b[d] = cb[d];
      if (cb[3 + d] > b[3 + d]) b[3 + d] = cb[3 + d];
    }
  }
  return node;
}

/* squared distance from q to the subtree box of `node` (0 inside) */
static inline double kd_box_d2(const orc_mesh *m, int32_t node, const double *q) {
  const double *b = m->kbox + 6 * node;
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    double t = q[d] < b[d] ? b[d] - q[d] : (q[d] > b[3 + d] ? q[d] - b[3 + d] : 0.0);
    s += t * t;
  }
  return s;
}

static void kd_nn_rec(const orc_mesh *m, int32_t node, const double *q, int32_t *best,
                      double *bd2, int64_t *visits) {
  if (node < 0) return;
  /* nothing in this subtree can be nearer than the best so far */
  if (kd_box_d2(m, node, q) > *bd2) return;
  ++*visits;
  int32_t p = m->kpt[node];
  double d2 = dist2(q, m->V + 3 * p);
  if (d2 < *bd2 || (d2 == *bd2 && p < *best)) { *bd2 = d2; *best = p; }
  int ax = m->kax[node];
  double diff = q[ax] - m->V[3 * p + ax];
  int32_t near = diff < 0 ? m->klo[node] : m->khi[node];
  int32_t far = diff < 0 ? m->khi[node] : m->klo[node];
  kd_nn_rec(m, near, q, best, bd2, visits);
  kd_nn_rec(m, far, q, best, bd2, visits);
}

static int32_t kd_nn(const orc_mesh *m, const double *q, int64_t *visits) {
  int32_t best = -1;
  double bd2 = INFINITY;
  int64_t v = 0;
  kd_nn_rec(m, m->kroot, q, &best, &bd2, &v);
  if (visits) *visits = v;
  return best;
}

/* nearest vertex strictly within squared distance r2 of q, or -1 */
static int32_t kd_nn_within(const orc_mesh *m, const double *q, double r2) {
  int32_t best = INT32_MAX;
  double bd2 = r2;
  int64_t v = 0;
  kd_nn_rec(m, m->kroot, q, &best, &bd2, &v);
  return (best == INT32_MAX || !(bd2 < r2)) ? -1 : best;
}

/* k nearest vertices other than `self`, sorted by distance */
static void kd_knn_rec(const orc_mesh *m, int32_t node, const double *q, int32_t self, int k,
                       int32_t *ids, double *d2s, int *cnt) {
  if (node < 0) return;
  if (*cnt == k && kd_box_d2(m, node, q) > d2s[k - 1]) return;
  int32_t p = m->kpt[node];
  if (p != self) {
    double d2 = dist2(q, m->V + 3 * p);
    if (*cnt < k || d2 < d2s[*cnt - 1]) {
      int j = *cnt < k ? (*cnt)++ : k - 1;
      while (j > 0 && d2s[j - 1] > d2) { d2s[j] = d2s[j - 1]; ids[j] = ids[j - 1]; --j; }
      d2s[j] = d2;
      ids[j] = p;
    }
  }
  int ax = m->kax[node];
  double diff = q[ax] - m->V[3 * p + ax];
  int32_t near = diff < 0 ? m->klo[node] : m->khi[node];
  int32_t far = diff < 0 ? m->khi[node] : m->klo[node];
  kd_knn_rec(m, near, q, self, k, ids, d2s, cnt);
  kd_knn_rec(m, far, q, self, k, ids, d2s, cnt);
}

/* ------------------------------------------------------------------ */
/* 6. Voronoi cell of v in V, clipped to D.                             */
/* Cell(v) is cut by the bisector half-spaces of nearby vertices until  */
/* every corner x of the polytope has no vertex strictly nearer than v: */
/* then all corners lie in the exact cell, which is convex, so the      */
/* polytope equals Cell(v) ∩ D.  The generators of the surviving        */
/* bisector faces are the Voronoi neighbours used by the flooding.      */
/* ------------------------------------------------------------------ */

static void bisector_plane(const orc_mesh *m, int32_t v, int32_t w, double widen, double *pl) {
  const double *a = m->V + 3 * v, *b = m->V + 3 * w;
  double n[3], mid[3];
  sub3(n, b, a);
  double len = sqrt(dot3(n, n));
  for (int d = 0; d < 3; ++d) { n[d] /= len; mid[d] = 0.5 * (a[d] + b[d]); }
  pl[0] = n[0]; pl[1] = n[1]; pl[2] = n[2];
  pl[3] = dot3(n, mid) + widen;
}

#define KNN_SEED 24

/* Cell(v) from a complete candidate list: the Voronoi cell of v is the
 * intersection of the bisector half-spaces of its Delaunay neighbours (every
 * other bisector is redundant), so clipping D by those alone gives it with
 * no certification.  The candidates come from a Delaunay triangulation of V
 * computed by a library (the paper's preprocessing takes its Voronoi
 * diagram from TetGen, Sec. 5; here qhull through scipy). */
static void compute_cell_from_candidates(const orc_mesh *m, int32_t v, opoly *exact,
                                         opoly *tmp) {
  poly_box(exact, m->dlo, m->dhi);
  for (int64_t j = m->cand_off[v]; j < m->cand_off[v + 1]; ++j) {
    double pl[4];
    bisector_plane(m, v, m->cand[j], 0.0, pl);
    poly_clip(exact, pl, m->cand[j], tmp, m->eps);
    poly_copy(exact, tmp);
  }
}

static void compute_cell_certified(const orc_mesh *m, int32_t v, opoly *exact, opoly *tmp) {
  const double *pv = m->V + 3 * v;
  poly_box(exact, m->dlo, m->dhi);
  int32_t ids[KNN_SEED];
  double d2s[KNN_SEED];
  int cnt = 0;
  kd_knn_rec(m, m->kroot, pv, v, KNN_SEED, ids, d2s, &cnt);
  int acap = 64, na = 0;
  int32_t *applied = (int32_t *)malloc(sizeof(int32_t) * acap);
  for (int i = 0; i < cnt; ++i) {
    double pl[4];
    bisector_plane(m, v, ids[i], 0.0, pl);
    poly_clip(exact, pl, ids[i], tmp, m->eps);
    poly_copy(exact, tmp);
    applied[na++] = ids[i];
  }
  double epsc = 1e-12 * m->diag * m->diag;
  /* every vertex outside the k-nearest set is at least r_k from v, so it
   * cannot be nearer than v to a corner closer to v than r_k / 2 */
  double safe2 = cnt == KNN_SEED ? 0.25 * d2s[KNN_SEED - 1] : INFINITY;
  for (int round = 0; round < 1000; ++round) {
    int changed = 0;
    int32_t viol[256];
    int nviol = 0;
    for (int i = 0; i < exact->np && nviol < 256; ++i) {
      const double *x = exact->pt + 3 * i;
      double r2 = dist2(x, pv);
      if (r2 <= safe2) continue;
      int32_t w = kd_nn_within(m, x, r2 - epsc);
      if (w < 0 || w == v) continue;
      {
        int seen = 0;
        for (int j = 0; j < na; ++j) if (applied[j] == w) { seen = 1; break; }
        for (int j = 0; j < nviol; ++j) if (viol[j] == w) { seen = 1; break; }
        if (!seen) viol[nviol++] = w;
      }
    }
    for (int j = 0; j < nviol; ++j) {
      double pl[4];
      bisector_plane(m, v, viol[j], 0.0, pl);
      poly_clip(exact, pl, viol[j], tmp, m->eps);
      poly_copy(exact, tmp);
      if (na + 1 > acap) { acap *= 2; applied = (int32_t *)realloc(applied, sizeof(int32_t) * acap); }
      applied[na++] = viol[j];
      changed = 1;
    }
    if (!changed) break;
  }
  free(applied);
}

static int compute_cell(const orc_mesh *m, int32_t v, opoly *exact, opoly *tmp,
                        int32_t **nbs, int *nnb) {
  if (m->cand)
    compute_cell_from_candidates(m, v, exact, tmp);
  else
    compute_cell_certified(m, v, exact, tmp);
  /* neighbours: generators of the surviving bisector faces */
  int k = 0;
  int32_t *out = (int32_t *)malloc(sizeof(int32_t) * (exact->nf + 1));
  for (int f = 0; f < exact->nf; ++f)
    if (exact->src[f] >= 0) {
      int dup = 0;
      for (int j = 0; j < k; ++j) if (out[j] == exact->src[f]) { dup = 1; break; }
      if (!dup) out[k++] = exact->src[f];
    }
  *nbs = out;
  *nnb = k;
  return 0;
}

typedef struct {
  orc_mesh *m;
  int32_t **nbs;
  int *nnb;
  opoly *scratch; /* 2 per thread */
} cell_ctx;

static void cell_body(void *vctx, int64_t i, int tid) {
  cell_ctx *x = (cell_ctx *)vctx;
  orc_mesh *m = x->m;
  opoly *ex = &x->scratch[2 * tid], *tmp = &x->scratch[2 * tid + 1];
  compute_cell(m, (int32_t)i, ex, tmp, &x->nbs[i], &x->nnb[i]);
  m->cvol[i] = poly_volume(ex);
  /* widened cell: D widened by delta, cut by the widened bisectors of the
   * Voronoi neighbours (fewer constraints -> a superset) */
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) { lo[d] = m->dlo[d] - m->delta; hi[d] = m->dhi[d] + m->delta; }
  opoly *c = &m->cell[i];
  poly_box(c, lo, hi);
  for (int j = 0; j < x->nnb[i]; ++j) {
    double pl[4];
    bisector_plane(m, (int32_t)i, x->nbs[i][j], m->delta, pl);
    poly_clip(c, pl, x->nbs[i][j], tmp, m->eps);
    poly_copy(c, tmp);
  }
}

/* ------------------------------------------------------------------ */
/* 7. Space-perp half-spaces (Eq. 4/5, Alg. A.1), widened by delta.     */
/* Face f: three planes through its edges, perpendicular to f, facing   */
/* into f.  Edge e: the two planes through its endpoints perpendicular  */
/* to e, and for every adjacent face the half-space on the far side     */
/* (away from the face) of the plane through e perpendicular to it.     */
/* ------------------------------------------------------------------ */

/* inward (into the face) unit normal of the plane through the face's edge
 * k (from F[k] to F[k+1]) that is perpendicular to the face */
static void face_edge_inward(const orc_mesh *m, int64_t f, int k, double *mm) {
  const int32_t *t = m->F + 3 * f;
  const double *a = m->V + 3 * t[0], *b = m->V + 3 * t[1], *c = m->V + 3 * t[2];
  double e1[3], e2[3], n[3], d[3];
  sub3(e1, b, a);
  sub3(e2, c, a);
  cross3(n, e1, e2);
  sub3(d, m->V + 3 * t[(k + 1) % 3], m->V + 3 * t[k]);
  cross3(mm, n, d);
  double l = sqrt(dot3(mm, mm));
  for (int i = 0; i < 3; ++i) mm[i] /= l;
}

/* writes up to 3 + (#faces) planes; returns the count */
static int perp_planes(const orc_mesh *m, int32_t type, int64_t id, double *pl, int cap) {
  int k = 0;
  if (type == ORC_FACE) {
    const int32_t *t = m->F + 3 * id;
    for (int j = 0; j < 3; ++j) {
      double mm[3];
      face_edge_inward(m, id, j, mm);
      const double *a = m->V + 3 * t[j];
      /* inside: mm.(x-a) >= 0  <=>  -mm.x <= -mm.a */
      pl[4 * k + 0] = -mm[0]; pl[4 * k + 1] = -mm[1]; pl[4 * k + 2] = -mm[2];
      pl[4 * k + 3] = -dot3(mm, a) + m->delta;
      ++k;
    }
    return k;
  }
  /* edge */
  const double *a = m->V + 3 * m->E[2 * id], *b = m->V + 3 * m->E[2 * id + 1];
  double u[3];
  sub3(u, b, a);
  double l = sqrt(dot3(u, u));
  for (int i = 0; i < 3; ++i) u[i] /= l;
  pl[0] = -u[0]; pl[1] = -u[1]; pl[2] = -u[2]; pl[3] = -dot3(u, a) + m->delta;
  pl[4] = u[0]; pl[5] = u[1]; pl[6] = u[2]; pl[7] = dot3(u, b) + m->delta;
  k = 2;
  for (int64_t j = m->efo[id]; j < m->efo[id + 1] && k < cap; ++j) {
    int64_t f = m->ef[j];
    if (f < 0 || m->fdeg[f]) continue;  /* a segment side adds no half-space */
    int le = -1;
    for (int s = 0; s < 3; ++s) if (m->fe[3 * f + s] == id) le = s;
    double mm[3];
    face_edge_inward(m, f, le, mm);
    /* away from f: mm.(x-a) <= 0 */
    pl[4 * k + 0] = mm[0]; pl[4 * k + 1] = mm[1]; pl[4 * k + 2] = mm[2];
    pl[4 * k + 3] = dot3(mm, a) + m->delta;
    ++k;
  }
  return k;
}

/* ------------------------------------------------------------------ */
/* 8. interception test on ConvexPoly(v,p) = Cell(v) ∩ Space-perp(p).   */
/* Thm. 5/6: if every corner x satisfies |x-v| <= Dist(x, l_e or pi_f)  */
/* then v cannot intercept p.  Relaxed here to g(x) = |x-v|^2 - Dist^2  */
/* + eta > 0 at some corner => keep.  Thm. 2: incident primitives are   */
/* always kept.  The Region box (Sec. 4.6) bounds ConvexPoly ∩ {g > 0}: */
/* a linear function on that set peaks at a corner with g >= 0 or where */
/* a polytope edge crosses g = 0 (g is a convex quadratic along an      */
/* edge), so those points give the exact box; it is padded by delta.    */
/* ------------------------------------------------------------------ */

typedef struct {
  int type;          /* ORC_EDGE: line through a with unit direction u; ORC_FACE: plane */
  double a[3], u[3];
} dist_prim;

static void make_dist_prim(const orc_mesh *m, int32_t type, int64_t id, dist_prim *dp) {
  dp->type = type;
  if (type == ORC_EDGE) {
    const double *a = m->V + 3 * m->E[2 * id], *b = m->V + 3 * m->E[2 * id + 1];
    memcpy(dp->a, a, sizeof(double) * 3);
    sub3(dp->u, b, a);
  } else {
    const int32_t *t = m->F + 3 * id;
    const double *a = m->V + 3 * t[0], *b = m->V + 3 * t[1], *c = m->V + 3 * t[2];
    double e1[3], e2[3];
    memcpy(dp->a, a, sizeof(double) * 3);
    sub3(e1, b, a);
    sub3(e2, c, a);
    cross3(dp->u, e1, e2);
  }
  double l = sqrt(dot3(dp->u, dp->u));
  for (int i = 0; i < 3; ++i) dp->u[i] /= l;
}

static inline double prim_dist2(const dist_prim *dp, const double *x) {
  double w[3];
  sub3(w, x, dp->a);
  double s = dot3(w, dp->u);
  if (dp->type == ORC_EDGE) return dot3(w, w) - s * s; /* Dist(x, l_e)^2 */
  return s * s;                                          /* Dist(x, pi_f)^2 */
}

static inline double gfun(const orc_mesh *m, const dist_prim *dp, const double *pv, const double *x) {
  return dist2(x, pv) - prim_dist2(dp, x) + m->eta;
}

static int incident(const orc_mesh *m, int32_t v, int32_t type, int64_t id) {
  if (type == ORC_EDGE) return m->E[2 * id] == v || m->E[2 * id + 1] == v;
  const int32_t *t = m->F + 3 * id;
  return t[0] == v || t[1] == v || t[2] == v;
}

/* returns 1 (interceptor, box written), 0 (not) */
static int intercept_test(const orc_mesh *m, int32_t v, int32_t type, int64_t id,
                          opoly *A, opoly *B, double *box, int32_t *ncorner) {
  double pl[4 * 16];
  int k = perp_planes(m, type, id, pl, 16);
  const opoly *cur = &m->cell[v];
  opoly *bufs[2] = {A, B};
  int which = 0;
  for (int j = 0; j < k; ++j) {
    poly_clip(cur, pl + 4 * j, -100 - j, bufs[which], m->eps);
    cur = bufs[which];
    which ^= 1;
    if (cur->nf == 0) break;
  }
  if (ncorner) *ncorner = cur->np;
  if (cur->nf == 0) return 0;
  dist_prim dp;
  make_dist_prim(m, type, id, &dp);
  const double *pv = m->V + 3 * v;
  int keep = incident(m, v, type, id);
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int have = 0;
#define GROW(x)                                        \
  do {                                                 \
    for (int d_ = 0; d_ < 3; ++d_) {                   \
      if ((x)[d_] < lo[d_]) lo[d_] = (x)[d_];          \
      if ((x)[d_] > hi[d_]) hi[d_] = (x)[d_];          \
    }                                                  \
    have = 1;                                          \
  } while (0)
  for (int f = 0; f < cur->nf; ++f) {
    int cn = cur->fc[f];
    const double *P = cur->pt + 3 * cur->fb[f];
    for (int i = 0; i < cn; ++i) {
      const double *x0 = P + 3 * i, *x1 = P + 3 * ((i + 1) % cn);
      double g0 = gfun(m, &dp, pv, x0), g1 = gfun(m, &dp, pv, x1);
      if (g0 > 0.0) { keep = 1; GROW(x0); }
      if ((g0 > 0.0) != (g1 > 0.0)) {
        /* g(t) along the edge is a quadratic: fit it from three samples */
        double xm[3];
        for (int d = 0; d < 3; ++d) xm[d] = 0.5 * (x0[d] + x1[d]);
        double gm = gfun(m, &dp, pv, xm);
        double qa = 2.0 * (g0 - 2.0 * gm + g1), qb = -3.0 * g0 + 4.0 * gm - g1, qc = g0;
        double roots[2];
        int nr = 0;
        if (fabs(qa) <= 1e-14 * (fabs(qb) + fabs(qc))) {
          if (qb != 0.0) roots[nr++] = -qc / qb;
        } else {
          double disc = qb * qb - 4.0 * qa * qc;
          if (disc < 0.0) disc = 0.0;
          double sq = sqrt(disc);
          double qq = -0.5 * (qb + (qb >= 0 ? sq : -sq));
          if (qq != 0.0) roots[nr++] = qc / qq;
          roots[nr++] = qq / qa;
        }
        for (int r = 0; r < nr; ++r) {
          double t = roots[r];
          if (!(t >= -1e-9 && t <= 1.0 + 1e-9)) continue;
          if (t < 0) t = 0;
          if (t > 1) t = 1;
          double xc[3];
          for (int d = 0; d < 3; ++d) xc[d] = x0[d] + t * (x1[d] - x0[d]);
          GROW(xc);
        }
      }
    }
  }
#undef GROW
  if (!keep) return 0;
  if (!have) { /* incident primitive with an empty relaxed region: box of the polytope */
    for (int i = 0; i < cur->np; ++i)
      for (int d = 0; d < 3; ++d) {
        double x = cur->pt[3 * i + d];
        if (x < lo[d]) lo[d] = x;
        if (x > hi[d]) hi[d] = x;
      }
  }
  for (int d = 0; d < 3; ++d) {
    box[d] = lo[d] - m->delta;
    box[3 + d] = hi[d] + m->delta;
  }
  return 1;
}

/* ------------------------------------------------------------------ */
/* 9. flooding inspection (Alg. 1): seeded with the primitive's         */
/* vertices, expanding to Voronoi neighbours only from interceptors;    */
/* a vertex enters the queue at most once.                              */
/* ------------------------------------------------------------------ */

typedef struct {
  orc_rec *r;
  int64_t n, cap;
  int64_t *stamp;  /* per vertex: last primitive that queued it (+1) */
  int32_t *queue;
  opoly A, B;
  int64_t inspections;
} flood_tls;

typedef struct {
  orc_mesh *m;
  flood_tls *tls;
} flood_ctx;

static void flood_body(void *vctx, int64_t i, int tid) {
  flood_ctx *x = (flood_ctx *)vctx;
  orc_mesh *m = x->m;
  flood_tls *T = &x->tls[tid];
  int32_t type;
  int64_t id;
  int32_t seeds[3];
  int ns;
  if (i < m->ne) {
    type = ORC_EDGE;
    id = i;
    seeds[0] = m->E[2 * id];
    seeds[1] = m->E[2 * id + 1];
    ns = 2;
  } else {
    type = ORC_FACE;
    id = i - m->ne;
    if (m->fdeg[id]) return;
    memcpy(seeds, m->F + 3 * id, sizeof(int32_t) * 3);
    ns = 3;
  }
  int64_t mark = i + 1;
  int64_t head = 0, tail = 0;
  for (int s = 0; s < ns; ++s) {
    T->stamp[seeds[s]] = mark;
    T->queue[tail++] = seeds[s];
  }
  while (head < tail) {
    int32_t v = T->queue[head++];
    double box[6];
    ++T->inspections;
    if (!intercept_test(m, v, type, id, &T->A, &T->B, box, NULL)) continue;
    if (T->n == T->cap) {
      T->cap = T->cap ? 2 * T->cap : 1024;
      T->r = (orc_rec *)realloc(T->r, sizeof(orc_rec) * T->cap);
    }
    orc_rec *r = &T->r[T->n++];
    r->v = v;
    r->type = type;
    r->id = (int32_t)id;
    memcpy(r->box, box, sizeof(box));
    for (int64_t j = m->nbo[v]; j < m->nbo[v + 1]; ++j) {
      int32_t w = m->nb[j];
      if (T->stamp[w] != mark) {
        T->stamp[w] = mark;
        T->queue[tail++] = w;
      }
    }
  }
}

static int cmp_rec_in_row(const void *x, const void *y) {
  const orc_rec *a = (const orc_rec *)x, *b = (const orc_rec *)y;
  if (a->type != b->type) return a->type - b->type;
  return (a->id > b->id) - (a->id < b->id);
}

/* ------------------------------------------------------------------ */
/* construction                                                         */
/* ------------------------------------------------------------------ */

orc_mesh *orc_create(const double *V, int64_t nv, const int32_t *F, int64_t nf,
                     double domain_scale, double domain_margin, double delta_rel,
                     int build_tables, int n_threads, int *status) {
  return orc_create_mixed(V, nv, F, nf, NULL, 0, domain_scale, domain_margin, delta_rel,
                          build_tables, n_threads, status);
}

orc_mesh *orc_create_mixed(const double *V, int64_t nv, const int32_t *F, int64_t nf,
                           const int32_t *S, int64_t ns, double domain_scale,
                           double domain_margin, double delta_rel, int build_tables,
                           int n_threads, int *status) {
  return orc_create_ex(V, nv, F, nf, S, ns, domain_scale, domain_margin, delta_rel,
                       build_tables, n_threads, NULL, NULL, status);
}

orc_mesh *orc_create_ex(const double *V, int64_t nv, const int32_t *F, int64_t nf,
                        const int32_t *S, int64_t ns, double domain_scale, double domain_margin,
                        double delta_rel, int build_tables, int n_threads,
                        const int64_t *cand_off, const int32_t *cand, int *status) {
  int st = (!V || nv <= 0 || (nf > 0 && !F) || (ns > 0 && !S) || (!cand_off != !cand))
               ? ORC_BAD_ARG
               : validate(V, nv, F, nf, S, ns);
  if (!st && cand) {
    if (cand_off[0] != 0) st = ORC_BAD_ARG;
    for (int64_t i = 0; i < nv && !st; ++i)
      if (cand_off[i + 1] < cand_off[i]) st = ORC_BAD_ARG;
    for (int64_t j = 0; !st && j < cand_off[nv]; ++j)
      if (cand[j] < 0 || cand[j] >= nv) st = ORC_BAD_INDEX;
    for (int64_t i = 0; i < nv && !st; ++i)
      for (int64_t j = cand_off[i]; j < cand_off[i + 1]; ++j)
        if (cand[j] == (int32_t)i) st = ORC_BAD_ARG;
  }
  if (st) { if (status) *status = st; return NULL; }
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
  m->cand_off = cand_off;
  m->cand = cand;
  m->nv = nv;
  m->nf = nf;
  m->ns = ns;
  m->V = (double *)malloc(sizeof(double) * 3 * nv);
  m->F = (int32_t *)malloc(sizeof(int32_t) * 3 * (nf > 0 ? nf : 1));
  m->S = (int32_t *)malloc(sizeof(int32_t) * 2 * (ns > 0 ? ns : 1));
  memcpy(m->V, V, sizeof(double) * 3 * nv);
  if (nf > 0) memcpy(m->F, F, sizeof(int32_t) * 3 * nf);
  if (ns > 0) memcpy(m->S, S, sizeof(int32_t) * 2 * ns);
  if (n_threads < 1) n_threads = 1;

  double t0 = now_ms();
  if ((st = build_topology(m))) { orc_destroy(m); if (status) *status = st; return NULL; }
  double t1 = now_ms();

  /* domain D */
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
  for (int64_t i = 0; i < nv; ++i)
    for (int d = 0; d < 3; ++d) {
      double x = V[3 * i + d];
      if (x < lo[d]) lo[d] = x;
      if (x > hi[d]) hi[d] = x;
    }
  double bd = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                   (hi[2] - lo[2]) * (hi[2] - lo[2]));
  for (int d = 0; d < 3; ++d) {
    double c = 0.5 * (lo[d] + hi[d]), h = 0.5 * (hi[d] - lo[d]) * domain_scale + domain_margin * bd;
    if (h <= 0) h = domain_margin > 0 ? domain_margin * bd : 1e-3 * bd;
    m->dlo[d] = c - h;
    m->dhi[d] = c + h;
  }
  m->diag = sqrt((m->dhi[0] - m->dlo[0]) * (m->dhi[0] - m->dlo[0]) +
                 (m->dhi[1] - m->dlo[1]) * (m->dhi[1] - m->dlo[1]) +
                 (m->dhi[2] - m->dlo[2]) * (m->dhi[2] - m->dlo[2]));
  m->delta = delta_rel * m->diag;
  m->eta = 2.0 * m->delta * m->diag + m->delta * m->delta;
  m->eps = 1e-13 * m->diag;

  /* KD tree */
  m->kpt = (int32_t *)malloc(sizeof(int32_t) * nv);
  m->klo = (int32_t *)malloc(sizeof(int32_t) * nv);
  m->khi = (int32_t *)malloc(sizeof(int32_t) * nv);
  m->kax = (int8_t *)malloc(nv);
  m->kbox = (double *)malloc(sizeof(double) * 6 * nv);
  int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * nv);
  for (int64_t i = 0; i < nv; ++i) idx[i] = (int32_t)i;
  int32_t next = 0;
  m->kroot = kd_build(m, idx, nv, 0, &next);
  free(idx);
  double t2 = now_ms();
  m->tms[0] = t1 - t0;
  m->tms[1] = t2 - t1;
  if (!build_tables) { if (status) *status = ORC_OK; return m; }

  /* Voronoi cells */
  m->cell = (opoly *)calloc(nv, sizeof(opoly));
  m->cvol = (double *)calloc(nv, sizeof(double));
  int32_t **nbs = (int32_t **)calloc(nv, sizeof(int32_t *));
  int *nnb = (int *)calloc(nv, sizeof(int));
  opoly *scratch = (opoly *)calloc(2 * n_threads, sizeof(opoly));
  cell_ctx cc = {m, nbs, nnb, scratch};
  parallel_for(nv, n_threads, 64, cell_body, &cc);
  for (int i = 0; i < 2 * n_threads; ++i) poly_free(&scratch[i]);
  free(scratch);
  m->nbo = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
  m->nbo[0] = 0;
  for (int64_t i = 0; i < nv; ++i) m->nbo[i + 1] = m->nbo[i] + nnb[i];
  m->nb = (int32_t *)malloc(sizeof(int32_t) * (m->nbo[nv] + 1));
  for (int64_t i = 0; i < nv; ++i) {
    memcpy(m->nb + m->nbo[i], nbs[i], sizeof(int32_t) * nnb[i]);
    free(nbs[i]);
  }
  free(nbs);
  free(nnb);
  m->cand_off = NULL; /* borrowed from the caller for the cell stage only */
  m->cand = NULL;
  double t3 = now_ms();

  /* flooding inspection over every edge and every face */
  flood_tls *tls = (flood_tls *)calloc(n_threads, sizeof(flood_tls));
  for (int t = 0; t < n_threads; ++t) {
    tls[t].stamp = (int64_t *)calloc(nv, sizeof(int64_t));
    tls[t].queue = (int32_t *)malloc(sizeof(int32_t) * (nv + 3));
  }
  flood_ctx fc = {m, tls};
  parallel_for(m->ne + m->nf, n_threads, 32, flood_body, &fc);
  int64_t total = 0;
  m->ninspect = 0;
  for (int t = 0; t < n_threads; ++t) { total += tls[t].n; m->ninspect += tls[t].inspections; }
  /* bucket by vertex, sort each row by (type, id) */
  m->nt = total;
  m->to = (int64_t *)calloc(nv + 1, sizeof(int64_t));
  for (int t = 0; t < n_threads; ++t)
    for (int64_t i = 0; i < tls[t].n; ++i) m->to[tls[t].r[i].v + 1]++;
  for (int64_t i = 0; i < nv; ++i) m->to[i + 1] += m->to[i];
  orc_rec *all = (orc_rec *)malloc(sizeof(orc_rec) * (total + 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nv + 1));
  memcpy(fill, m->to, sizeof(int64_t) * (nv + 1));
  for (int t = 0; t < n_threads; ++t) {
    for (int64_t i = 0; i < tls[t].n; ++i) all[fill[tls[t].r[i].v]++] = tls[t].r[i];
    free(tls[t].r);
    free(tls[t].stamp);
    free(tls[t].queue);
    poly_free(&tls[t].A);
    poly_free(&tls[t].B);
  }
  free(tls);
  free(fill);
  for (int64_t v = 0; v < nv; ++v)
    qsort(all + m->to[v], m->to[v + 1] - m->to[v], sizeof(orc_rec), cmp_rec_in_row);
  m->tt = (int32_t *)malloc(sizeof(int32_t) * (total + 1));
  m->ti = (int32_t *)malloc(sizeof(int32_t) * (total + 1));
  m->tb = (double *)malloc(sizeof(double) * 6 * (total + 1));
  for (int64_t i = 0; i < total; ++i) {
    m->tt[i] = all[i].type;
    m->ti[i] = all[i].id;
    memcpy(m->tb + 6 * i, all[i].box, sizeof(double) * 6);
  }
  free(all);
  double t4 = now_ms();
  m->tms[2] = t3 - t2;
  m->tms[3] = t4 - t3;
  if (status) *status = ORC_OK;
  return m;
}

void orc_destroy(orc_mesh *m) {
  if (!m) return;
  if (m->cell) {
    for (int64_t i = 0; i < m->nv; ++i) poly_free(&m->cell[i]);
    free(m->cell);
  }
  free(m->V); free(m->F); free(m->S); free(m->E); free(m->fe); free(m->efo); free(m->ef); free(m->fdeg);
  free(m->kpt); free(m->klo); free(m->khi); free(m->kax); free(m->kbox);
  free(m->cvol); free(m->nbo); free(m->nb);
  free(m->to); free(m->tt); free(m->ti); free(m->tb);
  free(m);
}

void orc_info(const orc_mesh *m, int64_t info[16], double dom[7]) {
  memset(info, 0, sizeof(int64_t) * 16);
  info[0] = m->nv;
  info[1] = m->nf;
  info[2] = m->ne;
  info[3] = m->nt;
  info[4] = m->ndeg;
  info[5] = m->nbo ? m->nbo[m->nv] : 0;
  info[6] = m->ninspect;
  for (int i = 0; i < 4; ++i) info[7 + i] = (int64_t)(m->tms[i] + 0.5);
  if (dom) {
    for (int d = 0; d < 3; ++d) { dom[d] = m->dlo[d]; dom[3 + d] = m->dhi[d]; }
    dom[6] = m->delta;
  }
}

void orc_edges(const orc_mesh *m, int32_t *E) { memcpy(E, m->E, sizeof(int32_t) * 2 * m->ne); }

void orc_table(const orc_mesh *m, int64_t *off, int32_t *type, int32_t *id, double *box) {
  if (!m->to) return;
  if (off) memcpy(off, m->to, sizeof(int64_t) * (m->nv + 1));
  if (type) memcpy(type, m->tt, sizeof(int32_t) * m->nt);
  if (id) memcpy(id, m->ti, sizeof(int32_t) * m->nt);
  if (box) memcpy(box, m->tb, sizeof(double) * 6 * m->nt);
}

int orc_cell_neighbors(const orc_mesh *m, int32_t v, int32_t *out, int cap) {
  if (!m->nbo || v < 0 || v >= m->nv) return -1;
  int k = (int)(m->nbo[v + 1] - m->nbo[v]);
  for (int i = 0; i < k && i < cap; ++i) out[i] = m->nb[m->nbo[v] + i];
  return k;
}

int orc_cell_corners(const orc_mesh *m, int32_t v, double *out, int cap) {
  if (!m->cell || v < 0 || v >= m->nv) return -1;
  const opoly *c = &m->cell[v];
  for (int i = 0; i < c->np && i < cap; ++i) memcpy(out + 3 * i, c->pt + 3 * i, sizeof(double) * 3);
  return c->np;
}

double orc_cell_volume(const orc_mesh *m, int32_t v) {
  if (!m->cvol || v < 0 || v >= m->nv) return -1.0;
  return m->cvol[v];
}

int orc_intercepts(const orc_mesh *m, int32_t v, int32_t ptype, int32_t pid, double box[6],
                   int32_t *ncorner) {
  if (!m->cell) return -1;
  opoly A = {0}, B = {0};
  int r = intercept_test(m, v, ptype, pid, &A, &B, box, ncorner);
  poly_free(&A);
  poly_free(&B);
  return r;
}

int orc_convexpoly(const orc_mesh *m, int32_t v, int32_t ptype, int32_t pid, double *out, int cap) {
  if (!m->cell) return -1;
  double pl[4 * 16];
  int k = perp_planes(m, ptype, pid, pl, 16);
  opoly A = {0}, B = {0};
  poly_copy(&A, &m->cell[v]);
  for (int j = 0; j < k && A.nf; ++j) {
    poly_clip(&A, pl + 4 * j, -100 - j, &B, m->eps);
    poly_copy(&A, &B);
  }
  int n = A.nf ? A.np : 0;
  for (int i = 0; i < n && i < cap; ++i) memcpy(out + 3 * i, A.pt + 3 * i, sizeof(double) * 3);
  poly_free(&A);
  poly_free(&B);
  return n;
}

int orc_clip_box(const double lo[3], const double hi[3], const double *planes, int k,
                 double *out, int cap) {
  opoly P = {0}, Q = {0};
  poly_box(&P, lo, hi);
  double diag = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                     (hi[2] - lo[2]) * (hi[2] - lo[2]));
  for (int j = 0; j < k; ++j) {
    poly_clip(&P, planes + 4 * j, j, &Q, 1e-13 * diag);
    poly_copy(&P, &Q);
  }
  int n = P.np;
  for (int i = 0; i < n && i < cap; ++i) memcpy(out + 3 * i, P.pt + 3 * i, sizeof(double) * 3);
  poly_free(&P);
  poly_free(&Q);
  return n;
}

/* ------------------------------------------------------------------ */
/* 10. query (Alg. A.2): nearest vertex by the KD tree, d_min = d(q,v), */
/* then every primitive of v's interception list (optionally only those */
/* whose Region box contains q): an edge through the slab test and the  */
/* distance to its line, a face through the prism test and the distance */
/* to its plane; keep the minimum.                                      */
/* ------------------------------------------------------------------ */

typedef struct {
  const orc_mesh *m;
  const double *q;
  int use_boxes;
  double *dist, *cp, *bw;
  int32_t *ptype, *bv, *nn;
  int64_t *pid, *cnt;
} q_ctx;

static void query_body(void *vctx, int64_t i, int tid) {
  (void)tid;
  q_ctx *x = (q_ctx *)vctx;
  const orc_mesh *m = x->m;
  const double *q = x->q + 3 * i;
  int64_t visits = 0, scanned = 0, te = 0, tf = 0;
  int32_t v = kd_nn(m, q, &visits);
  cand_t best, c;
  cand_vertex(m, v, q, &best);
  for (int64_t j = m->to[v]; j < m->to[v + 1]; ++j) {
    ++scanned;
    if (x->use_boxes) {
      const double *b = m->tb + 6 * j;
      if (q[0] < b[0] || q[1] < b[1] || q[2] < b[2] || q[0] > b[3] || q[1] > b[4] || q[2] > b[5])
        continue;
    }
    if (m->tt[j] == ORC_EDGE) {
      ++te;
      if (cand_edge(m, m->ti[j], q, &c) && cand_better(&c, &best)) best = c;
    } else {
      ++tf;
      if (cand_face(m, m->ti[j], q, &c) && cand_better(&c, &best)) best = c;
    }
  }
  cand_store(&best, i, x->dist, x->cp, x->ptype, x->pid, x->bv, x->bw);
  if (x->nn) x->nn[i] = v;
  if (x->cnt) {
    x->cnt[4 * i + 0] = visits;
    x->cnt[4 * i + 1] = scanned;
    x->cnt[4 * i + 2] = te;
    x->cnt[4 * i + 3] = tf;
  }
}

int orc_query(const orc_mesh *m, const double *q, int64_t n, int n_threads, int use_boxes,
              double *dist, double *cp, int32_t *ptype, int64_t *pid,
              int32_t *bv, double *bw, int32_t *nn, int64_t *cnt) {
  if (!m || !m->to || (!q && n)) return ORC_BAD_ARG;
  q_ctx x = {m, q, use_boxes, dist, cp, bw, ptype, bv, nn, pid, cnt};
  parallel_for(n, n_threads, 256, query_body, &x);
  return ORC_OK;
}

typedef struct { const orc_mesh *m; const double *q; int32_t *nn; int64_t *visits; } nn_ctx;
static void nn_body(void *vctx, int64_t i, int tid) {
  (void)tid;
  nn_ctx *x = (nn_ctx *)vctx;
  int64_t v = 0;
  x->nn[i] = kd_nn(x->m, x->q + 3 * i, &v);
  if (x->visits) x->visits[i] = v;
}
int orc_kdt_nn(const orc_mesh *m, const double *q, int64_t n, int32_t *nn, int64_t *visits) {
  if (!m || !nn) return ORC_BAD_ARG;
  nn_ctx x = {m, q, nn, visits};
  parallel_for(n, 1, 256, nn_body, &x);
  return ORC_OK;
}
