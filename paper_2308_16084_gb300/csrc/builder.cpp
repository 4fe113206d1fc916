// builder.cpp -- host preprocessing of the P2M query layout (Alg. A.1).
//
//   topology -> KD tree of V -> Voronoi cells of V clipped to D (k-nearest
//   seeding, then rounds of corner certification) -> flooding interception
//   inspection per edge and face (Alg. 1) with the convexity filter of
//   Thm. 5/6 -> Region boxes (Sec. 4.6) -> packed float32 layout.
//
// Every approximation errs toward a larger table: cells, Space-perp
// half-spaces and Region boxes are widened by delta, and the filter keeps a
// pair when |x-v|^2 - Dist(x)^2 + eta > 0 at some corner x of ConvexPoly,
// eta = 2 delta diag(D) + delta^2.  A float32 query that a rounding error
// puts just outside the exact cell of its nearest vertex therefore still
// finds its primitive in the list of the vertex the kernel picks.
#include "builder.h"
#include "flood_core.h"
#include "flood_warp.h"
#include "pack.h"
#include "quant.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <limits>
#include <memory>
#include <mutex>
#include <string>
#include <thread>

namespace p2m {
namespace {

// ---------------------------------------------------------------- vectors
// double-precision 3-vectors and their operations: the ones the flooding
// core shares with the device (flood_core.h)
using V3 = fc::D3;
using fc::cross;
using fc::dot;
using fc::len2;
using fc::lex_less;

// half-space n.x <= c, with the id of whatever generated it
struct Plane {
  V3 n;
  double c;
  int32_t src;
};

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// fn(i, thread) for i in [0, n) on `threads` threads, chunk items at a time.
// An exception thrown by fn (std::bad_alloc on a worker, say) stops the
// other workers at their next chunk and is rethrown here once all joined.
template <class F>
void parallel_for(int64_t n, int threads, int64_t chunk, F &&fn) {
  if (threads <= 1 || n <= chunk) {
    for (int64_t i = 0; i < n; ++i) fn(i, 0);
    return;
  }
  std::atomic<int64_t> next{0};
  std::exception_ptr failure;
  std::mutex failure_mu;
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&, t] {
      for (;;) {
        int64_t s = next.fetch_add(chunk);
        if (s >= n) break;
        int64_t e = std::min(n, s + chunk);
        try {
          for (int64_t i = s; i < e; ++i) fn(i, t);
        } catch (...) {
          std::lock_guard<std::mutex> g(failure_mu);
          if (!failure) failure = std::current_exception();
          next.store(n);
          break;
        }
      }
    });
  for (auto &th : pool) th.join();
  if (failure) std::rethrow_exception(failure);
}

// Host-side fault injection for tests: P2M_INJECT_BAD_ALLOC=<stage> makes a
// worker of that build stage ("cells", "flooding" or "packing") throw
// std::bad_alloc, as a failed allocation would.
bool inject_at(const char *stage) {
  const char *v = std::getenv("P2M_INJECT_BAD_ALLOC");
  return v && std::strcmp(v, stage) == 0;
}

// ------------------------------------------------------------- polytope
// Convex polytope as faces; every face keeps its plane and the loop of its
// corners, counter-clockwise seen from outside.  Cutting by a half-space
// clips every loop and closes the hole with a cap face whose loop is
// chained from the per-face exit/entry points, so corners shared by faces
// are produced bit-identically from both sides.
struct Poly {
  std::vector<Plane> pl;
  std::vector<int32_t> beg{0};  // loop of face f: pt[beg[f] .. beg[f+1])
  std::vector<V3> pt;
  void clear() {
    pl.clear();
    beg.assign(1, 0);
    pt.clear();
  }
  bool empty() const { return pl.empty(); }
  int nf() const { return (int)pl.size(); }
};

struct CutScratch {
  std::vector<double> s;
  std::vector<V3> seg_in, seg_out;
  std::vector<char> used;
};

void make_box(Poly &p, const double lo[3], const double hi[3]) {
  p.clear();
  auto face = [&](V3 n, double c, int src, V3 a, V3 b, V3 cc, V3 d) {
    p.pl.push_back({n, c, src});
    p.pt.push_back(a);
    p.pt.push_back(b);
    p.pt.push_back(cc);
    p.pt.push_back(d);
    p.beg.push_back((int32_t)p.pt.size());
  };
  double X0 = lo[0], Y0 = lo[1], Z0 = lo[2], X1 = hi[0], Y1 = hi[1], Z1 = hi[2];
  face({1, 0, 0}, X1, -1, {X1, Y0, Z0}, {X1, Y1, Z0}, {X1, Y1, Z1}, {X1, Y0, Z1});
  face({-1, 0, 0}, -X0, -2, {X0, Y0, Z0}, {X0, Y0, Z1}, {X0, Y1, Z1}, {X0, Y1, Z0});
  face({0, 1, 0}, Y1, -3, {X0, Y1, Z0}, {X0, Y1, Z1}, {X1, Y1, Z1}, {X1, Y1, Z0});
  face({0, -1, 0}, -Y0, -4, {X0, Y0, Z0}, {X1, Y0, Z0}, {X1, Y0, Z1}, {X0, Y0, Z1});
  face({0, 0, 1}, Z1, -5, {X0, Y0, Z1}, {X1, Y0, Z1}, {X1, Y1, Z1}, {X0, Y1, Z1});
  face({0, 0, -1}, -Z0, -6, {X0, Y0, Z0}, {X0, Y1, Z0}, {X1, Y1, Z0}, {X1, Y0, Z0});
}

using fc::crossing;

// Cut `in` by h into `out`.  Returns false (and leaves out untouched) when
// nothing lies beyond h.  An emptied polytope comes back with no faces.
bool cut(const Poly &in, const Plane &h, double eps, Poly &out, CutScratch &S) {
  const size_t np = in.pt.size();
  S.s.resize(np);
  bool beyond = false, within = false;
  for (size_t i = 0; i < np; ++i) {
    double s = dot(h.n, in.pt[i]) - h.c;
    S.s[i] = s;
    beyond |= s > eps;
    within |= s < -eps;
  }
  if (!beyond) return false;
  out.clear();
  if (!within) return true;
  S.seg_in.clear();
  S.seg_out.clear();
  for (int f = 0; f < in.nf(); ++f) {
    const int b = in.beg[f], k = in.beg[f + 1] - b;
    const size_t start = out.pt.size();
    bool has_x = false, has_y = false;
    V3 X{0, 0, 0}, Y{0, 0, 0};
    for (int i = 0; i < k; ++i) {
      const int ia = b + i, ib = b + (i + 1) % k;
      const double sa = S.s[ia], sb = S.s[ib];
      const bool ka = sa <= eps, kb = sb <= eps;
      if (ka) out.pt.push_back(in.pt[ia]);
      if (ka && !kb) {  // leaving the kept side
        if (sa >= -eps) {
          X = in.pt[ia];
        } else {
          X = crossing(in.pt[ia], in.pt[ib], sa, sb);
          out.pt.push_back(X);
        }
        has_x = true;
      } else if (!ka && kb) {  // coming back
        if (sb >= -eps) {
          Y = in.pt[ib];
        } else {
          Y = crossing(in.pt[ia], in.pt[ib], sa, sb);
          out.pt.push_back(Y);
        }
        has_y = true;
      }
    }
    if (out.pt.size() - start >= 3) {
      out.pl.push_back(in.pl[f]);
      out.beg.push_back((int32_t)out.pt.size());
    } else {
      out.pt.resize(start);
    }
    if (has_x && has_y && len2(X - Y) > eps * eps) {
      S.seg_in.push_back(Y);
      S.seg_out.push_back(X);
    }
  }
  // chain the cap loop: the face walks X -> Y along h, the cap walks Y -> X
  const int m = (int)S.seg_in.size();
  if (m >= 3) {
    S.used.assign(m, 0);
    const size_t start = out.pt.size();
    out.pt.push_back(S.seg_in[0]);
    V3 cur = S.seg_out[0];
    S.used[0] = 1;
    bool ok = true;
    for (int step = 1; step < m; ++step) {
      out.pt.push_back(cur);
      int best = -1;
      double bd = std::numeric_limits<double>::infinity();
      for (int j = 0; j < m; ++j)
        if (!S.used[j]) {
          double d = len2(S.seg_in[j] - cur);
          if (d < bd) {
            bd = d;
            best = j;
          }
        }
      if (best < 0 || bd > 1e6 * eps * eps) {
        ok = false;
        break;
      }
      S.used[best] = 1;
      cur = S.seg_out[best];
    }
    if (ok && len2(cur - S.seg_in[0]) <= 1e6 * eps * eps) {
      out.pl.push_back(h);
      out.beg.push_back((int32_t)out.pt.size());
    } else {
      // fall back: order the distinct cap points by angle in the plane
      out.pt.resize(start);
      std::vector<V3> q;
      for (int j = 0; j < m; ++j)
        for (V3 p : {S.seg_in[j], S.seg_out[j]}) {
          bool dup = false;
          for (V3 r : q) dup |= len2(r - p) <= 1e6 * eps * eps;
          if (!dup) q.push_back(p);
        }
      if (q.size() >= 3) {
        V3 c{0, 0, 0};
        for (V3 p : q) c = c + (1.0 / q.size()) * p;
        V3 t = std::fabs(h.n.x) < 0.6 ? V3{1, 0, 0} : V3{0, 1, 0};
        V3 u = cross(h.n, t);
        u = (1.0 / std::sqrt(len2(u))) * u;
        V3 w = cross(h.n, u);
        std::sort(q.begin(), q.end(), [&](V3 a, V3 b) {
          return std::atan2(dot(a - c, w), dot(a - c, u)) < std::atan2(dot(b - c, w), dot(b - c, u));
        });
        for (V3 p : q) out.pt.push_back(p);
        out.pl.push_back(h);
        out.beg.push_back((int32_t)out.pt.size());
      }
    }
  }
  if (out.nf() < 4) out.clear();
  return true;
}

// ---------------------------------------------------------------- mesh
struct Mesh {
  int64_t nv = 0, nf = 0, ne = 0;
  std::vector<V3> V;
  std::vector<int32_t> F;       // nf * 3
  std::vector<int32_t> E;       // ne * 2
  std::vector<int32_t> fedge;   // nf * 3, edge of (F[k], F[k+1])
  std::vector<int64_t> ef_off;  // ne + 1
  std::vector<int32_t> ef;      // edge -> faces
  std::vector<uint8_t> degenerate;
};

int validate(const float *V, int64_t nv, const int32_t *F, int64_t nf, const int32_t *S,
             int64_t ns, std::string &err) {
  if (nf < 0 || ns < 0 || nf + ns <= 0 || nv < 2) {
    err = "mesh has no triangles and no segments";
    return 2;
  }
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(V[i])) {
      err = "non-finite vertex coordinate";
      return 2;
    }
  std::vector<uint8_t> used(nv, 0);
  for (int64_t f = 0; f < nf; ++f) {
    int32_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
      err = "triangle index out of range";
      return 2;
    }
    if (a == b || b == c || a == c) {
      err = "triangle repeats a vertex";
      return 2;
    }
    used[a] = used[b] = used[c] = 1;
  }
  for (int64_t s = 0; s < ns; ++s) {
    int32_t a = S[2 * s], b = S[2 * s + 1];
    if (a < 0 || b < 0 || a >= nv || b >= nv) {
      err = "segment index out of range";
      return 2;
    }
    if (a == b) {
      err = "segment repeats a vertex";
      return 2;
    }
    used[a] = used[b] = 1;
  }
  for (int64_t i = 0; i < nv; ++i)
    if (!used[i]) {
      err = "vertex referenced by no triangle or segment";
      return 2;
    }
  std::vector<int32_t> ord(nv);
  for (int64_t i = 0; i < nv; ++i) ord[i] = (int32_t)i;
  std::sort(ord.begin(), ord.end(), [&](int32_t i, int32_t j) {
    return std::memcmp(V + 3 * i, V + 3 * j, 12) < 0 ||
           (std::memcmp(V + 3 * i, V + 3 * j, 12) == 0 && i < j);
  });
  for (int64_t i = 1; i < nv; ++i) {
    const float *p = V + 3 * ord[i], *q = V + 3 * ord[i - 1];
    if (p[0] == q[0] && p[1] == q[1] && p[2] == q[2]) {
      err = "duplicate vertex position";
      return 3;
    }
  }
  return 0;
}

// Edges: the unique (min, max) vertex pairs of the face sides and of the
// segments (Sec. 5, mixed primitives); a segment that repeats a face side
// is that edge.  Segment sides enter the edge -> faces lists as face -1.
void build_topology(Mesh &M, const int32_t *S, int64_t ns) {
  struct HalfEdge {
    int64_t key;  // min << 32 | max
    int32_t face;
    int32_t k;
  };
  std::vector<HalfEdge> h(3 * M.nf + ns);
  for (int64_t f = 0; f < M.nf; ++f)
    for (int k = 0; k < 3; ++k) {
      int64_t u = M.F[3 * f + k], w = M.F[3 * f + (k + 1) % 3];
      h[3 * f + k] = {std::min(u, w) << 32 | std::max(u, w), (int32_t)f, k};
    }
  for (int64_t s = 0; s < ns; ++s) {
    int64_t u = S[2 * s], w = S[2 * s + 1];
    h[3 * M.nf + s] = {std::min(u, w) << 32 | std::max(u, w), -1, 0};
  }
  std::sort(h.begin(), h.end(), [](const HalfEdge &a, const HalfEdge &b) {
    return a.key < b.key || (a.key == b.key && a.face < b.face);
  });
  M.fedge.assign(3 * M.nf, -1);
  M.E.clear();
  M.ef_off.assign(1, 0);
  M.ef.resize(h.size());
  for (size_t i = 0; i < h.size(); ++i) {
    if (i == 0 || h[i].key != h[i - 1].key) {
      M.E.push_back((int32_t)(h[i].key >> 32));
      M.E.push_back((int32_t)(h[i].key & 0xffffffff));
      M.ef_off.push_back(M.ef_off.back());
    }
    if (h[i].face >= 0) M.fedge[3 * h[i].face + h[i].k] = (int32_t)(M.E.size() / 2 - 1);
    M.ef[i] = h[i].face;
    M.ef_off.back()++;
  }
  M.ne = (int64_t)M.E.size() / 2;
  M.degenerate.assign(M.nf, 0);
  for (int64_t f = 0; f < M.nf; ++f) {
    V3 a = M.V[M.F[3 * f]], b = M.V[M.F[3 * f + 1]], c = M.V[M.F[3 * f + 2]];
    V3 e1 = b - a, e2 = c - a;
    double s = len2(e1) * len2(e2);
    if (!(len2(cross(e1, e2)) > 1e-24 * s)) M.degenerate[f] = 1;
  }
}

// -------------------------------------------------------------- KD tree
// Perfect binary tree with L = 2^depth leaves; heap order; leaf j holds the
// tree positions [j*n/L, (j+1)*n/L).  Median splits on the widest axis.
struct Tree {
  int depth = 0;
  int64_t L = 0, n = 0;
  std::vector<int32_t> order;   // position -> vertex
  std::vector<V3> P;            // points in tree order (double copies of float inputs)
  std::vector<double> box;      // (2L-1) * 6
  int64_t first(int64_t j) const { return (int64_t)(((__int128)j * n) / L); }
};

void build_tree(const Mesh &M, int leaf, Tree &T) {
  T.n = M.nv;
  int64_t want = (T.n + leaf - 1) / leaf;
  T.depth = 1;
  while (((int64_t)1 << T.depth) < want) ++T.depth;
  T.L = (int64_t)1 << T.depth;
  T.order.resize(T.n);
  for (int64_t i = 0; i < T.n; ++i) T.order[i] = (int32_t)i;
  T.box.assign((2 * T.L - 1) * 6, 0.0);
  struct Job {
    int64_t node, j0, j1;
  };
  std::vector<Job> st{{0, 0, T.L}};
  while (!st.empty()) {
    Job jb = st.back();
    st.pop_back();
    int64_t p0 = T.first(jb.j0), p1 = T.first(jb.j1);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t p = p0; p < p1; ++p) {
      V3 v = M.V[T.order[p]];
      double c[3] = {v.x, v.y, v.z};
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], c[d]);
        hi[d] = std::max(hi[d], c[d]);
      }
    }
    double *b = &T.box[6 * jb.node];
    for (int d = 0; d < 3; ++d) {
      b[d] = lo[d];
      b[3 + d] = hi[d];
    }
    if (jb.j1 - jb.j0 == 1) continue;
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    int64_t jm = (jb.j0 + jb.j1) / 2, pm = T.first(jm);
    auto key = [&](int32_t i) {
      V3 v = M.V[i];
      return ax == 0 ? v.x : (ax == 1 ? v.y : v.z);
    };
    std::nth_element(T.order.begin() + p0, T.order.begin() + pm, T.order.begin() + p1,
                     [&](int32_t a, int32_t c) {
                       double ka = key(a), kc = key(c);
                       return ka < kc || (ka == kc && a < c);
                     });
    st.push_back({2 * jb.node + 1, jb.j0, jm});
    st.push_back({2 * jb.node + 2, jm, jb.j1});
  }
  T.P.resize(T.n);
  for (int64_t p = 0; p < T.n; ++p) T.P[p] = M.V[T.order[p]];
}

inline double box_d2(const double *b, V3 q) {
  double dx = q.x < b[0] ? b[0] - q.x : (q.x > b[3] ? q.x - b[3] : 0.0);
  double dy = q.y < b[1] ? b[1] - q.y : (q.y > b[4] ? q.y - b[4] : 0.0);
  double dz = q.z < b[2] ? b[2] - q.z : (q.z > b[5] ? q.z - b[5] : 0.0);
  return dx * dx + dy * dy + dz * dz;
}

// The nearest tree position strictly closer than sqrt(r2), or -1; among
// positions at the same (double) distance the lowest.  The answer is thus
// fixed by the point set alone, whatever order a search visits it in (the
// device search prunes in float32 and must agree with this one).
int64_t nearest_within(const Tree &T, V3 q, double r2) {
  struct Item {
    int64_t node;
    double d2;
  };
  Item st[128];
  int sp = 0;
  int64_t best = -1;
  double bd = r2;
  st[sp++] = {0, box_d2(&T.box[0], q)};
  // a subtree may hold a better point while its box is nearer than the best
  // distance, or exactly as near once a best exists (a lower position)
  auto open = [&](double d2) { return d2 < bd || (best >= 0 && d2 == bd); };
  while (sp) {
    Item it = st[--sp];
    if (!open(it.d2)) continue;
    if (it.node >= T.L - 1) {
      int64_t j = it.node - (T.L - 1);
      for (int64_t p = T.first(j), e = T.first(j + 1); p < e; ++p) {
        double d = len2(T.P[p] - q);
        if (d < bd || (best >= 0 && d == bd && p < best)) {
          bd = d;
          best = p;
        }
      }
      continue;
    }
    int64_t c0 = 2 * it.node + 1, c1 = c0 + 1;
    double d0 = box_d2(&T.box[6 * c0], q), d1 = box_d2(&T.box[6 * c1], q);
    if (d0 > d1) {
      std::swap(c0, c1);
      std::swap(d0, d1);
    }
    if (open(d1)) st[sp++] = {c1, d1};
    if (open(d0)) st[sp++] = {c0, d0};
  }
  return best;
}

// k nearest tree positions to q excluding `self`, ascending
int k_nearest(const Tree &T, V3 q, int64_t self, int k, int64_t *ids, double *d2s) {
  struct Item {
    int64_t node;
    double d2;
  };
  Item st[128];
  int sp = 0, cnt = 0;
  st[sp++] = {0, box_d2(&T.box[0], q)};
  while (sp) {
    Item it = st[--sp];
    if (cnt == k && !(it.d2 < d2s[k - 1])) continue;
    if (it.node >= T.L - 1) {
      int64_t j = it.node - (T.L - 1);
      for (int64_t p = T.first(j), e = T.first(j + 1); p < e; ++p) {
        if (p == self) continue;
        double d = len2(T.P[p] - q);
        if (cnt < k || d < d2s[cnt - 1]) {
          int s = cnt < k ? cnt++ : k - 1;
          while (s > 0 && d2s[s - 1] > d) {
            d2s[s] = d2s[s - 1];
            ids[s] = ids[s - 1];
            --s;
          }
          d2s[s] = d;
          ids[s] = p;
        }
      }
      continue;
    }
    int64_t c0 = 2 * it.node + 1, c1 = c0 + 1;
    double d0 = box_d2(&T.box[6 * c0], q), d1 = box_d2(&T.box[6 * c1], q);
    if (d0 > d1) {
      std::swap(c0, c1);
      std::swap(d0, d1);
    }
    if (cnt < k || d1 < d2s[cnt - 1]) st[sp++] = {c1, d1};
    if (cnt < k || d0 < d2s[cnt - 1]) st[sp++] = {c0, d0};
  }
  return cnt;
}

// ------------------------------------------------------- Voronoi cells
// bisector half-space of tree positions a (own) and b, pushed out by w
inline Plane bisector(const Tree &T, int64_t a, int64_t b, double w) {
  V3 pa = T.P[a], pb = T.P[b], n = pb - pa;
  double l = std::sqrt(len2(n));
  n = (1.0 / l) * n;
  return {n, 0.5 * (dot(n, pa) + dot(n, pb)) + w, (int32_t)b};
}

constexpr int KSEED = 32;

struct CellWork {
  Poly poly;
  std::vector<int32_t> applied;  // tree positions whose bisectors cut it
  double safe2 = 0;              // corners nearer than this need no check
  bool done = false;
};

// distinct corners of a polytope (loops repeat shared corners bitwise)
void distinct_corners(const Poly &p, std::vector<V3> &out) {
  out = p.pt;
  std::sort(out.begin(), out.end(), lex_less);
  out.erase(std::unique(out.begin(), out.end(),
                        [](V3 a, V3 b) { return a.x == b.x && a.y == b.y && a.z == b.z; }),
            out.end());
}

// ------------------------------------------------------------- flooding
using Rec = FloodRec;  // table row (tree position), typed id, Region box

struct PrimGeom {  // what the filter needs about a primitive
  int type;        // 1 edge (line through a, unit u), 2 face (plane through a, unit u)
  V3 a, u;
};

}  // namespace

int build_layout(const float *Vin, int64_t nv, const int32_t *Fin, int64_t nf,
                 const int32_t *Sin, int64_t ns, const BuildParams &prm,
                 NearestService *nearest,
                 bool (*on_tree)(void *, const Layout &), void *ctx, Layout &out,
                 std::string &err) {
  const double t_start = now_ms();
  int st = validate(Vin, nv, Fin, nf, Sin, ns, err);
  if (st) return st;
  const int threads = prm.threads > 0 ? prm.threads
                                      : (int)std::max(1u, std::thread::hardware_concurrency());
  Mesh M;
  M.nv = nv;
  M.nf = nf;
  M.V.resize(nv);
  for (int64_t i = 0; i < nv; ++i) M.V[i] = {Vin[3 * i], Vin[3 * i + 1], Vin[3 * i + 2]};
  if (nf > 0) M.F.assign(Fin, Fin + 3 * nf);
  build_topology(M, Sin, ns);

  // domain D
  double vlo[3] = {1e300, 1e300, 1e300}, vhi[3] = {-1e300, -1e300, -1e300};
  for (const V3 &v : M.V) {
    double c[3] = {v.x, v.y, v.z};
    for (int d = 0; d < 3; ++d) {
      vlo[d] = std::min(vlo[d], c[d]);
      vhi[d] = std::max(vhi[d], c[d]);
    }
  }
  double bbd = std::sqrt((vhi[0] - vlo[0]) * (vhi[0] - vlo[0]) +
                         (vhi[1] - vlo[1]) * (vhi[1] - vlo[1]) +
                         (vhi[2] - vlo[2]) * (vhi[2] - vlo[2]));
  double Dlo[3], Dhi[3];
  for (int d = 0; d < 3; ++d) {
    double c = 0.5 * (vlo[d] + vhi[d]);
    double h = 0.5 * (vhi[d] - vlo[d]) * prm.domain_scale + prm.domain_margin * bbd;
    if (h <= 0) h = 1e-3 * bbd;
    Dlo[d] = c - h;
    Dhi[d] = c + h;
  }
  // the device squares float32 coordinate differences: D must stay far
  // inside sqrt(FLT_MAX) ~ 1.8e19
  for (int d = 0; d < 3; ++d)
    if (!(std::fabs(Dlo[d]) <= 1e18 && std::fabs(Dhi[d]) <= 1e18)) {
      err = "domain D reaches beyond +-1e18";
      return 9;
    }
  const double diag = std::sqrt((Dhi[0] - Dlo[0]) * (Dhi[0] - Dlo[0]) +
                                (Dhi[1] - Dlo[1]) * (Dhi[1] - Dlo[1]) +
                                (Dhi[2] - Dlo[2]) * (Dhi[2] - Dlo[2]));
  const double delta = prm.delta_rel * diag;
  const double eta = 2.0 * delta * diag + delta * delta;
  const double eps = 1e-13 * diag;

  Tree T;
  build_tree(M, std::max(2, std::min(32, prm.leaf_size)), T);

  // ---- device arrays of the KD tree (needed by the certification service)
  out = Layout();
  out.nv = nv;
  out.nf = nf;
  out.ne = M.ne;
  for (int d = 0; d < 3; ++d) {
    out.dom[d] = (float)Dlo[d];
    out.dom[3 + d] = (float)Dhi[d];
  }
  out.delta = (float)delta;
  out.kd_depth = T.depth;
  out.kd_points.resize(4 * nv);
  out.pos_of_vertex.resize(nv);
  for (int64_t p = 0; p < nv; ++p) {
    int32_t v = T.order[p];
    out.kd_points[4 * p + 0] = Vin[3 * v + 0];
    out.kd_points[4 * p + 1] = Vin[3 * v + 1];
    out.kd_points[4 * p + 2] = Vin[3 * v + 2];
    std::memcpy(&out.kd_points[4 * p + 3], &v, 4);
    out.pos_of_vertex[v] = (int32_t)p;
  }
  out.kd_nodes.resize((T.L - 1) * 12);
  for (int64_t i = 0; i < T.L - 1; ++i) {
    const double *c0 = &T.box[6 * (2 * i + 1)], *c1 = &T.box[6 * (2 * i + 2)];
    float *o = &out.kd_nodes[12 * i];
    // boxes of float points are exact in float
    o[0] = (float)c0[0]; o[1] = (float)c0[1]; o[2] = (float)c0[2]; o[3] = (float)c0[3];
    o[4] = (float)c0[4]; o[5] = (float)c0[5]; o[6] = (float)c1[0]; o[7] = (float)c1[1];
    o[8] = (float)c1[2]; o[9] = (float)c1[3]; o[10] = (float)c1[4]; o[11] = (float)c1[5];
  }
  for (int d = 0; d < 6; ++d) out.kd_root[d] = (float)T.box[d];
  if (on_tree && nearest && !on_tree(ctx, out)) nearest = nullptr;

  // ---- Voronoi cells: on the device service when asked (cell_core.h: the
  // same steps, the same values); the rows it hands back, or all of them,
  // here
  const double t_cells = now_ms();
  const double epsc = 1e-12 * diag * diag;
  const bool trace = std::getenv("P2M_BUILD_TRACE") != nullptr;
  std::vector<std::vector<int32_t>> nbr(nv);
  std::vector<Poly> cell(nv);  // widened cells (loops only: no planes)
  std::vector<int64_t> todo;   // rows whose cells are made here
  bool cells_done_on_device = false;
  int64_t rounds = 0, cert_queries = 0;  // the certification's counts over all rows
  if (prm.device_cells && nearest) {
    CellProblem cp;
    cp.nv = nv;
    for (int d = 0; d < 3; ++d) {
      cp.lo[d] = Dlo[d];
      cp.hi[d] = Dhi[d];
    }
    cp.eps = eps;
    cp.epsc = epsc;
    cp.delta = delta;
    CellResult cr;
    if (nearest->cells(cp, cr) && (int64_t)cr.gave_up.size() == nv &&
        (int64_t)cr.nb_off.size() == nv + 1 && (int64_t)cr.pt_off.size() == nv + 1 &&
        (int64_t)cr.beg_off.size() == nv + 1) {
      cells_done_on_device = true;
      rounds = cr.rounds;
      cert_queries = cr.queries;
      parallel_for(nv, threads, 1024, [&](int64_t p, int) {
        if (cr.gave_up[p]) return;
        nbr[p].assign(cr.nb.begin() + cr.nb_off[p], cr.nb.begin() + cr.nb_off[p + 1]);
        Poly &c = cell[p];
        c.pt.resize((size_t)(cr.pt_off[p + 1] - cr.pt_off[p]));
        for (size_t i = 0; i < c.pt.size(); ++i) {
          const double *x = &cr.pt[3 * ((size_t)cr.pt_off[p] + i)];
          c.pt[i] = {x[0], x[1], x[2]};
        }
        c.beg.assign(cr.beg.begin() + cr.beg_off[p], cr.beg.begin() + cr.beg_off[p + 1]);
      });
      for (int64_t p = 0; p < nv; ++p)
        if (cr.gave_up[p]) todo.push_back(p);
    }
  }
  if (!cells_done_on_device) {
    todo.resize(nv);
    for (int64_t p = 0; p < nv; ++p) todo[p] = p;
  }
  out.cells_device = nv - (int64_t)todo.size();
  out.cells_host = (int64_t)todo.size();
  const int64_t nt = (int64_t)todo.size();
  // k-nearest seeding of the rows in todo (cells[i] is row todo[i])
  std::vector<CellWork> cells(nt);
  std::vector<CutScratch> scratch(threads);
  std::vector<Poly> tmp(threads);
  const bool fail_cells = inject_at("cells");
  parallel_for(nt, threads, 64, [&](int64_t i, int t) {
    if (fail_cells && i == nt / 2) throw std::bad_alloc();
    const int64_t p = todo[i];
    CellWork &C = cells[i];
    make_box(C.poly, Dlo, Dhi);
    int64_t ids[KSEED];
    double d2s[KSEED];
    int k = k_nearest(T, T.P[p], p, KSEED, ids, d2s);
    for (int j = 0; j < k; ++j) {
      if (cut(C.poly, bisector(T, p, ids[j], 0.0), eps, tmp[t], scratch[t])) std::swap(C.poly, tmp[t]);
      C.applied.push_back((int32_t)ids[j]);
    }
    // no vertex outside the k nearest can be nearer than p to a corner that
    // lies within half the k-th distance of p
    C.safe2 = k == KSEED ? 0.25 * d2s[KSEED - 1] : std::numeric_limits<double>::infinity();
  });

  // optional trace of the cell stage on stderr (P2M_BUILD_TRACE=1)
  if (trace)
    std::fprintf(stderr, "p2m build: %lld cells on the device, seeding of %lld here %.0f ms\n",
                 (long long)out.cells_device, (long long)nt, now_ms() - t_cells);
  // ---- certification rounds: a corner x is settled when no vertex is
  // strictly nearer to x than the cell's own vertex (the exact search, on
  // the device when it offers one); a cell whose corners are all settled
  // equals Cell(v) ∩ D (it is convex and contains the cell)
  std::vector<std::vector<V3>> corner(nt);
  std::vector<int64_t> coff(nt + 1);
  int64_t host_rounds = 0;
  for (;;) {
    // far corners of the cells still open
    parallel_for(nt, threads, 256, [&](int64_t i, int) {
      auto &cv = corner[i];
      cv.clear();
      if (cells[i].done) return;
      std::vector<V3> all;
      distinct_corners(cells[i].poly, all);
      for (V3 x : all)
        if (len2(x - T.P[todo[i]]) > cells[i].safe2) cv.push_back(x);
      if (cv.empty()) cells[i].done = true;
    });
    coff[0] = 0;
    for (int64_t i = 0; i < nt; ++i) coff[i + 1] = coff[i] + (int64_t)corner[i].size();
    const int64_t nq = coff[nt];
    if (nq == 0) break;
    ++host_rounds;
    rounds = std::max(rounds, host_rounds);
    cert_queries += nq;
    const double t_round = now_ms();
    // the exact search of every corner: the nearest vertex strictly nearer
    // than the cell's own (-2: not answered, searched here)
    std::vector<int64_t> w_of(nq, -2);
    if (nearest) {
      std::vector<double> xs(3 * (size_t)nq), rs(nq);
      parallel_for(nt, threads, 256, [&](int64_t i, int) {
        for (size_t j = 0; j < corner[i].size(); ++j) {
          const int64_t g = coff[i] + (int64_t)j;
          const V3 x = corner[i][j];
          xs[3 * g] = x.x;
          xs[3 * g + 1] = x.y;
          xs[3 * g + 2] = x.z;
          rs[g] = len2(x - T.P[todo[i]]) - epsc;
        }
      });
      if (!nearest->within(xs.data(), rs.data(), nq, w_of.data()))
        std::fill(w_of.begin(), w_of.end(), -2);
    }
    std::atomic<int64_t> host_searches{0};
    parallel_for(nt, threads, 64, [&](int64_t i, int t) {
      CellWork &C = cells[i];
      if (corner[i].empty()) return;
      const int64_t p = todo[i];
      std::vector<int64_t> cand;
      for (size_t j = 0; j < corner[i].size(); ++j) {
        const V3 x = corner[i][j];
        int64_t w = w_of[coff[i] + (int64_t)j];
        if (w < -1) {
          w = nearest_within(T, x, len2(x - T.P[p]) - epsc);
          ++host_searches;
        }
        if (w >= 0 && w != p &&
            std::find(C.applied.begin(), C.applied.end(), (int32_t)w) == C.applied.end() &&
            std::find(cand.begin(), cand.end(), w) == cand.end())
          cand.push_back(w);
      }
      if (cand.empty()) {
        C.done = true;
        return;
      }
      // nearest first; equal distances in the order found
      std::stable_sort(cand.begin(), cand.end(), [&](int64_t a, int64_t b) {
        return len2(T.P[a] - T.P[p]) < len2(T.P[b] - T.P[p]);
      });
      for (int64_t w : cand) {
        if (cut(C.poly, bisector(T, p, w, 0.0), eps, tmp[t], scratch[t])) std::swap(C.poly, tmp[t]);
        C.applied.push_back((int32_t)w);
      }
    });
    if (trace)
      std::fprintf(stderr, "p2m build: round %lld: %lld corners, %lld searched on the host, "
                   "%.0f ms\n", (long long)host_rounds, (long long)nq,
                   (long long)host_searches.load(), now_ms() - t_round);
    if (host_rounds > 64) break;
  }
  corner.clear();
  corner.shrink_to_fit();

  // neighbours (generators of surviving bisector faces) and widened cells
  parallel_for(nt, threads, 64, [&](int64_t i, int t) {
    const int64_t p = todo[i];
    auto &nb = nbr[p];
    for (const Plane &h : cells[i].poly.pl)
      if (h.src >= 0 && std::find(nb.begin(), nb.end(), h.src) == nb.end()) nb.push_back(h.src);
    double wlo[3], whi[3];
    for (int d = 0; d < 3; ++d) {
      wlo[d] = Dlo[d] - delta;
      whi[d] = Dhi[d] + delta;
    }
    Poly &c = cell[p];
    make_box(c, wlo, whi);
    for (int32_t w : nb)
      if (cut(c, bisector(T, p, w, delta), eps, tmp[t], scratch[t])) std::swap(c, tmp[t]);
    c.pl.clear();
    c.pl.shrink_to_fit();
    cells[i].poly.clear();
    cells[i].poly.pl.shrink_to_fit();
    cells[i].poly.pt.shrink_to_fit();
    cells[i].applied.clear();
    cells[i].applied.shrink_to_fit();
  });
  cells.clear();
  cells.shrink_to_fit();
  int64_t npairs = 0;
  for (auto &nb : nbr) npairs += (int64_t)nb.size();
  out.nb_off.assign(nv + 1, 0);
  for (int64_t p = 0; p < nv; ++p) out.nb_off[p + 1] = out.nb_off[p] + (uint32_t)nbr[p].size();
  out.nb.resize(npairs);
  out.nbp.resize(4 * npairs);
  for (int64_t p = 0; p < nv; ++p)
    for (size_t k = 0; k < nbr[p].size(); ++k) {
      const uint32_t w = (uint32_t)nbr[p][k], j = out.nb_off[p] + (uint32_t)k;
      out.nb[j] = w;
      std::memcpy(&out.nbp[4 * (size_t)j], &out.kd_points[4 * (size_t)w], 12);
      std::memcpy(&out.nbp[4 * (size_t)j + 3], &w, 4);
    }
  const double t_flood = now_ms();

  // ---- flooding inspection (Alg. 1) over every edge and every face
  auto face_inward = [&](int64_t f, int k) {
    // unit normal of the plane through edge k of face f, perpendicular to
    // the face, pointing into the face
    V3 a = M.V[M.F[3 * f]], b = M.V[M.F[3 * f + 1]], c = M.V[M.F[3 * f + 2]];
    V3 n = cross(b - a, c - a);
    V3 d = M.V[M.F[3 * f + (k + 1) % 3]] - M.V[M.F[3 * f + k]];
    V3 m = cross(n, d);
    return (1.0 / std::sqrt(len2(m))) * m;
  };
  struct TLS {
    std::vector<Rec> recs;
    std::vector<int64_t> seen;
    std::vector<int32_t> queue;
    Poly A, B, C;
    CutScratch S;
    std::vector<double> gv;
    std::unique_ptr<fc::Work> W{new fc::Work};
    int64_t inspections = 0, bounded = 0, unbounded = 0;
  };
  std::vector<TLS> tls(threads);
  for (auto &x : tls) {
    x.seen.assign(nv, -1);
    x.queue.resize(nv + 3);
  }
  // what the flooding of primitive i needs: its Space-perp half-spaces, the
  // filter's geometry, its seeds (vertex ids) and typed id; false for a
  // degenerate face, which is not flooded
  struct PrimData {
    Plane perp[16];
    int np = 0;
    PrimGeom g;
    int32_t seeds[3] = {-1, -1, -1};
    int ns = 0;
    int32_t tid = 0;
  };
  auto setup = [&](int64_t i, PrimData &P) -> bool {
    Plane *perp = P.perp;
    int &np_ = P.np;
    PrimGeom &g = P.g;
    int32_t *seeds = P.seeds;
    int &nseed = P.ns;
    int32_t &tid = P.tid;
    if (i < M.ne) {
      int64_t e = i;
      V3 a = M.V[M.E[2 * e]], b = M.V[M.E[2 * e + 1]];
      V3 u = b - a;
      u = (1.0 / std::sqrt(len2(u))) * u;
      perp[np_++] = {-1.0 * u, -dot(u, a) + delta, -10};
      perp[np_++] = {u, dot(u, b) + delta, -11};
      for (int64_t j = M.ef_off[e]; j < M.ef_off[e + 1] && np_ < 16; ++j) {
        int64_t f = M.ef[j];
        if (f < 0 || M.degenerate[f]) continue;  // a segment side adds no half-space
        int k = M.fedge[3 * f] == e ? 0 : (M.fedge[3 * f + 1] == e ? 1 : 2);
        V3 m = face_inward(f, k);  // the far side of f: m.(x - a) <= 0
        perp[np_++] = {m, dot(m, a) + delta, (int32_t)(-12 - j)};
      }
      g = {1, a, u};
      seeds[0] = M.E[2 * e];
      seeds[1] = M.E[2 * e + 1];
      nseed = 2;
      tid = (int32_t)(1u << 30 | (uint32_t)e);
    } else {
      int64_t f = i - M.ne;
      if (M.degenerate[f]) return false;
      for (int k = 0; k < 3; ++k) {
        V3 m = face_inward(f, k);  // inside: m.(x - p_k) >= 0
        V3 pk = M.V[M.F[3 * f + k]];
        perp[np_++] = {-1.0 * m, -dot(m, pk) + delta, -20 - k};
      }
      V3 a = M.V[M.F[3 * f]], b = M.V[M.F[3 * f + 1]], c = M.V[M.F[3 * f + 2]];
      V3 n = cross(b - a, c - a);
      g = {2, a, (1.0 / std::sqrt(len2(n))) * n};
      for (int k = 0; k < 3; ++k) seeds[k] = M.F[3 * f + k];
      nseed = 3;
      tid = (int32_t)(2u << 30 | (uint32_t)f);
    }
    return true;
  };
  // ---- the flooding problem in flat arrays (fc::Flat), read alike by the
  // host core, the device kernel and (cells only) the unbounded fallback:
  // the widened cells, then every non-degenerate primitive
  std::vector<int64_t> pt_off(nv + 1, 0), beg_off(nv + 1, 0);
  for (int64_t p = 0; p < nv; ++p) {
    pt_off[p + 1] = pt_off[p] + (int64_t)cell[p].pt.size();
    beg_off[p + 1] = beg_off[p] + (int64_t)cell[p].beg.size();
  }
  std::vector<V3> cpt((size_t)pt_off[nv]);
  std::vector<int32_t> cbeg((size_t)beg_off[nv]);
  parallel_for(nv, threads, 1024, [&](int64_t p, int) {
    Poly &c = cell[p];
    std::copy(c.pt.begin(), c.pt.end(), cpt.begin() + pt_off[p]);
    std::copy(c.beg.begin(), c.beg.end(), cbeg.begin() + beg_off[p]);
    c = Poly();
  });
  cell.clear();
  cell.shrink_to_fit();
  const int64_t nprim = M.ne + M.nf;
  std::vector<int32_t> prim_np(nprim, -1);  // -1: not flooded (degenerate face)
  parallel_for(nprim, threads, 4096, [&](int64_t i, int) {
    PrimData P;
    if (setup(i, P)) prim_np[i] = P.np;
  });
  std::vector<int64_t> idx;  // problem index -> primitive
  std::vector<int64_t> perp_off(1, 0);
  for (int64_t i = 0; i < nprim; ++i)
    if (prim_np[i] >= 0) {
      idx.push_back(i);
      perp_off.push_back(perp_off.back() + prim_np[i]);
    }
  std::vector<int32_t>().swap(prim_np);
  const int64_t nk = (int64_t)idx.size();
  std::vector<double> fperp(4 * (size_t)perp_off[nk]), fg(6 * (size_t)nk);
  std::vector<int32_t> gtype(nk), srow(3 * (size_t)nk), svid(3 * (size_t)nk), tids(nk);
  parallel_for(nk, threads, 4096, [&](int64_t k, int) {
    PrimData P;
    setup(idx[k], P);
    for (int j = 0; j < P.np; ++j) {
      double *h = &fperp[4 * (size_t)(perp_off[k] + j)];
      h[0] = P.perp[j].n.x;
      h[1] = P.perp[j].n.y;
      h[2] = P.perp[j].n.z;
      h[3] = P.perp[j].c;
    }
    gtype[k] = P.g.type;
    const double gg[6] = {P.g.a.x, P.g.a.y, P.g.a.z, P.g.u.x, P.g.u.y, P.g.u.z};
    std::copy(gg, gg + 6, fg.begin() + 6 * k);
    for (int j = 0; j < 3; ++j) {
      svid[3 * k + j] = j < P.ns ? P.seeds[j] : -1;
      srow[3 * k + j] = j < P.ns ? out.pos_of_vertex[P.seeds[j]] : -1;
    }
    tids[k] = P.tid;
  });
  fc::Flat fl;
  fl.pt_off = pt_off.data();
  fl.pt = cpt.data();
  fl.beg_off = beg_off.data();
  fl.beg = cbeg.data();
  fl.pos = T.P.data();
  fl.vids = T.order.data();
  fl.nbo = out.nb_off.data();
  fl.nbs = out.nb.data();
  fl.perp_off = perp_off.data();
  fl.perp = fperp.data();
  fl.gtype = gtype.data();
  fl.g = fg.data();
  fl.seed_row = srow.data();
  fl.seed_vid = svid.data();
  fl.tid = tids.data();
  // row p's cell as a Poly, for the unbounded fallback (the planes of its
  // faces are not needed by the flooding, only their loops)
  auto cell_poly = [&](int64_t p, Poly &c) {
    c.pt.assign(cpt.begin() + pt_off[p], cpt.begin() + pt_off[p + 1]);
    c.beg.assign(cbeg.begin() + beg_off[p], cbeg.begin() + beg_off[p + 1]);
    c.pl.assign(c.beg.size() - 1, Plane{{0, 0, 0}, 0, -1});
  };

  // the unbounded host flooding of a primitive the shared core
  // (flood_core.h) gives up: the same steps on growable buffers, with the cap
  // loop ordered by angle where it cannot be chained; stamp marks its visits
  auto flood_unbounded = [&](int64_t stamp, const PrimData &P, TLS &X) {
    const Plane *perp = P.perp;
    const int np_ = P.np;
    const PrimGeom &g = P.g;
    const int32_t *seeds = P.seeds;
    const int nseed = P.ns;
    const int32_t tid = P.tid;
    auto gval = [&](V3 x, V3 pv) {
      V3 w = x - g.a;
      double s = dot(w, g.u);
      double dist2 = g.type == 1 ? len2(w) - s * s : s * s;
      return len2(x - pv) - dist2 + eta;
    };
    int64_t head = 0, tail = 0;
    for (int s = 0; s < nseed; ++s) {
      int64_t p = out.pos_of_vertex[seeds[s]];
      X.seen[p] = stamp;
      X.queue[tail++] = (int32_t)p;
    }
    while (head < tail) {
      const int64_t p = X.queue[head++];
      ++X.inspections;
      // ConvexPoly(v, prim) = Cell(v) ∩ Space-perp(prim).  A half-space that
      // leaves every point of the cell beyond it empties the result whatever
      // the order of the cuts (later corners are convex combinations of the
      // cell's), so that case is settled before any cut is made.
      cell_poly(p, X.C);
      const Poly *cur = &X.C;
      bool emptied = false;
      for (int j = 0; j < np_ && !emptied; ++j) {
        bool all_beyond = true;
        for (const V3 &x : cur->pt)
          if (!(dot(perp[j].n, x) - perp[j].c > eps)) {
            all_beyond = false;
            break;
          }
        emptied = all_beyond && !cur->pt.empty();
      }
      if (emptied) continue;
      Poly *bufs[2] = {&X.A, &X.B};
      int wsel = 0;
      for (int j = 0; j < np_ && !cur->empty(); ++j) {
        if (cut(*cur, perp[j], eps, *bufs[wsel], X.S)) {
          cur = bufs[wsel];
          wsel ^= 1;
        }
      }
      if (cur->empty()) continue;
      const V3 pv = T.P[p];
      const int32_t vid = T.order[p];
      bool keep = (g.type == 1) ? (seeds[0] == vid || seeds[1] == vid)
                                : (seeds[0] == vid || seeds[1] == vid || seeds[2] == vid);
      double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
      bool have = false;
      auto grow = [&](V3 x) {
        blo[0] = std::min(blo[0], x.x); bhi[0] = std::max(bhi[0], x.x);
        blo[1] = std::min(blo[1], x.y); bhi[1] = std::max(bhi[1], x.y);
        blo[2] = std::min(blo[2], x.z); bhi[2] = std::max(bhi[2], x.z);
        have = true;
      };
      // g at every loop point once (each point ends two loop edges)
      X.gv.resize(cur->pt.size());
      for (size_t q = 0; q < cur->pt.size(); ++q) X.gv[q] = gval(cur->pt[q], pv);
      for (int f = 0; f < cur->nf(); ++f) {
        const int b0 = cur->beg[f], k = cur->beg[f + 1] - b0;
        for (int q = 0; q < k; ++q) {
          V3 x0 = cur->pt[b0 + q], x1 = cur->pt[b0 + (q + 1) % k];
          double g0 = X.gv[b0 + q], g1 = X.gv[b0 + (q + 1) % k];
          if (g0 > 0) {
            keep = true;
            grow(x0);
          }
          if ((g0 > 0) != (g1 > 0)) {
            // g restricted to the edge is a quadratic in t: bracket its zero
            V3 d = x1 - x0, w0 = x0 - g.a, r0 = x0 - pv;
            double du = dot(d, g.u), wu = dot(w0, g.u);
            double A, B, Cc;
            if (g.type == 1) {  // |x-v|^2 - (|w|^2 - (w.u)^2)
              A = len2(d) - (len2(d) - du * du);
              B = 2 * dot(r0, d) - 2 * (dot(w0, d) - wu * du);
              Cc = len2(r0) - (len2(w0) - wu * wu) + eta;
            } else {            // |x-v|^2 - (w.u)^2
              A = len2(d) - du * du;
              B = 2 * dot(r0, d) - 2 * wu * du;
              Cc = len2(r0) - wu * wu + eta;
            }
            double tb[2];
            fc::edge_crossing(A, B, Cc, g0 > 0, &tb[0], &tb[1]);
            grow(x0 + tb[0] * d);
            grow(x0 + tb[1] * d);
          }
        }
      }
      if (!keep) continue;
      if (!have)
        for (V3 x : cur->pt) grow(x);
      Rec r;
      r.row = (int32_t)p;
      r.tid = tid;
      for (int d = 0; d < 3; ++d) {
        float l = (float)(blo[d] - delta), h = (float)(bhi[d] + delta);
        if ((double)l > blo[d] - delta) l = std::nextafter(l, -INFINITY);
        if ((double)h < bhi[d] + delta) h = std::nextafter(h, INFINITY);
        r.box[d] = l;
        r.box[3 + d] = h;
      }
      X.recs.push_back(r);
      for (int32_t w : nbr[p])
        if (X.seen[w] != stamp) {
          X.seen[w] = stamp;
          X.queue[tail++] = w;
        }
    }
  };
  auto prim_of_tid = [&](int32_t tid) -> int64_t {
    const int64_t id = tid & ((1 << 30) - 1);
    return ((uint32_t)tid >> 30) == 1 ? id : M.ne + id;
  };

  const double t_flat = now_ms();
  if (trace) std::fprintf(stderr, "p2m build: flooding problem %.0f ms\n", t_flat - t_flood);
  // the host side of the shared core
  struct HostEnv : fc::Flat {
    int64_t *seen;
    int64_t stamp;
    std::vector<Rec> *recs;
    void mark_seed(int32_t p) { seen[p] = stamp; }
    bool mark(int32_t w, const int32_t *, int64_t) {
      if (seen[w] == stamp) return false;
      seen[w] = stamp;
      return true;
    }
    void emit(int32_t row, int32_t typed_id, const float box[6]) {
      Rec r;
      r.row = row;
      r.tid = typed_id;
      for (int d = 0; d < 6; ++d) r.box[d] = box[d];
      recs->push_back(r);
    }
  };
  // P2M_FLOOD_UNBOUNDED=1 floods every primitive with the unbounded code;
  // P2M_FLOOD_LANES=1 floods with the device kernel's warp algorithm
  // (flood_warp.h, its 32 lanes run one after another) before the bounded
  // core: checks that these paths build the same layout
  auto env_flag = [](const char *name) {
    const char *v = std::getenv(name);
    return v && std::atoi(v) != 0;
  };
  const bool only_unbounded = env_flag("P2M_FLOOD_UNBOUNDED");
  const bool lanes = env_flag("P2M_FLOOD_LANES");
  std::vector<std::unique_ptr<fw::WarpWork>> lane_work(lanes ? threads : 0);
  for (auto &w : lane_work) w.reset(new fw::WarpWork);
  const bool fail_flooding = inject_at("flooding");
  // primitive k flooded here by worker t: the bounded core, else the
  // unbounded code
  auto flood_here = [&](int64_t k, int t) {
    TLS &X = tls[t];
    HostEnv env;
    static_cast<fc::Flat &>(env) = fl;
    env.seen = X.seen.data();
    env.stamp = 2 * k;
    env.recs = &X.recs;
    const size_t r0 = X.recs.size();
    int64_t insp = 0;
    if (lanes && !only_unbounded) {
      if (fw::flood_warp(*lane_work[t], env, k, eps, delta, eta, insp) == 0) {
        X.inspections += insp;
        ++X.bounded;
        return;
      }
      X.recs.resize(r0);
    }
    fc::Prim fp;
    if (!only_unbounded && fl.load(k, fp) &&
        fc::flood_prim(fp, eps, delta, eta, env, *X.W, X.queue.data(), (int64_t)X.queue.size(),
                       insp) == 0) {
      X.inspections += insp;
      ++X.bounded;
      return;
    }
    X.recs.resize(r0);
    ++X.unbounded;
    PrimData P;
    setup(idx[k], P);
    flood_unbounded(2 * k + 1, P, X);
  };

  // On the device service, when asked, side by side with the host: the
  // device floods primitives from the front of [0, nk) in a few calls, each
  // taking a share of what nobody has taken yet, while host workers flood
  // from the back, a small block at a time, and take up first what an
  // earlier call handed back.  Which side floods a primitive changes none of
  // its records, and every row is sorted into a total order when packed, so
  // the layout is the same whatever the split.
  std::vector<uint8_t> host_todo;  // empty: the host floods everything
  int64_t n_device = 0, n_beside = 0, device_calls = 0, device_returned = 0;
  std::vector<Rec> drec;  // the device's records (row -1: dropped)
  if (prm.device_flood && nearest && nk > 0) {
    FloodProblem pb;
    pb.nv = nv;
    pb.cell_pt_off = pt_off.data();
    pb.cell_pt = &cpt.data()->x;
    pb.cell_beg_off = beg_off.data();
    pb.cell_beg = cbeg.data();
    pb.pv = &T.P.data()->x;
    pb.vid = T.order.data();
    pb.nb_off = out.nb_off.data();
    pb.nb = out.nb.data();
    pb.perp = fperp.data();
    pb.eps = eps;
    pb.delta = delta;
    pb.eta = eta;
    // host workers beside the thread that drives the device; the device
    // floods about as fast as 30 Grace cores (390 k against 13 k primitives
    // a second on the 1.3M-triangle mesh); its first share is, unless set,
    // 22.5 / (22.5 + workers) of all, a little less than that rate gives it,
    // and each later call takes 0.6 of what is left while that is at least
    // flood_min_share primitives
    const int nw = prm.flood_host_workers >= 0 ? std::min(prm.flood_host_workers, threads)
                   : (threads > 2 ? threads - 1 : 1);
    constexpr int64_t kBlock = 64;
    const int64_t min_share = std::max<int64_t>(1, prm.flood_min_share);
    const double first = prm.flood_first_share >= 0 ? std::min(1.0, prm.flood_first_share)
                                                    : 22.5 / (22.5 + nw);
    std::mutex mu;
    int64_t front = 0, back = nk;    // [front, back): not taken yet
    std::vector<int64_t> returned;   // handed back by a finished device call
    size_t returned_at = 0;          // returned[0 .. returned_at): taken up
    bool stop = false;
    std::exception_ptr failure;
    std::atomic<int64_t> beside{0};
    auto worker = [&](int t) {
      int64_t mine = 0;
      try {
        if (fail_flooding) throw std::bad_alloc();
        for (;;) {
          int64_t k0 = 0, k1 = 0, hb = -1;
          {
            std::lock_guard<std::mutex> g(mu);
            if (stop) break;
            if (returned_at < returned.size()) {
              hb = returned[returned_at++];
            } else if (back > front) {
              k1 = back;
              k0 = std::max(front, back - kBlock);
              back = k0;
            } else {
              break;
            }
          }
          if (hb >= 0) {
            flood_here(hb, t);
            continue;
          }
          for (int64_t k = k1 - 1; k >= k0; --k) flood_here(k, t);
          mine += k1 - k0;
        }
      } catch (...) {
        std::lock_guard<std::mutex> g(mu);
        if (!failure) failure = std::current_exception();
        stop = true;
      }
      beside += mine;
    };
    // one device call on [k0, k1): the problem's per-primitive arrays from
    // k0 on (the offsets stay absolute, into the whole arrays)
    int64_t dinsp = 0;
    auto device_call = [&](int64_t k0, int64_t k1, std::vector<uint8_t> &gave) {
      FloodProblem sub = pb;
      sub.n = k1 - k0;
      sub.perp_off = perp_off.data() + k0;
      sub.gtype = gtype.data() + k0;
      sub.g = fg.data() + 6 * k0;
      sub.seed_row = srow.data() + 3 * k0;
      sub.seed_vid = svid.data() + 3 * k0;
      sub.tid = tids.data() + k0;
      std::vector<Rec> r;
      int64_t insp = 0;
      if (!nearest->flood(sub, r, gave, insp) || (int64_t)gave.size() != sub.n) return false;
      ++device_calls;
      dinsp += insp;
      if (drec.empty()) drec.swap(r);
      else drec.insert(drec.end(), r.begin(), r.end());
      return true;
    };
    front = std::max<int64_t>(1, std::min<int64_t>(nk, (int64_t)std::ceil(first * (double)nk)));
    int64_t k0 = 0, k1 = front;
    std::vector<std::thread> pool;
    try {
      for (int t = 0; t < nw; ++t) pool.emplace_back(worker, t);
      for (;;) {
        std::vector<uint8_t> gave;
        const bool ok = device_call(k0, k1, gave);
        std::lock_guard<std::mutex> g(mu);
        if (!ok) {
          front = k0;  // the workers take the range back (front == k1 until now)
          break;
        }
        for (int64_t k = k0; k < k1; ++k)
          if (gave[k - k0]) returned.push_back(k);
          else ++n_device;
        const int64_t left = back - front;
        if (stop || left < min_share) break;
        k0 = front;
        k1 = front + (int64_t)std::ceil(0.6 * left);
        front = k1;
      }
    } catch (...) {
      std::lock_guard<std::mutex> g(mu);
      if (!failure) failure = std::current_exception();
      stop = true;
    }
    for (auto &th : pool) th.join();
    if (failure) std::rethrow_exception(failure);
    n_beside = beside.load();
    device_returned = (int64_t)returned.size();
    // what the workers did not take up is flooded below; the device's
    // records of every primitive it handed back are dropped
    host_todo.assign(nk, 0);
    for (size_t j = returned_at; j < returned.size(); ++j) host_todo[returned[j]] = 1;
    // and a range nobody took (a failed call's, given back after the
    // workers had finished)
    for (int64_t k = front; k < back; ++k) host_todo[k] = 1;
    std::vector<uint8_t> prim_gave(nprim, 0);
    for (int64_t k : returned) prim_gave[idx[k]] = 1;
    std::vector<int64_t>().swap(returned);
    const int64_t nd = (int64_t)drec.size();
    parallel_for((nd + 4095) / 4096, threads, 16, [&](int64_t c, int) {
      for (int64_t j = 4096 * c; j < std::min(nd, 4096 * (c + 1)); ++j) {
        Rec &r = drec[j];
        const int64_t pi = prim_of_tid(r.tid);
        if (!(r.row >= 0 && r.row < nv && pi >= 0 && pi < nprim && !prim_gave[pi])) r.row = -1;
      }
    });
    tls[0].inspections += dinsp;
  }

  const double t_host_flood = now_ms();
  if (trace && !host_todo.empty())
    std::fprintf(stderr,
                 "p2m build: device flooding %.0f ms (%lld primitives in %lld calls, %lld handed "
                 "back; %lld flooded here beside it)\n",
                 t_host_flood - t_flat, (long long)n_device, (long long)device_calls,
                 (long long)device_returned, (long long)n_beside);
  parallel_for(nk, threads, 32, [&](int64_t k, int t) {
    if (fail_flooding && k == nk / 2) throw std::bad_alloc();
    if (!host_todo.empty() && !host_todo[k]) return;
    flood_here(k, t);
  });

  const double t_pack = now_ms();
  if (trace) std::fprintf(stderr, "p2m build: host flooding %.0f ms\n", t_pack - t_host_flood);
  // ---- pack the CSR table in row (tree) order
  int64_t total = 0, insp = 0;
  out.flood_device = n_device;
  out.flood_bounded = out.flood_unbounded = 0;
  for (auto &x : tls) {
    insp += x.inspections;
    out.flood_bounded += x.bounded;
    out.flood_unbounded += x.unbounded;
  }
  // ---- packing: the code frame, then the table on the device service when
  // asked (pack_core.h: the same steps and words), else here
  float qstep[3], qbase[3];
  for (int d = 0; d < 3; ++d) {
    float flo = (float)(Dlo[d] - 4 * delta), fhi = (float)(Dhi[d] + 4 * delta);
    out.qframe_lo[d] = flo;
    out.qframe_inv[d] = (float)((double)(kQMax - 16) / ((double)fhi - (double)flo));
  }
  q_frame_derive(out.qframe_lo, out.qframe_inv, qstep, qbase);
  int64_t maxl = 0;
  std::atomic<int64_t> bad_boxes{0};
  bool packed = false;
  if (prm.device_pack && nearest) {
    std::vector<PackPart> parts;
    for (auto &x : tls) parts.push_back({x.recs.data(), (int64_t)x.recs.size()});
    parts.push_back({drec.data(), (int64_t)drec.size()});
    int64_t ml = 0, bad = 0;
    if (nearest->pack(nv, parts, out.qframe_lo, out.qframe_inv, out, ml, bad)) {
      packed = true;
      maxl = ml;
      bad_boxes = bad;
      total = out.row_off[nv];
      out.pack_device = 1;
      tls.clear();
      std::vector<Rec>().swap(drec);
    }
  }
  if (!packed) {
  // bucket the records by row: counts and then positions taken with atomic
  // increments, in parallel over blocks of every record list (the order
  // inside a row is fixed by the sort below, a total order)
  std::vector<std::vector<Rec> *> srcs;
  for (auto &x : tls) srcs.push_back(&x.recs);
  srcs.push_back(&drec);
  std::vector<std::pair<int, int64_t>> blocks;  // (list, first record)
  for (size_t q = 0; q < srcs.size(); ++q)
    for (int64_t j = 0; j < (int64_t)srcs[q]->size(); j += 1 << 16) blocks.push_back({(int)q, j});
  auto for_records = [&](auto &&fn) {
    parallel_for((int64_t)blocks.size(), threads, 1, [&](int64_t bi, int) {
      const std::vector<Rec> &v = *srcs[blocks[bi].first];
      const int64_t j0 = blocks[bi].second, j1 = std::min<int64_t>(j0 + (1 << 16), v.size());
      for (int64_t j = j0; j < j1; ++j)
        if (v[j].row >= 0) fn(v[j]);
    });
  };
  out.row_off.assign(nv + 1, 0);
  for_records([&](const Rec &r) { __atomic_fetch_add(&out.row_off[r.row + 1], 1u, __ATOMIC_RELAXED); });
  total = 0;
  for (int64_t p = 0; p < nv; ++p) {
    total += out.row_off[p + 1];
    if (total >= ((int64_t)1 << 32)) {
      err = "interception table exceeds 2^32 entries";
      return 9;
    }
    out.row_off[p + 1] += out.row_off[p];
  }
  std::unique_ptr<Rec[]> all(new Rec[total > 0 ? total : 1]);  // filled below, no zeroing
  {
    std::vector<uint32_t> fill(out.row_off.begin(), out.row_off.end() - 1);
    for_records([&](const Rec &r) {
      all[__atomic_fetch_add(&fill[r.row], 1u, __ATOMIC_RELAXED)] = r;
    });
  }
  tls.clear();
  std::vector<Rec>().swap(drec);
  // spatial order inside every row (Morton code of the box centre within the
  // union of the row's boxes), then chunks of kChunk consecutive entries
  auto spread = [](uint32_t v) {
    v &= 0x3ff;
    v = (v | (v << 16)) & 0x030000FF;
    v = (v | (v << 8)) & 0x0300F00F;
    v = (v | (v << 4)) & 0x030C30C3;
    v = (v | (v << 2)) & 0x09249249;
    return v;
  };
  // per thread: (Morton key << 32 | typed id, position) of a row, and the
  // row in that order (typed ids are distinct in a row: a total order)
  std::vector<std::vector<std::pair<uint64_t, uint32_t>>> sort_keys(threads);
  std::vector<std::vector<Rec>> sort_tmp(threads);
  const bool fail_packing = inject_at("packing");
  parallel_for(nv, threads, 1024, [&](int64_t p, int t) {
    if (fail_packing && p == nv / 2) throw std::bad_alloc();
    Rec *b = all.get() + out.row_off[p], *e = all.get() + out.row_off[p + 1];
    if (e - b < 2) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (Rec *it = b; it != e; ++it)
      for (int d = 0; d < 3; ++d) {
        float c = 0.5f * (it->box[d] + it->box[3 + d]);
        lo[d] = std::min(lo[d], c);
        hi[d] = std::max(hi[d], c);
      }
    auto key = [&](const Rec &r) {
      uint32_t k[3];
      for (int d = 0; d < 3; ++d) {
        float ext = hi[d] - lo[d];
        float u = ext > 0 ? (0.5f * (r.box[d] + r.box[3 + d]) - lo[d]) / ext : 0.f;
        k[d] = (uint32_t)std::min(1023.f, std::max(0.f, u * 1024.f));
      }
      return spread(k[0]) | (spread(k[1]) << 1) | (spread(k[2]) << 2);
    };
    auto &ks = sort_keys[t];
    ks.resize(e - b);
    for (int64_t j = 0; j < e - b; ++j)
      ks[j] = {(uint64_t)key(b[j]) << 32 | (uint32_t)b[j].tid, (uint32_t)j};
    std::sort(ks.begin(), ks.end());
    auto &row_copy = sort_tmp[t];
    row_copy.assign(b, e);
    for (size_t j = 0; j < ks.size(); ++j) b[j] = row_copy[ks[j].second];
  });
  sort_keys.clear();
  sort_tmp.clear();
  for (int64_t p = 0; p < nv; ++p) maxl = std::max<int64_t>(maxl, out.row_off[p + 1] - out.row_off[p]);

  // ---- chunks of every row, and the 15-bit box codes (quant.h)
  out.chunk_off.assign(nv + 1, 0);
  for (int64_t p = 0; p < nv; ++p) {
    uint32_t len = out.row_off[p + 1] - out.row_off[p];
    out.chunk_off[p + 1] = out.chunk_off[p] + (len + Layout::kChunk - 1) / Layout::kChunk;
  }
  out.chunks.assign(4 * (size_t)out.chunk_off[nv], 0u);
  out.entries.assign(4 * (size_t)total, 0u);
  parallel_for(nv, threads, 1024, [&](int64_t p, int) {
    uint32_t c = out.chunk_off[p];
    for (uint32_t j = out.row_off[p]; j < out.row_off[p + 1]; j += Layout::kChunk, ++c) {
      uint32_t cnt = std::min<uint32_t>(Layout::kChunk, out.row_off[p + 1] - j);
      float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (uint32_t k = j; k < j + cnt; ++k)
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::min(lo[d], all[k].box[d]);
          hi[d] = std::max(hi[d], all[k].box[3 + d]);
        }
      // chunk codes: the entries' hull, two codes wider on each side, so
      // that an entry test that passes implies a chunk test that passes
      // (the entry frame is never coarser than this one)
      uint32_t cl[3], ch[3];
      for (int d = 0; d < 3; ++d) {
        const uint32_t a = q_code(lo[d], out.qframe_lo[d], out.qframe_inv[d]);
        const uint32_t b = q_code(hi[d], out.qframe_lo[d], out.qframe_inv[d]);
        cl[d] = a >= 2 ? a - 2 : 0;
        ch[d] = std::min(kQMax, b + 2);
      }
      uint32_t *cw = &out.chunks[4 * (size_t)c];
      q_words(cl, ch, cw);
      // entry frame: origin from the chunk codes, scale inv_g * 2^e with the
      // largest e that keeps the entries clear of the frame's top code
      float clo[3], cinv[3];
      uint32_t w3 = 0;
      for (int d = 0; d < 3; ++d) {
        clo[d] = q_chunk_lo(cl[d], qstep[d], qbase[d]);
        const double ext = std::max((double)hi[d] - (double)clo[d], 0.0);
        uint32_t e = 0;
        while (e < 60 && ext * (double)out.qframe_inv[d] * std::ldexp(1.0, (int)e + 1) <=
                             (double)(kQMax - 64))
          ++e;
        w3 |= e << (8 * d);
      }
      cw[3] = w3;
      for (int d = 0; d < 3; ++d) cinv[d] = q_chunk_inv(out.qframe_inv[d], w3, d);
      for (uint32_t k = j; k < j + cnt; ++k) {
        uint32_t *ew = &out.entries[4 * (size_t)k];
        ew[0] = (uint32_t)all[k].tid;
        uint32_t el[3], eh[3];
        for (int d = 0; d < 3; ++d) {
          el[d] = q_code(all[k].box[d], clo[d], cinv[d]);
          eh[d] = q_code(all[k].box[3 + d], clo[d], cinv[d]);
          // inside the frame, never clamped: queries far outside fail
          if (el[d] < 1 || eh[d] >= kQMax) ++bad_boxes;
        }
        q_words(el, eh, ew + 1);
      }
    }
  });
  // second level: codes of every kChunk consecutive chunks of a row (their
  // hull, so a chunk that passes lies in a super-chunk that passes)
  out.super_off.assign(nv + 1, 0);
  for (int64_t p = 0; p < nv; ++p) {
    uint32_t nc = out.chunk_off[p + 1] - out.chunk_off[p];
    out.super_off[p + 1] = out.super_off[p] + (nc + Layout::kChunk - 1) / Layout::kChunk;
  }
  out.supers.assign(4 * (size_t)out.super_off[nv], 0u);
  parallel_for(nv, threads, 1024, [&](int64_t p, int) {
    uint32_t sidx = out.super_off[p];
    for (uint32_t c = out.chunk_off[p]; c < out.chunk_off[p + 1]; c += Layout::kChunk, ++sidx) {
      uint32_t ce = std::min<uint32_t>(c + Layout::kChunk, out.chunk_off[p + 1]);
      uint32_t sl[3] = {kQMax, kQMax, kQMax}, sh[3] = {0, 0, 0};
      for (uint32_t k = c; k < ce; ++k) {
        uint32_t cl[3], ch[3];
        q_unwords(&out.chunks[4 * (size_t)k], cl, ch);
        for (int d = 0; d < 3; ++d) {
          sl[d] = std::min(sl[d], cl[d]);
          sh[d] = std::max(sh[d], ch[d]);
        }
      }
      q_words(sl, sh, &out.supers[4 * (size_t)sidx]);
    }
  });
  }  // host packing
  if (bad_boxes.load()) {
    err = "internal error: a Region box does not fit the code frame of its chunk";
    return 5;
  }

  // ---- geometry records
  out.edges = M.E;
  out.edge_rec.resize(8 * M.ne);
  for (int64_t e = 0; e < M.ne; ++e) {
    const float *a = Vin + 3 * M.E[2 * e], *b = Vin + 3 * M.E[2 * e + 1];
    float dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    double l2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
    float *o = &out.edge_rec[8 * e];
    o[0] = a[0]; o[1] = a[1]; o[2] = a[2]; o[3] = (float)(1.0 / l2);
    o[4] = dx; o[5] = dy; o[6] = dz; o[7] = 0.f;
  }
  out.face_rec.resize(12 * nf);
  out.tris.resize(4 * nf);
  int64_t ndeg = 0;
  for (int64_t f = 0; f < nf; ++f) {
    const float *a = Vin + 3 * M.F[3 * f], *b = Vin + 3 * M.F[3 * f + 1], *c = Vin + 3 * M.F[3 * f + 2];
    double e1[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
    double e2[3] = {(double)c[0] - a[0], (double)c[1] - a[1], (double)c[2] - a[2]};
    double d00 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    double d01 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    double d11 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    double den = d00 * d11 - d01 * d01;
    float *o = &out.face_rec[12 * f];
    o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
    o[4] = (float)e1[0]; o[5] = (float)e1[1]; o[6] = (float)e1[2];
    o[8] = (float)e2[0]; o[9] = (float)e2[1]; o[10] = (float)e2[2];
    if (M.degenerate[f]) {
      ++ndeg;
      o[3] = o[7] = o[11] = std::numeric_limits<float>::quiet_NaN();
    } else {
      o[3] = (float)(d11 / den);
      o[7] = (float)(d01 / den);
      o[11] = (float)(d00 / den);
    }
    for (int k = 0; k < 3; ++k) out.tris[4 * f + k] = M.F[3 * f + k];
    out.tris[4 * f + 3] = 0;
  }
  out.n_entries = total;
  out.max_list = maxl;
  out.neighbour_pairs = npairs;
  out.inspections = insp;
  out.cert_rounds = rounds;
  out.cert_queries = cert_queries;
  out.n_degenerate = ndeg;
  const double t_end = now_ms();
  if (trace) std::fprintf(stderr, "p2m build: packing %.0f ms\n", t_end - t_pack);
  out.ms_total = t_end - t_start;
  out.ms_cells = t_flood - t_cells;
  out.ms_inspect = t_end - t_flood;
  return 0;
}

}  // namespace p2m
