// flood_core.h -- the flooding inspection of one primitive (Alg. 1) as the
// host builder runs it, and the types, flat problem view and cut primitive
// that the device kernel's warp version (flood_warp.h) shares with it.
//
// For a primitive p (an edge or a face) the flood starts at p's vertices and
// visits Voronoi neighbours breadth first.  At each visited vertex v it forms
// ConvexPoly(v, p) = Cell(v) ∩ Space-perp(p) by cutting v's widened cell with
// p's half-spaces (Sec. 4.4), applies the relaxed filter of Thm. 5/6 at the
// polytope's corners, and for an intercepting pair emits the Region box of
// Sec. 4.6: the corners where the filter function is positive plus a tight
// bracket of the filter's zero along every polytope edge that changes sign
// (edge_crossing), widened by delta and rounded outward to float32.  Only
// intercepting vertices spread the flood.
//
// Every step is plain IEEE double arithmetic (+, -, *, /, sqrt) in a fixed
// order, and both compilers are told not to fuse multiply-adds, so the warp
// version computes every value as this one does and the records agree bit
// for bit.  The work buffers have
// fixed capacities; a primitive that would overflow one, or whose cap loop
// cannot be chained point to point, is given up (return 1) and its caller
// floods it with unbounded host code.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define P2M_HD __host__ __device__ __forceinline__
#else
#define P2M_HD inline
#endif

namespace p2m {
namespace fc {

struct D3 {
  double x, y, z;
};
P2M_HD D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
P2M_HD D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
P2M_HD D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
P2M_HD double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
P2M_HD D3 cross(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
P2M_HD double len2(D3 a) { return dot(a, a); }
P2M_HD bool lex_less(D3 a, D3 b) {
  if (a.x != b.x) return a.x < b.x;
  if (a.y != b.y) return a.y < b.y;
  return a.z < b.z;
}
// Order-preserving 64-bit key of a double that is not NaN: its bits with the
// sign flipped so that the keys order like the values (+0 and -0 share one
// key, as they compare equal).  Comparisons of keys run on the integer units
// instead of the double-precision pipe.
P2M_HD uint64_t order_key(double v) {
  uint64_t u;
  memcpy(&u, &v, 8);
  if (u == 0x8000000000000000ull) u = 0;
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
P2M_HD bool dless(double a, double b) { return order_key(a) < order_key(b); }
// the selection rules of std::min / std::max (first argument on ties),
// compared on the keys
P2M_HD double dmin(double a, double b) { return dless(b, a) ? b : a; }
P2M_HD double dmax(double a, double b) { return dless(a, b) ? b : a; }

// Where the filter crosses zero on one polytope edge x(t) = x0 + t (x1 - x0),
// 0 <= t <= 1, whose end values g(x0), g(x1) lie on opposite sides of zero
// (pos0: g(x0) > 0).  Along the edge the filter is the quadratic
// p(t) = (A t + B) t + C with A >= 0 (its Hessian is positive semidefinite),
// so the sign change brackets exactly one root.  The root's closed form
// (the quadratic formula in its stable form) is tried first: a bracket 2^-40
// of the edge wide around it is taken when p has the end values' signs at
// its ends.  Otherwise the root is enclosed by a regula falsi iteration that
// keeps the bracket, with the Illinois rule (the retained end's value is
// halved when the same end is kept twice), until the bracket is 2^-40 of
// the edge or 64 steps have passed.  [*ta, *tb] receives the bracket.  The caller adds the points at both ends of the bracket to
// the Region box: their box contains the segment between them, hence the
// crossing, whatever the rounding of p.  If p disagrees with the end values
// at an end (rounding at a crossing that close to it) that end is returned
// as a zero-width bracket.
P2M_HD void edge_crossing(double A, double B, double C, bool pos0, double *ta, double *tb) {
  const double sg = pos0 ? 1.0 : -1.0;  // f = sg * p: positive at t = 0
  double lo = 0.0, hi = 1.0;
  double flo = sg * C, fhi = sg * ((A + B) + C);
  if (!(flo > 0.0)) {
    *ta = *tb = 0.0;
    return;
  }
  if (fhi > 0.0) {
    *ta = *tb = 1.0;
    return;
  }
  // The root from the quadratic formula in its stable form (the larger-
  // magnitude root as q / A, the other as C / q), bracketed 2^-40 wide and
  // accepted when the signs of p at the bracket's ends confirm it; where they
  // do not (rounding near a double root, say) the iteration below runs.
  {
    double t = -1.0;
    if (A == 0.0) {
      if (B != 0.0) t = -C / B;
    } else {
      const double disc = B * B - 4.0 * A * C;
      if (disc >= 0.0) {
        const double sq = sqrt(disc);
        const double q = -0.5 * (B >= 0.0 ? B + sq : B - sq);
        if (q != 0.0) {
          const double r1 = q / A, r2 = C / q;
          t = (r1 > 0.0 && r1 < 1.0) ? r1 : r2;
        }
      }
    }
    if (t > 0.0 && t < 1.0) {
      double a = t - 0x1p-41, b = t + 0x1p-41;
      if (!(a > 0.0)) a = 0.0;
      if (!(b < 1.0)) b = 1.0;
      const double fa = sg * ((A * a + B) * a + C), fb = sg * ((A * b + B) * b + C);
      if (fa > 0.0 && !(fb > 0.0)) {
        *ta = a;
        *tb = b;
        return;
      }
    }
  }
  int kept = 0;  // +1: lo moved last, -1: hi moved last
  for (int it = 0; it < 64 && hi - lo > 0x1p-40; ++it) {
    double t = (lo * fhi - hi * flo) / (fhi - flo);
    if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
    const double ft = sg * ((A * t + B) * t + C);
    if (ft > 0.0) {
      lo = t;
      flo = ft;
      if (kept == 1) fhi *= 0.5;
      kept = 1;
    } else {
      hi = t;
      fhi = ft;
      if (kept == -1) flo *= 0.5;
      kept = -1;
    }
  }
  *ta = lo;
  *tb = hi;
}

// half-space n.x <= c
struct HS {
  D3 n;
  double c;
};

constexpr int kMaxF = 96;    // faces of a work polytope
constexpr int kMaxP = 512;   // loop points of a work polytope (or of a cell)
constexpr int kMaxPerp = 16; // Space-perp half-spaces of one primitive

// work polytope: face f's loop is pt[beg[f] .. beg[f+1]); src[f] is the id
// of whatever generated face f's plane (kept by cut for the Voronoi cells,
// whose neighbours are the generators of their faces)
struct WPoly {
  int nf, np;
  int32_t beg[kMaxF + 1];
  int32_t src[kMaxF];
  D3 pt[kMaxP];
};

// read-only polytope: a cell in the caller's storage or a work polytope
// (src: the faces' generators, or null where nobody needs them)
struct PView {
  const D3 *pt;
  const int32_t *beg;  // nf + 1 loop starts
  int nf, np;
  const int32_t *src;
};
P2M_HD PView view(const WPoly &w) { return {w.pt, w.beg, w.nf, w.np, w.src}; }

struct Work {
  WPoly A, B;
  double s[kMaxP];  // signed distances in a cut; the filter values afterwards
  D3 seg_in[kMaxF], seg_out[kMaxF];
  uint8_t used[kMaxF];
};

// what the flooding of one primitive needs
struct Prim {
  HS perp[kMaxPerp];  // Space-perp(p), widened by delta
  int np;
  int gtype;          // 1: line through ga with unit direction gu; 2: plane through ga, unit normal gu
  D3 ga, gu;
  int32_t seed_row[3], seed_vid[3];  // its vertices: table rows and vertex ids
  int ns;
  int32_t tid;        // typed id, type << 30 | id
};

// The flooding problem in flat arrays, read the same way on both sides.
// Rows are KD-tree positions.  Cell p: points pt[pt_off[p] .. pt_off[p+1]),
// its nf face loops starting at the offsets beg[beg_off[p] ..
// beg_off[p+1]) relative to its first point (nf + 1 of them, the last one
// the point count).  Primitive i: half-spaces perp[perp_off[i] ..
// perp_off[i+1]) as (n, c) quadruples, filter geometry g[6i .. 6i+6) (a,
// unit u) of type gtype[i], seeds seed_row / seed_vid[3i ..] (2 for an
// edge, 3 for a face) and typed id tid[i].
struct Flat {
  const int64_t *pt_off;
  const D3 *pt;
  const int64_t *beg_off;
  const int32_t *beg;
  const D3 *pos;        // vertex positions by row
  const int32_t *vids;  // vertex ids by row
  const uint32_t *nbo, *nbs;  // Voronoi neighbours (rows), CSR by row
  const int64_t *perp_off;
  const double *perp;
  const int32_t *gtype;
  const double *g;
  const int32_t *seed_row, *seed_vid, *tid;

  P2M_HD PView cell(int32_t p) const {
    const int64_t b0 = beg_off[p], p0 = pt_off[p];
    return {pt + p0, beg + b0, (int)(beg_off[p + 1] - b0 - 1), (int)(pt_off[p + 1] - p0),
            nullptr};
  }
  P2M_HD D3 pv(int32_t p) const { return pos[p]; }
  P2M_HD int32_t vid(int32_t p) const { return vids[p]; }
  P2M_HD int64_t nb_begin(int32_t p) const { return nbo[p]; }
  P2M_HD int64_t nb_end(int32_t p) const { return nbo[p + 1]; }
  P2M_HD int32_t nb(int64_t j) const { return (int32_t)nbs[j]; }
  // primitive i as the core takes it; false if it has too many half-spaces
  P2M_HD bool load(int64_t i, Prim &P) const {
    const int64_t j0 = perp_off[i], np = perp_off[i + 1] - j0;
    if (np < 0 || np > kMaxPerp) return false;
    P.np = (int)np;
    for (int j = 0; j < P.np; ++j) {
      const double *h = perp + 4 * (j0 + j);
      P.perp[j] = {{h[0], h[1], h[2]}, h[3]};
    }
    P.gtype = gtype[i];
    P.ga = {g[6 * i], g[6 * i + 1], g[6 * i + 2]};
    P.gu = {g[6 * i + 3], g[6 * i + 4], g[6 * i + 5]};
    P.ns = P.gtype == 1 ? 2 : 3;
    for (int k = 0; k < 3; ++k) {
      P.seed_row[k] = seed_row[3 * i + k];
      P.seed_vid[k] = seed_vid[3 * i + k];
    }
    P.tid = tid[i];
    return true;
  }
};

enum { kCutNone = 0, kCutDone = 1, kCutGiveUp = 2 };

// crossing of segment ab with the plane, computed from the lexicographically
// smaller end so that the two faces sharing the segment get the same point
P2M_HD D3 crossing(D3 a, D3 b, double sa, double sb) {
  if (lex_less(b, a)) {
    D3 t = a;
    a = b;
    b = t;
    double u = sa;
    sa = sb;
    sb = u;
  }
  double t = sa / (sa - sb);
  return a + t * (b - a);
}

// Cut `in` by the half-space n.x <= c into `out`: every loop is clipped and
// the hole is closed by a cap face chained from the loops' exit and entry
// points.  kCutNone: nothing lies beyond (out untouched); kCutDone: out
// holds the result (no faces when emptied); kCutGiveUp: a capacity would be
// exceeded or the cap could not be chained.  A kept face keeps its
// generator (in.src, -1 without one), the cap gets hsrc.
P2M_HD int cut(PView in, D3 hn, double hc, double eps, WPoly &out, Work &W,
               int32_t hsrc = -1) {
  if (in.np > kMaxP) return kCutGiveUp;
  bool beyond = false, within = false;
  for (int i = 0; i < in.np; ++i) {
    double s = dot(hn, in.pt[i]) - hc;
    W.s[i] = s;
    beyond |= s > eps;
    within |= s < -eps;
  }
  if (!beyond) return kCutNone;
  out.nf = 0;
  out.np = 0;
  out.beg[0] = 0;
  if (!within) return kCutDone;
  int m = 0;
  for (int f = 0; f < in.nf; ++f) {
    const int b = in.beg[f], k = in.beg[f + 1] - b;
    const int start = out.np;
    bool has_x = false, has_y = false;
    D3 X{0, 0, 0}, Y{0, 0, 0};
    for (int i = 0; i < k; ++i) {
      const int ia = b + i, ib = b + (i + 1) % k;
      const double sa = W.s[ia], sb = W.s[ib];
      const bool ka = sa <= eps, kb = sb <= eps;
      if (ka) {
        if (out.np >= kMaxP) return kCutGiveUp;
        out.pt[out.np++] = in.pt[ia];
      }
      if (ka && !kb) {  // leaving the kept side
        if (sa >= -eps) {
          X = in.pt[ia];
        } else {
          X = crossing(in.pt[ia], in.pt[ib], sa, sb);
          if (out.np >= kMaxP) return kCutGiveUp;
          out.pt[out.np++] = X;
        }
        has_x = true;
      } else if (!ka && kb) {  // coming back
        if (sb >= -eps) {
          Y = in.pt[ib];
        } else {
          Y = crossing(in.pt[ia], in.pt[ib], sa, sb);
          if (out.np >= kMaxP) return kCutGiveUp;
          out.pt[out.np++] = Y;
        }
        has_y = true;
      }
    }
    if (out.np - start >= 3) {
      if (out.nf >= kMaxF) return kCutGiveUp;
      out.src[out.nf] = in.src ? in.src[f] : -1;
      out.beg[++out.nf] = out.np;
    } else {
      out.np = start;
    }
    if (has_x && has_y && len2(X - Y) > eps * eps) {
      if (m >= kMaxF) return kCutGiveUp;
      W.seg_in[m] = Y;
      W.seg_out[m] = X;
      ++m;
    }
  }
  // the cap loop: each face walks X -> Y along the plane, the cap Y -> X
  if (m >= 3) {
    for (int j = 0; j < m; ++j) W.used[j] = 0;
    if (out.np + m > kMaxP || out.nf >= kMaxF) return kCutGiveUp;
    out.pt[out.np++] = W.seg_in[0];
    D3 cur = W.seg_out[0];
    W.used[0] = 1;
    for (int step = 1; step < m; ++step) {
      out.pt[out.np++] = cur;
      int best = -1;
      double bd = INFINITY;
      for (int j = 0; j < m; ++j)
        if (!W.used[j]) {
          double d = len2(W.seg_in[j] - cur);
          if (d < bd) {
            bd = d;
            best = j;
          }
        }
      if (best < 0 || bd > 1e6 * eps * eps) return kCutGiveUp;
      W.used[best] = 1;
      cur = W.seg_out[best];
    }
    if (!(len2(cur - W.seg_in[0]) <= 1e6 * eps * eps)) return kCutGiveUp;
    out.src[out.nf] = hsrc;
    out.beg[++out.nf] = out.np;
  }
  if (out.nf < 4) {
    out.nf = 0;
    out.np = 0;
  }
  return kCutDone;
}

// Flood primitive P.  Env supplies the mesh side (Flat's accessors):
//   PView cell(row), D3 pv(row), int32_t vid(row),
//   int64_t nb_begin(row), nb_end(row), int32_t nb(j)  (Voronoi neighbours),
// and the caller's side:
//   void mark_seed(row), bool mark(row, queue, tail)   (true when first seen),
//   void emit(row, tid, const float box[6]).
// queue holds qcap rows.  Returns 0 when done (insp = vertices inspected),
// 1 when given up (records already emitted for P must be dropped).
template <class Env>
P2M_HD int flood_prim(const Prim &P, double eps, double delta, double eta, Env &env, Work &W,
                      int32_t *queue, int64_t qcap, int64_t &insp) {
  int64_t head = 0, tail = 0;
  insp = 0;
  if (qcap < P.ns) return 1;
  for (int s = 0; s < P.ns; ++s) {
    env.mark_seed(P.seed_row[s]);
    queue[tail++] = P.seed_row[s];
  }
  while (head < tail) {
    const int32_t p = queue[head++];
    ++insp;
    const PView cell = env.cell(p);
    // a half-space with every point of the cell beyond it empties the
    // result whatever the order of the cuts
    bool emptied = false;
    for (int j = 0; j < P.np && !emptied; ++j) {
      bool all_beyond = true;
      for (int q = 0; q < cell.np; ++q)
        if (!(dot(P.perp[j].n, cell.pt[q]) - P.perp[j].c > eps)) {
          all_beyond = false;
          break;
        }
      emptied = all_beyond && cell.np > 0;
    }
    if (emptied) continue;
    PView cur = cell;
    WPoly *bufs[2] = {&W.A, &W.B};
    int wsel = 0;
    for (int j = 0; j < P.np && cur.nf > 0; ++j) {
      const int r = cut(cur, P.perp[j].n, P.perp[j].c, eps, *bufs[wsel], W);
      if (r == kCutGiveUp) return 1;
      if (r == kCutDone) {
        cur = view(*bufs[wsel]);
        wsel ^= 1;
      }
    }
    if (cur.nf == 0) continue;
    if (cur.np > kMaxP) return 1;
    const D3 pv = env.pv(p);
    const int32_t vid = env.vid(p);
    bool keep = (P.gtype == 1)
                    ? (P.seed_vid[0] == vid || P.seed_vid[1] == vid)
                    : (P.seed_vid[0] == vid || P.seed_vid[1] == vid || P.seed_vid[2] == vid);
    double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
    bool have = false;
    // the filter function |x-v|^2 - Dist(x)^2 + eta at every loop point
    double *gv = W.s;
    for (int q = 0; q < cur.np; ++q) {
      const D3 x = cur.pt[q];
      const D3 w = x - P.ga;
      const double s = dot(w, P.gu);
      const double dist2 = P.gtype == 1 ? len2(w) - s * s : s * s;
      gv[q] = len2(x - pv) - dist2 + eta;
    }
    for (int f = 0; f < cur.nf; ++f) {
      const int b0 = cur.beg[f], k = cur.beg[f + 1] - b0;
      for (int q = 0; q < k; ++q) {
        const D3 x0 = cur.pt[b0 + q], x1 = cur.pt[b0 + (q + 1) % k];
        const double g0 = gv[b0 + q], g1 = gv[b0 + (q + 1) % k];
        if (g0 > 0) {
          keep = true;
          blo[0] = dmin(blo[0], x0.x); bhi[0] = dmax(bhi[0], x0.x);
          blo[1] = dmin(blo[1], x0.y); bhi[1] = dmax(bhi[1], x0.y);
          blo[2] = dmin(blo[2], x0.z); bhi[2] = dmax(bhi[2], x0.z);
          have = true;
        }
        if ((g0 > 0) != (g1 > 0)) {
          // the filter along the edge is a quadratic in t: bracket its zero
          const D3 d = x1 - x0, w0 = x0 - P.ga, r0 = x0 - pv;
          const double du = dot(d, P.gu), wu = dot(w0, P.gu);
          double A, B, Cc;
          if (P.gtype == 1) {  // |x-v|^2 - (|w|^2 - (w.u)^2)
            A = len2(d) - (len2(d) - du * du);
            B = 2 * dot(r0, d) - 2 * (dot(w0, d) - wu * du);
            Cc = len2(r0) - (len2(w0) - wu * wu) + eta;
          } else {             // |x-v|^2 - (w.u)^2
            A = len2(d) - du * du;
            B = 2 * dot(r0, d) - 2 * wu * du;
            Cc = len2(r0) - wu * wu + eta;
          }
          double tb[2];
          edge_crossing(A, B, Cc, g0 > 0, &tb[0], &tb[1]);
          for (int r = 0; r < 2; ++r) {
            const D3 x = x0 + tb[r] * d;
            blo[0] = dmin(blo[0], x.x); bhi[0] = dmax(bhi[0], x.x);
            blo[1] = dmin(blo[1], x.y); bhi[1] = dmax(bhi[1], x.y);
            blo[2] = dmin(blo[2], x.z); bhi[2] = dmax(bhi[2], x.z);
            have = true;
          }
        }
      }
    }
    if (!keep) continue;
    if (!have)
      for (int q = 0; q < cur.np; ++q) {
        const D3 x = cur.pt[q];
        blo[0] = dmin(blo[0], x.x); bhi[0] = dmax(bhi[0], x.x);
        blo[1] = dmin(blo[1], x.y); bhi[1] = dmax(bhi[1], x.y);
        blo[2] = dmin(blo[2], x.z); bhi[2] = dmax(bhi[2], x.z);
      }
    float box[6];
    for (int d = 0; d < 3; ++d) {
      float l = (float)(blo[d] - delta), h = (float)(bhi[d] + delta);
      if ((double)l > blo[d] - delta) l = nextafterf(l, -INFINITY);
      if ((double)h < bhi[d] + delta) h = nextafterf(h, INFINITY);
      box[d] = l;
      box[3 + d] = h;
    }
    env.emit(p, P.tid, box);
    for (int64_t j = env.nb_begin(p); j < env.nb_end(p); ++j) {
      const int32_t w = env.nb(j);
      if (env.mark(w, queue, tail)) {
        if (tail >= qcap) return 1;
        queue[tail++] = w;
      }
    }
  }
  return 0;
}

}  // namespace fc
}  // namespace p2m
