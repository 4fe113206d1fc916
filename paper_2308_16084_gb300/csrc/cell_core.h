// cell_core.h -- the pieces of the builder's Voronoi-cell stage (Alg. A.1's
// cells, clipped to D) that the host builder's steps fix and the device's
// warp version (cell_warp.h) takes as they are: the cell box, the bisector
// half-space, the 32-nearest search with the host's traversal (so that
// equal distances keep the host's order), and the corner order used to sort
// and deduplicate a cell's corners.  Every value is plain IEEE double
// arithmetic in the host's order, compiled without fused multiply-adds on
// both sides.
#pragma once

#include <cstring>

#include "flood_core.h"

namespace p2m {
namespace cc {

using fc::D3;
using fc::dot;
using fc::len2;

constexpr int kSeedK = 32;     // nearest vertices whose bisectors seed a cell
constexpr int kRounds = 65;    // certification rounds at most
constexpr int kApplied = 256;  // bisectors one cell may apply
constexpr int kKnnStack = 128;

// what every cell shares: the domain D, the cut tolerance eps, the
// certification slack epsc on squared distances and the widening delta
struct CellParams {
  double lo[3], hi[3];
  double eps, epsc, delta;
};

enum { kCellOk = 0, kCellGiveUp = 1 };

// the box lo..hi as a polytope: faces +x, -x, +y, -y, +z, -z (generators
// -1 .. -6), each loop counter-clockwise seen from outside
template <class Poly>
P2M_HD void make_box(Poly &p, const double lo[3], const double hi[3]) {
  const double X0 = lo[0], Y0 = lo[1], Z0 = lo[2], X1 = hi[0], Y1 = hi[1], Z1 = hi[2];
  const D3 pts[24] = {{X1, Y0, Z0}, {X1, Y1, Z0}, {X1, Y1, Z1}, {X1, Y0, Z1},
                      {X0, Y0, Z0}, {X0, Y0, Z1}, {X0, Y1, Z1}, {X0, Y1, Z0},
                      {X0, Y1, Z0}, {X0, Y1, Z1}, {X1, Y1, Z1}, {X1, Y1, Z0},
                      {X0, Y0, Z0}, {X1, Y0, Z0}, {X1, Y0, Z1}, {X0, Y0, Z1},
                      {X0, Y0, Z1}, {X1, Y0, Z1}, {X1, Y1, Z1}, {X0, Y1, Z1},
                      {X0, Y0, Z0}, {X0, Y1, Z0}, {X1, Y1, Z0}, {X1, Y0, Z0}};
  for (int i = 0; i < 24; ++i) p.pt[i] = pts[i];
  for (int f = 0; f <= 6; ++f) p.beg[f] = 4 * f;
  for (int f = 0; f < 6; ++f) p.src[f] = -1 - f;
  p.nf = 6;
  p.np = 24;
}

// bisector half-space n.x <= c of vertices pa (own side) and pb, pushed out
// by w
P2M_HD void bisector(D3 pa, D3 pb, double w, D3 &n, double &c) {
  const D3 d = pb - pa;
  const double l = sqrt(len2(d));
  n = (1.0 / l) * d;
  c = 0.5 * (dot(n, pa) + dot(n, pb)) + w;
}

P2M_HD double box_d2(const double b[6], D3 q) {
  const double dx = q.x < b[0] ? b[0] - q.x : (q.x > b[3] ? q.x - b[3] : 0.0);
  const double dy = q.y < b[1] ? b[1] - q.y : (q.y > b[4] ? q.y - b[4] : 0.0);
  const double dz = q.z < b[2] ? b[2] - q.z : (q.z > b[5] ? q.z - b[5] : 0.0);
  return dx * dx + dy * dy + dz * dz;
}

using fc::order_key;

// corners are ranked and deduplicated on order_key: the integer comparison
// gives the order and equality of the doubles
P2M_HD bool corner_less(const D3 &a, const D3 &b) {
  const uint64_t ax = order_key(a.x), bx = order_key(b.x);
  if (ax != bx) return ax < bx;
  const uint64_t ay = order_key(a.y), by = order_key(b.y);
  if (ay != by) return ay < by;
  return order_key(a.z) < order_key(b.z);
}

P2M_HD bool corner_same(const D3 &a, const D3 &b) {
  return a.x == b.x && a.y == b.y && a.z == b.z;
}

// The 32 nearest tree positions to q other than self, ascending, with the
// host's traversal (nearer child first, a subtree entered while it may
// still hold a nearer point), so that equal distances keep the host's
// order.  Env: nleaf0() (internal nodes), leaf_first(j), pos(p),
// child_boxes(node, b0, b1).  Returns the count, -1 if the stack would
// overflow.
template <class Env>
P2M_HD int k_nearest(const Env &env, D3 q, int64_t self, int64_t *ids, double *d2s) {
  const int k = kSeedK;
  int64_t st_node[kKnnStack];
  double st_d2[kKnnStack];
  int sp = 0, cnt = 0;
  st_node[sp] = 0;
  st_d2[sp++] = 0.0;  // the root's distance is never compared (cnt is 0)
  const int64_t nleaf0 = env.nleaf0();
  while (sp) {
    --sp;
    const int64_t node = st_node[sp];
    const double nd2 = st_d2[sp];
    if (cnt == k && !(nd2 < d2s[k - 1])) continue;
    if (node >= nleaf0) {
      const int64_t j = node - nleaf0;
      for (int64_t p = env.leaf_first(j), e = env.leaf_first(j + 1); p < e; ++p) {
        if (p == self) continue;
        const double d = len2(env.pos(p) - q);
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
    int64_t c0 = 2 * node + 1, c1 = c0 + 1;
    double b0[6], b1[6];
    env.child_boxes(node, b0, b1);
    double d0 = box_d2(b0, q), d1 = box_d2(b1, q);
    if (d0 > d1) {
      const int64_t tc = c0;
      c0 = c1;
      c1 = tc;
      const double td = d0;
      d0 = d1;
      d1 = td;
    }
    if (sp + 2 > kKnnStack) return -1;
    if (cnt < k || d1 < d2s[cnt - 1]) {
      st_node[sp] = c1;
      st_d2[sp++] = d1;
    }
    if (cnt < k || d0 < d2s[cnt - 1]) {
      st_node[sp] = c0;
      st_d2[sp++] = d0;
    }
  }
  return cnt;
}

P2M_HD bool has_row(const int32_t *a, int n, int32_t w) {
  for (int i = 0; i < n; ++i)
    if (a[i] == w) return true;
  return false;
}

}  // namespace cc
}  // namespace p2m
