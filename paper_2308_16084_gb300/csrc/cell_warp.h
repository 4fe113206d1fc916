// cell_warp.h -- the Voronoi cell of one vertex clipped to the domain D
// (Alg. A.1's cells), made by the 32 lanes of a warp in the host builder's
// rounds.
//
// The steps and their order are the host builder's: the box D cut by the
// bisectors of the 32 nearest vertices (nearest first); then rounds in
// which every distinct corner farther from the vertex than half the 32nd
// distance asks the exact search for a vertex strictly nearer to it than
// the cell's own, and the cell is cut by the bisectors of the vertices found
// (not applied yet, first found first, then ordered by their distance to the
// cell's vertex, ties in that order), until no corner finds one or 65 rounds
// have passed.  The generators of the surviving faces are the vertex's
// Voronoi neighbours; the widened cell is the box D +- delta cut by their
// bisectors pushed out by delta, in face order.
//
// The phases here are what happens to one cell between the searches: the
// seeding (cell_seed), a round's distinct far corners (round_corners), the
// pick of the vertices found and their cuts (round_apply), and the widened
// cell (cell_widen).  The caller keeps each cell's state (CellSlot) between
// them and runs every round's searches for all cells at once.  Spread over
// the lanes: the cuts (fw::warp_cut: one point, then one face per lane) and
// the ranking and filtering of the corners (one corner per lane).  Lane 0
// runs the 32-nearest search and the pick.  Every value is the host's
// double-precision operation in the host's order (no fused multiply-adds on
// either side), so the cell equals the host builder's bit for bit; a cell
// whose polytope outgrows the warp's buffers, whose cap loop cannot be
// chained (the host then orders the cap by angle) or whose search gives up
// is handed back.  Sections as in flood_warp.h: compiled for the host, the
// lanes run one after another.
#pragma once

#include "cell_core.h"
#include "flood_warp.h"

namespace p2m {
namespace cw {

using fc::D3;
using fc::len2;

enum { kOpen = 0, kDone = 1, kGaveUp = 2 };

constexpr int kSettled = 192;  // settled corners a cell remembers

// one cell's state between the phases
struct CellSlot {
  fw::WPoly poly;                  // the cell so far
  int32_t applied[cc::kApplied];   // rows whose bisectors cut it
  int n_applied;
  int status;                      // kOpen, kDone or kGaveUp
  int rounds;                      // rounds in which it had far corners
  int m;                           // its far corners in the current round
  int64_t corner_at;               // where they are in the round's search list
  int64_t queries;                 // far corners searched over all rounds
  double safe2;                    // corners nearer than this need no search
  // far corners whose search found no vertex, or only one already applied:
  // the same corner (bit for bit) gets the same answer in a later round, so
  // it is not searched again
  D3 settled[kSettled];
  int n_settled;
};

// per-warp work space besides the cut's (fw::WarpWork)
struct CellExtra {
  D3 corner[fw::kWP];       // the polytope's points, then the round's far corners
  D3 sorted[fw::kWP];       // the points in corner order
  int32_t rank[fw::kWP];    // each point's place in that order, then the kept ones'
  int32_t keep[fw::kWP];    // 1: first of its run and beyond the safe radius
  int32_t cand[fw::kWP];
  double cand_d[fw::kWP];
  int64_t knn_id[cc::kSeedK];
  double knn_d2[cc::kSeedK];
  int32_t nb[fw::kWF];
  int nb_n, n_cand, m, k, flag;
  unsigned long long out_at[3];  // output offsets of a widened cell
};

P2M_HD fw::View slot_view(const CellSlot &c) { return fw::view_of(c.poly); }

// the polytope *w copied into the slot (lanes share the copy)
P2M_HD void store_poly(CellSlot &c, const fw::WPoly &w) {
  P2M_LANES(l)
    for (int i = l; i < w.np; i += 32) c.poly.pt[i] = w.pt[i];
    for (int f = l; f <= w.nf; f += 32) c.poly.beg[f] = w.beg[f];
    for (int f = l; f < w.nf; f += 32) c.poly.src[f] = w.src[f];
  P2M_END_LANES
  P2M_LANE0 {
    c.poly.nf = w.nf;
    c.poly.np = w.np;
  }
  P2M_SYNC;
}

// `in` cut by the bisector of rows p and w pushed out by `push` (cap
// generator w) into the warp buffer that `in` does not hold; when the cut
// changes the polytope, *cur becomes that buffer and `in` views it (*cur
// null: `in` is still the caller's polytope).  false: the cut gave up.
template <class Env>
P2M_HD bool bisector_cut(fw::WarpWork &S, const Env &env, fw::View &in, fw::WPoly *&cur,
                         int64_t p, int64_t w, double push, double eps) {
  D3 n;
  double c;
  cc::bisector(env.pos(p), env.pos(w), push, n, c);
  fw::WPoly *dst = (cur == &S.A) ? &S.B : &S.A;
  const int r = fw::warp_cut(S, in, n, c, eps, *dst, (int32_t)w);
  if (r == fw::kGiveUp) return false;
  if (r == fw::kDone) {
    cur = dst;
    in = fw::view_of(*cur);
  }
  return true;
}

// Seeding of row p's cell: the box D cut by the bisectors of the 32 nearest
// vertices, nearest first.  Env: as cc::k_nearest.
template <class Env>
P2M_HD void cell_seed(fw::WarpWork &S, CellExtra &X, const Env &env, int64_t p,
                      const cc::CellParams &cp, CellSlot &c) {
  const D3 pv = env.pos(p);
  P2M_LANE0 {
    cc::make_box(S.A, cp.lo, cp.hi);
    X.k = cc::k_nearest(env, pv, p, X.knn_id, X.knn_d2);
    c.status = kOpen;
    c.rounds = 0;
    c.queries = 0;
    c.m = 0;
    c.n_settled = 0;
  }
  P2M_SYNC;
  const int k = X.k;
  bool ok = k >= 0;
  fw::WPoly *cur = &S.A;
  fw::View in = fw::view_of(S.A);
  for (int i = 0; i < k && ok; ++i) ok = bisector_cut(S, env, in, cur, p, X.knn_id[i], 0.0, cp.eps);
  if (ok) store_poly(c, *cur);
  P2M_LANE0 {
    if (!ok) {
      c.status = kGaveUp;
    } else {
      for (int i = 0; i < k; ++i) c.applied[i] = (int32_t)X.knn_id[i];
      c.n_applied = k;
      // no vertex outside the 32 nearest can be nearer than p to a corner
      // within half the 32nd distance of p
      c.safe2 = k == cc::kSeedK ? 0.25 * X.knn_d2[cc::kSeedK - 1] : (double)INFINITY;
    }
  }
  P2M_SYNC;
}

// The distinct corners of the cell farther from its vertex pv than the safe
// radius, in corner order, into X.corner[0 .. m); returns m.
P2M_HD int round_corners(CellExtra &X, const CellSlot &c, D3 pv) {
  const fw::WPoly &P = c.poly;
  const int np = P.np;
  const double safe2 = c.safe2;
  // the points ranked in corner order (equal points by index)
  P2M_LANES(l)
    for (int i = l; i < np; i += 32) X.corner[i] = P.pt[i];
  P2M_END_LANES
  P2M_LANES(l)
    for (int i = l; i < np; i += 32) {
      const D3 a = X.corner[i];
      int r = 0;
      for (int j = 0; j < np; ++j) {
        const D3 b = X.corner[j];
        if (cc::corner_less(b, a) || (j < i && !cc::corner_less(a, b))) ++r;
      }
      X.rank[i] = r;
    }
  P2M_END_LANES
  P2M_LANES(l)
    for (int i = l; i < np; i += 32) X.sorted[X.rank[i]] = X.corner[i];
  P2M_END_LANES
  P2M_LANES(l)
    for (int j = l; j < np; j += 32) {
      const D3 x = X.sorted[j];
      const bool first = j == 0 || !cc::corner_same(x, X.sorted[j - 1]);
      X.keep[j] = (first && len2(x - pv) > safe2) ? 1 : 0;
    }
  P2M_END_LANES
  P2M_LANE0 {
    int m = 0;
    for (int j = 0; j < np; ++j) {
      X.rank[j] = m;
      m += X.keep[j];
    }
    X.m = m;
  }
  P2M_SYNC;
  P2M_LANES(l)
    for (int j = l; j < np; j += 32)
      if (X.keep[j]) X.corner[X.rank[j]] = X.sorted[j];
  P2M_END_LANES
  return X.m;
}

// bit-for-bit equality (a miss only costs a search)
P2M_HD bool same_bits(const D3 &a, const D3 &b) {
  uint64_t u[3], v[3];
  memcpy(u, &a, 24);
  memcpy(v, &b, 24);
  return u[0] == v[0] && u[1] == v[1] && u[2] == v[2];
}

// Of the round's far corners X.corner[0 .. m), the ones the cell has not
// settled in an earlier round, in order, into X.sorted[0 .. ms); returns ms.
P2M_HD int round_unsettled(CellExtra &X, const CellSlot &c, int m) {
  const int ns = c.n_settled;
  P2M_LANES(l)
    for (int j = l; j < m; j += 32) {
      const D3 x = X.corner[j];
      int known = 0;
      for (int t = 0; t < ns && !known; ++t) known = same_bits(x, c.settled[t]) ? 1 : 0;
      X.keep[j] = 1 - known;
    }
  P2M_END_LANES
  P2M_LANE0 {
    int ms = 0;
    for (int j = 0; j < m; ++j) {
      X.rank[j] = ms;
      ms += X.keep[j];
    }
    X.m = ms;
  }
  P2M_SYNC;
  P2M_LANES(l)
    for (int j = l; j < m; j += 32)
      if (X.keep[j]) X.sorted[X.rank[j]] = X.corner[j];
  P2M_END_LANES
  return X.m;
}

// After the round's searches (the cell's c.m searched corners xs[3i ..],
// wres[i] the answer for each, -2 where the search gave up): the vertices
// found that were not applied yet, first found first, then nearest first,
// cut into the cell; the corners that found none remembered as settled.  No
// vertex found: the cell is done.
template <class Env>
P2M_HD void round_apply(fw::WarpWork &S, CellExtra &X, const Env &env, int64_t p,
                        const cc::CellParams &cp, CellSlot &c, const double *xs,
                        const int64_t *wres) {
  const D3 pv = env.pos(p);
  P2M_LANE0 {
    int flag = 0, nc = 0;
    for (int i = 0; i < c.m; ++i) {
      const int64_t w = wres[i];
      if (w == -2) {
        flag = 1;
        break;
      }
      const bool applied = w >= 0 && cc::has_row(c.applied, c.n_applied, (int32_t)w);
      if (w >= 0 && w != p && !applied && !cc::has_row(X.cand, nc, (int32_t)w)) {
        X.cand[nc] = (int32_t)w;
        X.cand_d[nc] = len2(env.pos(w) - pv);
        ++nc;
      }
      if ((w == -1 || applied) && c.n_settled < kSettled)
        c.settled[c.n_settled++] = {xs[3 * i], xs[3 * i + 1], xs[3 * i + 2]};
    }
    for (int i = 1; i < nc; ++i) {
      const int32_t w = X.cand[i];
      const double d = X.cand_d[i];
      int j = i;
      while (j > 0 && d < X.cand_d[j - 1]) {
        X.cand[j] = X.cand[j - 1];
        X.cand_d[j] = X.cand_d[j - 1];
        --j;
      }
      X.cand[j] = w;
      X.cand_d[j] = d;
    }
    if (c.n_applied + nc > cc::kApplied) flag = 1;
    X.n_cand = nc;
    X.flag = flag;
    if (flag) c.status = kGaveUp;
    else if (nc == 0) c.status = kDone;
  }
  P2M_SYNC;
  if (X.flag || X.n_cand == 0) return;
  const int nc = X.n_cand;
  fw::WPoly *cur = nullptr;
  fw::View in = slot_view(c);
  bool ok = true;
  for (int i = 0; i < nc && ok; ++i) ok = bisector_cut(S, env, in, cur, p, X.cand[i], 0.0, cp.eps);
  if (ok && cur) store_poly(c, *cur);
  P2M_LANE0 {
    if (!ok) {
      c.status = kGaveUp;
    } else {
      for (int i = 0; i < nc; ++i) c.applied[c.n_applied + i] = X.cand[i];
      c.n_applied += nc;
    }
  }
  P2M_SYNC;
}

// The neighbours (generators of the cell's bisector faces, in face order,
// into X.nb) and the widened cell: the box D +- delta cut by their
// bisectors pushed out by delta.  *out: the widened cell (S.A or S.B);
// false: a cut gave up.
template <class Env>
P2M_HD bool cell_widen(fw::WarpWork &S, CellExtra &X, const Env &env, int64_t p,
                       const cc::CellParams &cp, const CellSlot &c, const fw::WPoly *&out) {
  P2M_LANE0 {
    int nn = 0;
    for (int f = 0; f < c.poly.nf; ++f) {
      const int32_t w = c.poly.src[f];
      if (w >= 0 && !cc::has_row(X.nb, nn, w)) X.nb[nn++] = w;
    }
    X.nb_n = nn;
    double wlo[3], whi[3];
    for (int d = 0; d < 3; ++d) {
      wlo[d] = cp.lo[d] - cp.delta;
      whi[d] = cp.hi[d] + cp.delta;
    }
    cc::make_box(S.A, wlo, whi);
  }
  P2M_SYNC;
  fw::WPoly *cur = &S.A;
  fw::View in = fw::view_of(S.A);
  const int nn = X.nb_n;
  for (int i = 0; i < nn; ++i)
    if (!bisector_cut(S, env, in, cur, p, X.nb[i], cp.delta, cp.eps)) return false;
  out = cur;
  return true;
}

}  // namespace cw
}  // namespace p2m
