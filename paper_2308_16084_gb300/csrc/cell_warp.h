// cell_warp.h -- the Voronoi cell of one vertex clipped to the domain D
// (Alg. A.1's cells) made by the 32 lanes of a warp.
//
// The steps and their order are the host builder's (cell_core.h): the box D
// cut by the bisectors of the 32 nearest vertices (nearest first); then
// rounds in which every distinct corner farther from the vertex than half
// the 32nd distance asks the exact search for a vertex strictly nearer to it
// than the cell's own, and the cell is cut by the bisectors of the vertices
// found (not applied yet, first found first, then ordered by their distance
// to the cell's vertex, ties in that order), until no corner finds one or 65
// rounds have passed.  The generators of the surviving faces are the
// vertex's Voronoi neighbours; the widened cell is the box D +- delta cut by
// their bisectors pushed out by delta, in face order.
//
// Spread over the lanes: the cuts (fw::warp_cut: one point, then one face
// per lane), the ranking of the corners (one corner per lane against all),
// the filter of the distinct corners and their exact searches (one corner
// per lane).  Lane 0 runs the 32-nearest search, picks the candidates and
// chains the cap loops.  Every value is the host's double-precision
// operation in the host's order (no fused multiply-adds on either side), so
// the cell equals the host builder's bit for bit; a cell whose polytope
// outgrows the warp's buffers, whose cap loop cannot be chained (the host
// then orders the cap by angle) or whose exact search gives up is handed
// back.  Sections as in flood_warp.h: compiled for the host, the lanes run
// one after another.
#pragma once

#include "cell_core.h"
#include "flood_warp.h"

namespace p2m {
namespace cw {

using fc::D3;
using fc::len2;

// per-warp state besides the cut's work space (fw::WarpWork)
struct CellExtra {
  D3 corner[fw::kWP];       // the polytope's points, then a round's distinct corners
  D3 sorted[fw::kWP];       // the points in corner order
  int32_t rank[fw::kWP];    // each point's place in that order, then the kept ones'
  int32_t keep[fw::kWP];    // 1: first of its run and beyond the safe radius
  int64_t wres[fw::kWP];    // the exact search's answer for each corner
  int32_t applied[cc::kApplied];
  int32_t cand[fw::kWP];
  double cand_d[fw::kWP];
  int64_t knn_id[cc::kSeedK];
  double knn_d2[cc::kSeedK];
  int32_t nb[fw::kWF];
  int nb_n, n_applied, n_cand, m, k, flag, rounds;
  int64_t queries;
  unsigned long long out_at[3];  // the kernel's output offsets for this cell
};

// *cur cut by the bisector of rows p and w pushed out by `push` (cap
// generator w); the buffers swap when the cut changed the cell.  false: the
// cut gave up.
template <class Env>
P2M_HD bool bisector_cut(fw::WarpWork &S, const Env &env, fw::WPoly *&cur, fw::WPoly *&other,
                         int64_t p, int64_t w, double push, double eps) {
  D3 n;
  double c;
  cc::bisector(env.pos(p), env.pos(w), push, n, c);
  const int r = fw::warp_cut(S, fw::view_of(*cur), n, c, eps, *other, (int32_t)w);
  if (r == fw::kGiveUp) return false;
  if (r == fw::kDone) {
    fw::WPoly *t = cur;
    cur = other;
    other = t;
  }
  return true;
}

// The cell of row p.  Env: as cc::k_nearest, plus within(x, r2) (the
// nearest row strictly closer to x than sqrt(r2), lowest row on ties; -1
// none, -2 gave up).  On cc::kCellOk *out is the widened cell (S.A or S.B)
// and X.nb[0 .. X.nb_n) the neighbours; X.rounds, X.queries count the
// certification's rounds and searched corners.
template <class Env>
P2M_HD int cell_warp(fw::WarpWork &S, CellExtra &X, const Env &env, int64_t p,
                     const cc::CellParams &cp, const fw::WPoly *&out) {
  const D3 pv = env.pos(p);
  fw::WPoly *cur = &S.A, *other = &S.B;
  P2M_LANE0 {
    cc::make_box(*cur, cp.lo, cp.hi);
    X.k = cc::k_nearest(env, pv, p, X.knn_id, X.knn_d2);
    X.rounds = 0;
    X.queries = 0;
  }
  P2M_SYNC;
  const int k = X.k;
  if (k < 0) return cc::kCellGiveUp;
  // seeding: the bisectors of the nearest vertices, nearest first
  for (int i = 0; i < k; ++i)
    if (!bisector_cut(S, env, cur, other, p, X.knn_id[i], 0.0, cp.eps)) return cc::kCellGiveUp;
  P2M_LANE0 {
    for (int i = 0; i < k; ++i) X.applied[i] = (int32_t)X.knn_id[i];
    X.n_applied = k;
  }
  P2M_SYNC;
  // a corner within half the 32nd distance of p has no nearer vertex
  // outside the 32 nearest
  const double safe2 = k == cc::kSeedK ? 0.25 * X.knn_d2[cc::kSeedK - 1] : (double)INFINITY;
  for (int round = 0; round < cc::kRounds; ++round) {
    const int np = cur->np;
    // the points ranked in corner order (equal points by index)
    P2M_LANES(l)
      for (int i = l; i < np; i += 32) X.corner[i] = cur->pt[i];
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
    // the distinct corners farther than the safe radius, in order
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
    const int m = X.m;
    if (m == 0) break;
    // the exact search of every corner
    P2M_LANES(l)
      for (int i = l; i < m; i += 32) {
        const D3 x = X.corner[i];
        X.wres[i] = env.within(x, len2(x - pv) - cp.epsc);
      }
    P2M_END_LANES
    // the vertices found, first found first, then nearest first
    P2M_LANE0 {
      ++X.rounds;
      X.queries += m;
      int flag = 0, nc = 0;
      for (int i = 0; i < m; ++i) {
        const int64_t w = X.wres[i];
        if (w == -2) {
          flag = 1;
          break;
        }
        if (w >= 0 && w != p && !cc::has_row(X.applied, X.n_applied, (int32_t)w) &&
            !cc::has_row(X.cand, nc, (int32_t)w)) {
          X.cand[nc] = (int32_t)w;
          X.cand_d[nc] = len2(env.pos(w) - pv);
          ++nc;
        }
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
      if (X.n_applied + nc > cc::kApplied) flag = 1;
      X.n_cand = nc;
      X.flag = flag;
    }
    P2M_SYNC;
    if (X.flag) return cc::kCellGiveUp;
    const int nc = X.n_cand;
    if (nc == 0) break;
    for (int i = 0; i < nc; ++i)
      if (!bisector_cut(S, env, cur, other, p, X.cand[i], 0.0, cp.eps)) return cc::kCellGiveUp;
    P2M_LANE0 {
      for (int i = 0; i < nc; ++i) X.applied[X.n_applied + i] = X.cand[i];
      X.n_applied += nc;
    }
    P2M_SYNC;
  }
  // neighbours (the generators of the surviving bisector faces), then the
  // widened cell
  P2M_LANE0 {
    int nn = 0;
    for (int f = 0; f < cur->nf; ++f) {
      const int32_t w = cur->src[f];
      if (w >= 0 && !cc::has_row(X.nb, nn, w)) X.nb[nn++] = w;
    }
    X.nb_n = nn;
    double wlo[3], whi[3];
    for (int d = 0; d < 3; ++d) {
      wlo[d] = cp.lo[d] - cp.delta;
      whi[d] = cp.hi[d] + cp.delta;
    }
    cc::make_box(*other, wlo, whi);
  }
  P2M_SYNC;
  {
    fw::WPoly *t = cur;
    cur = other;
    other = t;
  }
  const int nn = X.nb_n;
  for (int i = 0; i < nn; ++i)
    if (!bisector_cut(S, env, cur, other, p, X.nb[i], cp.delta, cp.eps)) return cc::kCellGiveUp;
  out = cur;
  return cc::kCellOk;
}

}  // namespace cw
}  // namespace p2m
