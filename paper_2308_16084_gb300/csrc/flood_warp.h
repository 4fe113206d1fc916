// flood_warp.h -- the flooding inspection of one primitive (Alg. 1) by the
// 32 lanes of a warp.
//
// The same steps as fc::flood_prim (flood_core.h), with the per-point work
// spread over the lanes: the signed distances of a cut, the emptiness
// check, the filter values and the Region-box candidates are computed one
// point per lane; the per-face bookkeeping of a cut one face per lane, its
// output placed by a prefix sum over the faces so that every loop comes out
// in the serial order; the cap chaining, the record and the queue appends
// by lane 0.  Every value is computed by the same operations as in the
// serial core, and a box is a minimum / maximum (exact, independent of the
// order), so the records are the serial core's bit for bit.
//
// Work lives in a per-warp block (WarpWork, shared memory on the device)
// with its own capacities; a primitive that would overflow one is given up
// (return 1) and flooded by the host.
//
// The code is written in sections: P2M_LANES(l) { ... } P2M_END_LANES runs
// its body once per lane l, and the code between sections is uniform (every
// lane computes the same values from shared state; only lane 0 writes
// shared state, in P2M_LANE0 blocks).  No lane reads, inside a section, what
// another lane writes in that section.  On the device a section is bracketed
// by __syncwarp(); compiled for the host it is a loop over the 32 lanes,
// which runs the same arithmetic serially.
#pragma once

#include <cstring>

#include "flood_core.h"

#if defined(__CUDA_ARCH__)
#define P2M_LANES(l) \
  __syncwarp();      \
  {                  \
    const int l = (int)(threadIdx.x & 31u);
#define P2M_END_LANES \
  }                   \
  __syncwarp();
#define P2M_LANE0 if ((threadIdx.x & 31u) == 0u)
#define P2M_SYNC __syncwarp()
#else
#define P2M_LANES(l) for (int l = 0; l < 32; ++l) {
#define P2M_END_LANES }
#define P2M_LANE0
#define P2M_SYNC ((void)0)
#endif

namespace p2m {
namespace fw {

using fc::D3;
using fc::dmax;
using fc::dmin;
using fc::edge_crossing;
using fc::dot;
using fc::len2;

constexpr int kWP = 256;    // loop points of a work polytope
constexpr int kWIn = 512;   // loop points of a polytope being read (a cell may be larger)
constexpr int kWF = 64;     // faces of a work polytope
constexpr int kWQ = 1024;   // vertices one primitive may visit

struct WPoly {
  int nf, np;
  int32_t beg[kWF + 1];
  int32_t src[kWF];  // generator of each face's plane (fc::WPoly)
  D3 pt[kWP];
};

// polytope being read: a cell in global memory or a WPoly of this warp
// (src: the faces' generators, or null)
struct View {
  const D3 *pt;
  const int32_t *beg;
  int nf, np;
  const int32_t *src;
};

struct WarpWork {
  WPoly A, B;
  double s[kWIn];         // signed distances of a cut; filter values after the cuts
  int16_t nxt[kWIn];      // successor of every loop point in its loop
  int32_t queue[kWQ];
  D3 seg_in[kWF], seg_out[kWF];  // per face: its cap segment (Y -> X)
  int32_t fcnt[kWF], foff[kWF], frank[kWF];
  uint8_t fseg[kWF];      // 1: face has a cap segment (2 once chained)
  uint8_t fone[kWF];      // 1: face's loop leaves and enters the kept side at most once
  int32_t red_i[32];
  double red_d[32][6];    // per-lane box candidates (lo xyz, hi xyz)
  double box[6];          // their minimum / maximum
  fc::Prim P;
  int64_t head, tail;
  int64_t item;           // the primitive this warp floods (device work queue)
  int flag;               // uniform result of a lane-0 step
  int cnt_np, cnt_nf;
};

P2M_HD View view_of(const WPoly &w) { return {w.pt, w.beg, w.nf, w.np, w.src}; }

enum { kNone = 0, kDone = 1, kGiveUp = 2 };

// cut `in` by n.x <= c into `out` (fc::cut, lane-parallel; a kept face
// keeps its generator, the cap gets hsrc)
P2M_HD int warp_cut(WarpWork &S, View in, D3 hn, double hc, double eps, WPoly &out,
                    int32_t hsrc = -1) {
  if (in.np > kWIn || in.nf > kWF) return kGiveUp;
  // every point's signed distance and its class, kept in S.nxt while the
  // cut runs (bit 0: s <= eps, on the kept side; bit 1: s >= -eps, not
  // strictly inside), so that the passes below compare no double again
  P2M_LANES(l)
    bool b = false, w = false;
    for (int i = l; i < in.np; i += 32) {
      const double s = dot(hn, in.pt[i]) - hc;
      S.s[i] = s;
      const bool beyond = s > eps, inside = s < -eps;
      b |= beyond;
      w |= inside;
      S.nxt[i] = (int16_t)((beyond ? 0 : 1) | (inside ? 0 : 2));
    }
    S.red_i[l] = (b ? 1 : 0) | (w ? 2 : 0);
  P2M_END_LANES
  int any = 0;
  for (int l = 0; l < 32; ++l) any |= S.red_i[l];
  if (!(any & 1)) return kNone;
  if (!(any & 2)) {
    P2M_LANE0 {
      out.nf = 0;
      out.np = 0;
      out.beg[0] = 0;
    }
    P2M_SYNC;
    return kDone;
  }
  // pass 1: every face's output count and cap segment
  P2M_LANES(l)
    for (int f = l; f < in.nf; f += 32) {
      const int b = in.beg[f], k = in.beg[f + 1] - b;
      int cnt = 0, turns = 0;
      bool has_x = false, has_y = false;
      D3 X{0, 0, 0}, Y{0, 0, 0};
      for (int i = 0; i < k; ++i) {
        const int ia = b + i, ib = b + (i + 1) % k;
        const double sa = S.s[ia], sb = S.s[ib];
        const int ca = S.nxt[ia], cb = S.nxt[ib];
        const bool ka = (ca & 1) != 0, kb = (cb & 1) != 0;
        if (ka) ++cnt;
        turns += ka != kb;
        if (ka && !kb) {
          if (ca & 2) {
            X = in.pt[ia];
          } else {
            X = fc::crossing(in.pt[ia], in.pt[ib], sa, sb);
            ++cnt;
          }
          has_x = true;
        } else if (!ka && kb) {
          if (cb & 2) {
            Y = in.pt[ib];
          } else {
            Y = fc::crossing(in.pt[ia], in.pt[ib], sa, sb);
            ++cnt;
          }
          has_y = true;
        }
      }
      S.fcnt[f] = cnt >= 3 ? cnt : 0;
      const bool hs = has_x && has_y && len2(X - Y) > eps * eps;
      S.fseg[f] = hs ? 1 : 0;
      // the exit and entry points, kept for pass 2 when the loop crosses
      // once each way (then pass 2's crossings are these)
      S.fone[f] = turns <= 2 ? 1 : 0;
      S.seg_in[f] = Y;
      S.seg_out[f] = X;
    }
  P2M_END_LANES
  // placement of the kept faces, in face order
  P2M_LANE0 {
    int np = 0, nf = 0, m = 0;
    for (int f = 0; f < in.nf; ++f) {
      S.foff[f] = np;
      S.frank[f] = nf;
      if (S.fcnt[f] > 0) {
        np += S.fcnt[f];
        ++nf;
      }
      m += S.fseg[f];
    }
    S.cnt_np = np;
    S.cnt_nf = nf;
    S.flag = (np + (m >= 3 ? m : 0) > kWP || nf + 1 > kWF) ? 1 : 0;
    S.red_i[0] = m;
  }
  P2M_SYNC;
  if (S.flag) return kGiveUp;
  const int m = S.red_i[0];
  // pass 2: every kept face writes its loop where the placement put it
  P2M_LANES(l)
    for (int f = l; f < in.nf; f += 32) {
      if (S.fcnt[f] == 0) continue;
      const int b = in.beg[f], k = in.beg[f + 1] - b;
      int o = S.foff[f];
      const bool one = S.fone[f] != 0;
      for (int i = 0; i < k; ++i) {
        const int ia = b + i, ib = b + (i + 1) % k;
        const double sa = S.s[ia], sb = S.s[ib];
        const int ca = S.nxt[ia], cb = S.nxt[ib];
        const bool ka = (ca & 1) != 0, kb = (cb & 1) != 0;
        if (ka) out.pt[o++] = in.pt[ia];
        if (ka && !kb) {
          if (!(ca & 2))
            out.pt[o++] = one ? S.seg_out[f] : fc::crossing(in.pt[ia], in.pt[ib], sa, sb);
        } else if (!ka && kb) {
          if (!(cb & 2))
            out.pt[o++] = one ? S.seg_in[f] : fc::crossing(in.pt[ia], in.pt[ib], sa, sb);
        }
      }
      out.beg[S.frank[f]] = S.foff[f];
      out.src[S.frank[f]] = in.src ? in.src[f] : -1;
    }
  P2M_END_LANES
  // the cap loop, chained from segment to segment (segments in face order,
  // as the serial core keeps them): each step takes the first unused
  // segment whose entry point is nearest to the current point.  The lanes
  // compute the distances, one segment each; the first minimum is found on
  // integer keys (a non-negative double's bits order like its value), so
  // the choice is the serial loop's.
  int nf = S.cnt_nf, np = S.cnt_np;
  P2M_LANE0 { out.beg[nf] = np; }
  int ok = 1;
  if (m >= 3) {
    int first = 0;
    while (!S.fseg[first]) ++first;
    P2M_LANE0 {
      out.pt[np] = S.seg_in[first];
      S.fseg[first] = 2;
    }
    ++np;
    D3 cur = S.seg_out[first];
    for (int step = 1; step < m && ok; ++step) {
      P2M_LANE0 { out.pt[np] = cur; }
      ++np;
      P2M_LANES(l)
        uint64_t bk = ~0ull;
        int bf = -1;
        for (int f = l; f < in.nf; f += 32)
          if (S.fseg[f] == 1) {
            const double d = len2(S.seg_in[f] - cur);
            uint64_t key;
            memcpy(&key, &d, 8);
            if (key < bk) {
              bk = key;
              bf = f;
            }
          }
        memcpy(&S.red_d[l][0], &bk, 8);
        S.red_i[l] = bf;
      P2M_END_LANES
      uint64_t bk = ~0ull;
      int best = -1;
      for (int t = 0; t < 32; ++t) {
        uint64_t key;
        memcpy(&key, &S.red_d[t][0], 8);
        const int f = S.red_i[t];
        if (f >= 0 && (key < bk || (key == bk && f < best))) {
          bk = key;
          best = f;
        }
      }
      double bd;
      memcpy(&bd, &bk, 8);
      if (best < 0 || bd > 1e6 * eps * eps) {
        ok = 0;
      } else {
        P2M_LANE0 { S.fseg[best] = 2; }
        cur = S.seg_out[best];
      }
      P2M_SYNC;
    }
    if (ok && !(len2(cur - S.seg_in[first]) <= 1e6 * eps * eps)) ok = 0;
    if (ok) {
      P2M_LANE0 {
        out.src[nf] = hsrc;
        out.beg[nf + 1] = np;
      }
      ++nf;
    }
  }
  if (nf < 4) {
    nf = 0;
    np = 0;
  }
  P2M_LANE0 {
    out.nf = nf;
    out.np = np;
  }
  P2M_SYNC;
  return ok ? kDone : kGiveUp;
}

// minimum / maximum of the lanes' box candidates, one column per lane
// (exact, so independent of the order but for the sign of a zero, which the
// widening by delta and the rounding to float32 do not see)
P2M_HD void reduce_box(WarpWork &S) {
  P2M_LANES(l)
    if (l < 6) {
      double v = S.red_d[0][l];
      for (int t = 1; t < 32; ++t) v = l < 3 ? dmin(v, S.red_d[t][l]) : dmax(v, S.red_d[t][l]);
      S.box[l] = v;
    }
  P2M_END_LANES
}

// Flood primitive k of the flat problem with the warp.  Env: fc::Flat's
// accessors and emit(row, tid, box).  seen: null, or the warp's array of one
// stamp per row (zero at first), which then marks the rows queued for k
// (stamp k + 1) instead of a scan of the queue.  Returns 0 when done (insp =
// vertices inspected), 1 when given up (records already emitted for it must
// be dropped).
template <class Env>
P2M_HD int flood_warp(WarpWork &S, Env &env, int64_t k, double eps, double delta, double eta,
                      int64_t &insp, int32_t *seen = nullptr) {
  const int32_t stamp = (int32_t)(k + 1);
  insp = 0;
  P2M_LANE0 { S.flag = env.load(k, S.P) ? 0 : 1; }
  P2M_SYNC;
  if (S.flag) return 1;
  const fc::Prim &P = S.P;
  P2M_LANE0 {
    for (int s = 0; s < P.ns; ++s) {
      S.queue[s] = P.seed_row[s];
      if (seen) seen[P.seed_row[s]] = stamp;
    }
    S.head = 0;
    S.tail = P.ns;
  }
  P2M_SYNC;
  while (S.head < S.tail) {
    const int32_t p = S.queue[S.head];
    P2M_SYNC;
    P2M_LANE0 { ++S.head; }
    P2M_SYNC;
    ++insp;
    const fc::PView cv = env.cell(p);
    const View cell{cv.pt, cv.beg, cv.nf, cv.np, nullptr};
    // a half-space with every point of the cell beyond it empties the result
    bool emptied = false;
    for (int j = 0; j < P.np && !emptied; ++j) {
      P2M_LANES(l)
        bool all_b = true;
        for (int q = l; q < cell.np; q += 32)
          if (!(dot(P.perp[j].n, cell.pt[q]) - P.perp[j].c > eps)) {
            all_b = false;
            break;
          }
        S.red_i[l] = all_b ? 1 : 0;
      P2M_END_LANES
      bool all_beyond = true;
      for (int l = 0; l < 32; ++l) all_beyond = all_beyond && S.red_i[l] != 0;
      emptied = all_beyond && cell.np > 0;
    }
    if (emptied) continue;
    View cur = cell;
    WPoly *bufs[2] = {&S.A, &S.B};
    int wsel = 0;
    for (int j = 0; j < P.np && cur.nf > 0; ++j) {
      const int r = warp_cut(S, cur, P.perp[j].n, P.perp[j].c, eps, *bufs[wsel]);
      if (r == kGiveUp) return 1;
      if (r == kDone) {
        cur = view_of(*bufs[wsel]);
        wsel ^= 1;
      }
    }
    if (cur.nf == 0) continue;
    if (cur.np > kWIn || cur.nf > kWF) return 1;
    const D3 pv = env.pv(p);
    const int32_t vid = env.vid(p);
    bool keep = (P.gtype == 1)
                    ? (P.seed_vid[0] == vid || P.seed_vid[1] == vid)
                    : (P.seed_vid[0] == vid || P.seed_vid[1] == vid || P.seed_vid[2] == vid);
    // filter values and loop successors
    P2M_LANES(l)
      for (int q = l; q < cur.np; q += 32) {
        const D3 x = cur.pt[q];
        const D3 w = x - P.ga;
        const double s = dot(w, P.gu);
        const double dist2 = P.gtype == 1 ? len2(w) - s * s : s * s;
        S.s[q] = len2(x - pv) - dist2 + eta;
      }
      for (int f = l; f < cur.nf; f += 32) {
        const int b0 = cur.beg[f], kk = cur.beg[f + 1] - b0;
        for (int q = 0; q < kk; ++q) S.nxt[b0 + q] = (int16_t)(b0 + (q + 1) % kk);
      }
    P2M_END_LANES
    // Region-box candidates: positive corners and the roots on loop edges
    // whose ends differ in sign
    P2M_LANES(l)
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      int kh = 0;
      for (int i = l; i < cur.np; i += 32) {
        const int i1 = S.nxt[i];
        const D3 x0 = cur.pt[i], x1 = cur.pt[i1];
        const double g0 = S.s[i], g1 = S.s[i1];
        if (g0 > 0) {
          kh = 3;
          lo[0] = dmin(lo[0], x0.x); hi[0] = dmax(hi[0], x0.x);
          lo[1] = dmin(lo[1], x0.y); hi[1] = dmax(hi[1], x0.y);
          lo[2] = dmin(lo[2], x0.z); hi[2] = dmax(hi[2], x0.z);
        }
        if ((g0 > 0) != (g1 > 0)) {
          const D3 d = x1 - x0, w0 = x0 - P.ga, r0 = x0 - pv;
          const double du = dot(d, P.gu), wu = dot(w0, P.gu);
          double A, B, Cc;
          if (P.gtype == 1) {
            A = len2(d) - (len2(d) - du * du);
            B = 2 * dot(r0, d) - 2 * (dot(w0, d) - wu * du);
            Cc = len2(r0) - (len2(w0) - wu * wu) + eta;
          } else {
            A = len2(d) - du * du;
            B = 2 * dot(r0, d) - 2 * wu * du;
            Cc = len2(r0) - wu * wu + eta;
          }
          double tb[2];
          edge_crossing(A, B, Cc, g0 > 0, &tb[0], &tb[1]);
          for (int r = 0; r < 2; ++r) {
            const D3 x = x0 + tb[r] * d;
            lo[0] = dmin(lo[0], x.x); hi[0] = dmax(hi[0], x.x);
            lo[1] = dmin(lo[1], x.y); hi[1] = dmax(hi[1], x.y);
            lo[2] = dmin(lo[2], x.z); hi[2] = dmax(hi[2], x.z);
            kh |= 2;
          }
        }
      }
      S.red_i[l] = kh;
      for (int d = 0; d < 3; ++d) {
        S.red_d[l][d] = lo[d];
        S.red_d[l][3 + d] = hi[d];
      }
    P2M_END_LANES
    bool have = false;
    for (int l = 0; l < 32; ++l) {
      keep = keep || (S.red_i[l] & 1);
      have = have || (S.red_i[l] & 2);
    }
    if (!keep) continue;
    if (have) reduce_box(S);
    else {
      P2M_LANES(l)
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int q = l; q < cur.np; q += 32) {
          const D3 x = cur.pt[q];
          lo[0] = dmin(lo[0], x.x); hi[0] = dmax(hi[0], x.x);
          lo[1] = dmin(lo[1], x.y); hi[1] = dmax(hi[1], x.y);
          lo[2] = dmin(lo[2], x.z); hi[2] = dmax(hi[2], x.z);
        }
        for (int d = 0; d < 3; ++d) {
          S.red_d[l][d] = lo[d];
          S.red_d[l][3 + d] = hi[d];
        }
      P2M_END_LANES
      reduce_box(S);
    }
    P2M_LANE0 {
      float box[6];
      for (int d = 0; d < 3; ++d) {
        const double blo = S.box[d], bhi = S.box[3 + d];
        float lw = (float)(blo - delta), h = (float)(bhi + delta);
        if ((double)lw > blo - delta) lw = nextafterf(lw, -INFINITY);
        if ((double)h < bhi + delta) h = nextafterf(h, INFINITY);
        box[d] = lw;
        box[3 + d] = h;
      }
      env.emit(p, P.tid, box);
    }
    // unseen Voronoi neighbours join the queue in neighbour order (the
    // neighbours of a vertex are distinct, so checking a batch against the
    // queue as it stood before the batch is the serial check)
    const int64_t nb0 = env.nb_begin(p), nb1 = env.nb_end(p);
    for (int64_t base = nb0; base < nb1; base += 32) {
      const int64_t tail0 = S.tail;
      P2M_LANES(l)
        int isnew = 0;
        if (base + l < nb1) {
          const int32_t w = env.nb(base + l);
          isnew = 1;
          if (seen) {
            isnew = seen[w] != stamp;
          } else {
            for (int64_t q = 0; q < tail0; ++q)
              if (S.queue[q] == w) {
                isnew = 0;
                break;
              }
          }
        }
        S.red_i[l] = isnew;
      P2M_END_LANES
      P2M_LANE0 {
        S.flag = 0;
        for (int l = 0; l < 32 && !S.flag; ++l)
          if (S.red_i[l]) {
            if (S.tail >= kWQ) {
              S.flag = 1;
            } else {
              const int32_t w = env.nb(base + l);
              S.queue[S.tail++] = w;
              if (seen) seen[w] = stamp;
            }
          }
      }
      P2M_SYNC;
      if (S.flag) return 1;
    }
  }
  return 0;
}

}  // namespace fw
}  // namespace p2m
