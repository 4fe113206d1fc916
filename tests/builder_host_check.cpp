// Host check of the product builder, compiled by tests/test_builder_sanitized.py
// with AddressSanitizer and UBSan.  Reads one mesh file (counts, float32
// vertices, int32 triangles and segments, domain scale and margin) and
//   1. builds the layout on the host;
//   2. builds it again through a stand-in for the device services: the
//      certification searches answered by brute force under the same rule
//      (the nearest tree position strictly inside the bound, lowest
//      position on ties), the Voronoi cells made in the device's rounds by
//      its warp phases (cell_warp.h, lanes one after another) with every
//      seventh cell handed back to the host, the packing by pack_core.h's
//      steps (rows in reverse order), and the flooding run with the device kernel's warp
//      algorithm (flood_warp.h, lanes one after another, row stamps as on
//      the device), and requires
//      every table, box code, neighbour list and count to equal the host
//      build's;
//   3. injects an allocation failure into each build stage and requires
//      std::bad_alloc to reach the caller.
// Prints "OK" when every check holds.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "builder.h"
#include "cell_core.h"
#include "cell_warp.h"
#include "flood_core.h"
#include "flood_warp.h"
#include "pack_core.h"

using namespace p2m;

namespace {

struct LaneEnv : fc::Flat {
  std::vector<FloodRec> *rec;
  void emit(int32_t row, int32_t typed_id, const float box[6]) {
    FloodRec r;
    r.row = row;
    r.tid = typed_id;
    for (int d = 0; d < 6; ++d) r.box[d] = box[d];
    rec->push_back(r);
  }
};

// the KD tree as the device's cell kernel reads it (the layout's float
// points and child boxes), with the exact search done by brute force
struct CellEnv {
  const Layout *L;
  int64_t nleaf0() const { return ((int64_t)1 << L->kd_depth) - 1; }
  int64_t leaf_first(int64_t j) const { return (j * L->nv) >> L->kd_depth; }
  fc::D3 pos(int64_t p) const {
    return {(double)L->kd_points[4 * p], (double)L->kd_points[4 * p + 1],
            (double)L->kd_points[4 * p + 2]};
  }
  void child_boxes(int64_t node, double b0[6], double b1[6]) const {
    const float *o = &L->kd_nodes[12 * node];
    for (int d = 0; d < 6; ++d) {
      b0[d] = o[d];
      b1[d] = o[6 + d];
    }
  }
  int64_t within(fc::D3 x, double r2) const {
    double best = r2;
    int64_t bi = -1;
    for (int64_t p = 0; p < L->nv; ++p) {
      const double d = fc::len2(pos(p) - x);
      if (d < best) {
        best = d;
        bi = p;
      }
    }
    return bi;
  }
};

struct StandIn : NearestService {
  const Layout *L = nullptr;
  int flood_calls = 0;     // flooding calls answered
  int64_t hand_back = 0;   // > 0: every hand_back-th primitive of a call handed back too
  bool cells(const CellProblem &pb, CellResult &out) override {
    CellEnv env{L};
    cc::CellParams cp;
    for (int d = 0; d < 3; ++d) {
      cp.lo[d] = pb.lo[d];
      cp.hi[d] = pb.hi[d];
    }
    cp.eps = pb.eps;
    cp.epsc = pb.epsc;
    cp.delta = pb.delta;
    std::unique_ptr<fw::WarpWork> S(new fw::WarpWork);
    std::unique_ptr<cw::CellExtra> X(new cw::CellExtra);
    const int64_t nv = pb.nv;
    std::vector<cw::CellSlot> slots(nv);
    // the device's rounds: seeding, then per round every open cell's far
    // corners, all of them searched, every cell cut by what its corners found
    for (int64_t p = 0; p < nv; ++p) {
      if (p % 7 == 3) slots[p].status = cw::kGaveUp;
      else cw::cell_seed(*S, *X, env, p, cp, slots[p]);
    }
    for (int round = 0; round < cc::kRounds; ++round) {
      std::vector<double> xs, rs;
      for (int64_t p = 0; p < nv; ++p) {
        cw::CellSlot &c = slots[p];
        if (c.status != cw::kOpen) continue;
        const fc::D3 pv = env.pos(p);
        const int m = cw::round_corners(*X, c, pv);
        const int ms = m > 0 ? cw::round_unsettled(*X, c, m) : 0;
        c.m = 0;
        if (m > 0) {
          c.rounds += 1;
          c.queries += m;
        }
        if (ms == 0) {
          c.status = cw::kDone;
          continue;
        }
        c.m = ms;
        c.corner_at = (int64_t)rs.size();
        for (int j = 0; j < ms; ++j) {
          const fc::D3 x = X->sorted[j];
          xs.push_back(x.x);
          xs.push_back(x.y);
          xs.push_back(x.z);
          rs.push_back(fc::len2(x - pv) - pb.epsc);
        }
      }
      if (rs.empty()) {
        bool open = false;
        for (const auto &c : slots) open |= c.status == cw::kOpen;
        if (!open) break;
        continue;
      }
      std::vector<int64_t> wres(rs.size());
      for (size_t j = 0; j < rs.size(); ++j)
        wres[j] = env.within({xs[3 * j], xs[3 * j + 1], xs[3 * j + 2]}, rs[j]);
      for (int64_t p = 0; p < nv; ++p) {
        cw::CellSlot &c = slots[p];
        if (c.status == cw::kOpen && c.m > 0)
          cw::round_apply(*S, *X, env, p, cp, c, &xs[3 * c.corner_at], &wres[c.corner_at]);
      }
    }
    out = CellResult();
    out.gave_up.assign(nv, 0);
    out.nb_off.assign(1, 0);
    out.pt_off.assign(1, 0);
    out.beg_off.assign(1, 0);
    for (int64_t p = 0; p < nv; ++p) {
      const fw::WPoly *w = nullptr;
      if (slots[p].status == cw::kGaveUp || !cw::cell_widen(*S, *X, env, p, cp, slots[p], w)) {
        out.gave_up[p] = 1;
      } else {
        for (int i = 0; i < w->np; ++i) {
          out.pt.push_back(w->pt[i].x);
          out.pt.push_back(w->pt[i].y);
          out.pt.push_back(w->pt[i].z);
        }
        for (int f = 0; f <= w->nf; ++f) out.beg.push_back(w->beg[f]);
        for (int i = 0; i < X->nb_n; ++i) out.nb.push_back(X->nb[i]);
        out.rounds = std::max<int64_t>(out.rounds, slots[p].rounds);
        out.queries += slots[p].queries;
      }
      out.pt_off.push_back((int64_t)out.pt.size() / 3);
      out.beg_off.push_back((int64_t)out.beg.size());
      out.nb_off.push_back((int64_t)out.nb.size());
    }
    return true;
  }
  // the device's packing: records bucketed by row in reverse order, every
  // row sorted on pack_core.h's keys, chunks and super-chunks encoded by it
  bool pack(int64_t nv, const std::vector<PackPart> &parts, const float qlo[3],
            const float qinv[3], Layout &out, int64_t &max_list, int64_t &bad_boxes) override {
    std::vector<std::vector<FloodRec>> rows(nv);
    for (auto it = parts.rbegin(); it != parts.rend(); ++it)
      for (int64_t j = it->n - 1; j >= 0; --j)
        if (it->rec[j].row >= 0) rows[it->rec[j].row].push_back(it->rec[j]);
    pk::Frame fr;
    for (int d = 0; d < 3; ++d) {
      fr.lo[d] = qlo[d];
      fr.inv[d] = qinv[d];
    }
    q_frame_derive(fr.lo, fr.inv, fr.step, fr.base);
    out.row_off.assign(nv + 1, 0);
    out.chunk_off.assign(nv + 1, 0);
    out.super_off.assign(nv + 1, 0);
    max_list = 0;
    for (int64_t p = 0; p < nv; ++p) {
      const uint32_t len = (uint32_t)rows[p].size();
      max_list = std::max<int64_t>(max_list, len);
      out.row_off[p + 1] = out.row_off[p] + len;
      const uint32_t nc = (len + pk::kChunk - 1) / pk::kChunk;
      out.chunk_off[p + 1] = out.chunk_off[p] + nc;
      out.super_off[p + 1] = out.super_off[p] + (nc + pk::kChunk - 1) / pk::kChunk;
    }
    out.entries.assign(4 * (size_t)out.row_off[nv], 0u);
    out.chunks.assign(4 * (size_t)out.chunk_off[nv], 0u);
    out.supers.assign(4 * (size_t)out.super_off[nv], 0u);
    bad_boxes = 0;
    for (int64_t p = 0; p < nv; ++p) {
      auto &r = rows[p];
      if (r.size() >= 2) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (const FloodRec &x : r) pk::centre_bounds_add(x, lo, hi);
        std::sort(r.begin(), r.end(), [&](const FloodRec &a, const FloodRec &b) {
          return pk::row_key(a, lo, hi) < pk::row_key(b, lo, hi);
        });
      }
      uint32_t c = out.chunk_off[p];
      for (uint32_t j = 0; j < r.size(); j += pk::kChunk, ++c) {
        const uint32_t cnt = std::min<uint32_t>(pk::kChunk, (uint32_t)r.size() - j);
        bad_boxes += pk::encode_chunk(r.data() + j, cnt, fr.lo, fr.inv, fr.step, fr.base,
                                      &out.chunks[4 * (size_t)c],
                                      &out.entries[4 * (size_t)(out.row_off[p] + j)]);
      }
      uint32_t sidx = out.super_off[p];
      for (uint32_t k = out.chunk_off[p]; k < out.chunk_off[p + 1]; k += pk::kChunk, ++sidx)
        pk::encode_super(&out.chunks[4 * (size_t)k],
                         std::min<uint32_t>(pk::kChunk, out.chunk_off[p + 1] - k),
                         &out.supers[4 * (size_t)sidx]);
    }
    return true;
  }
  bool within(const double *xyz, const double *r2, int64_t n, int64_t *out) override {
    for (int64_t i = 0; i < n; ++i) {
      double best = r2[i];
      int64_t bi = -1;
      for (int64_t p = 0; p < L->nv; ++p) {
        const double dx = xyz[3 * i] - (double)L->kd_points[4 * p],
                     dy = xyz[3 * i + 1] - (double)L->kd_points[4 * p + 1],
                     dz = xyz[3 * i + 2] - (double)L->kd_points[4 * p + 2];
        const double d = dx * dx + dy * dy + dz * dz;
        if (d < best) {
          best = d;
          bi = p;
        }
      }
      out[i] = bi;
    }
    return true;
  }
  bool flood(const FloodProblem &pb, std::vector<FloodRec> &out, std::vector<uint8_t> &gave_up,
             int64_t &inspections) override {
    LaneEnv env;
    env.pt_off = pb.cell_pt_off;
    env.pt = (const fc::D3 *)pb.cell_pt;
    env.beg_off = pb.cell_beg_off;
    env.beg = pb.cell_beg;
    env.pos = (const fc::D3 *)pb.pv;
    env.vids = pb.vid;
    env.nbo = pb.nb_off;
    env.nbs = pb.nb;
    env.perp_off = pb.perp_off;
    env.perp = pb.perp;
    env.gtype = pb.gtype;
    env.g = pb.g;
    env.seed_row = pb.seed_row;
    env.seed_vid = pb.seed_vid;
    env.tid = pb.tid;
    env.rec = &out;
    gave_up.assign(pb.n, 0);
    inspections = 0;
    std::unique_ptr<fw::WarpWork> S(new fw::WarpWork);
    std::vector<int32_t> seen(pb.nv, 0);  // the device's row stamps
    for (int64_t i = pb.n - 1; i >= 0; --i) {  // any order: the host sorts
      int64_t k = 0;
      const int r = fw::flood_warp(*S, env, i, pb.eps, pb.delta, pb.eta, k, seen.data());
      // records of a given-up primitive stay in: the host drops them
      gave_up[i] = r != 0 || (hand_back > 0 && i % hand_back == hand_back - 1);
      if (!gave_up[i]) inspections += k;
    }
    ++flood_calls;
    return true;
  }
};

bool same(const Layout &A, const Layout &B) {
  return A.entries == B.entries && A.chunks == B.chunks && A.supers == B.supers &&
         A.row_off == B.row_off && A.chunk_off == B.chunk_off && A.super_off == B.super_off &&
         A.nb == B.nb && A.nb_off == B.nb_off && A.nbp == B.nbp && A.kd_points == B.kd_points &&
         A.kd_nodes == B.kd_nodes && A.edge_rec == B.edge_rec && A.face_rec == B.face_rec &&
         A.inspections == B.inspections && A.n_entries == B.n_entries &&
         A.max_list == B.max_list && A.neighbour_pairs == B.neighbour_pairs &&
         A.cert_rounds == B.cert_rounds && A.cert_queries == B.cert_queries;
}

}  // namespace

#define CHECK(c)                                         \
  do {                                                   \
    if (!(c)) {                                          \
      std::printf("FAILED %s (line %d)\n", #c, __LINE__); \
      return 1;                                          \
    }                                                    \
  } while (0)

int main(int argc, char **argv) {
  if (argc < 2) return 2;
  FILE *f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t nv, nf, ns;
  CHECK(std::fread(&nv, 8, 1, f) == 1 && std::fread(&nf, 8, 1, f) == 1 &&
        std::fread(&ns, 8, 1, f) == 1);
  std::vector<float> V(3 * nv);
  std::vector<int32_t> F(3 * nf + 1), S(2 * ns + 1);
  double sc[2];
  CHECK(std::fread(V.data(), 4, 3 * nv, f) == (size_t)(3 * nv));
  CHECK(nf == 0 || std::fread(F.data(), 4, 3 * nf, f) == (size_t)(3 * nf));
  CHECK(ns == 0 || std::fread(S.data(), 4, 2 * ns, f) == (size_t)(2 * ns));
  CHECK(std::fread(sc, 8, 2, f) == 2);
  std::fclose(f);
  BuildParams prm;
  prm.domain_scale = sc[0];
  prm.domain_margin = sc[1];
  prm.threads = 4;
  const int32_t *Fp = nf ? F.data() : nullptr, *Sp = ns ? S.data() : nullptr;
  std::string err;

  Layout host;
  CHECK(build_layout(V.data(), nv, Fp, nf, Sp, ns, prm, nullptr, nullptr, nullptr, host, err) == 0);

  StandIn svc;
  BuildParams prm2 = prm;
  prm2.device_flood = true;
  prm2.device_cells = true;
  prm2.device_pack = true;
  Layout dev;
  auto on_tree = [](void *ctx, const Layout &L) {
    ((StandIn *)ctx)->L = &L;
    return true;
  };
  CHECK(build_layout(V.data(), nv, Fp, nf, Sp, ns, prm2, &svc, on_tree, &svc, dev, err) == 0);
  CHECK(dev.flood_device > 0);
  CHECK(dev.cells_device > 0 && dev.cells_host > 0);
  CHECK(dev.pack_device == 1 && host.pack_device == 0);
  CHECK(host.cells_device == 0 && host.cells_host == nv);
  CHECK(same(host, dev));

  // the flooding in several device calls on sub-ranges of the primitives
  // (no host workers beside it: the calls' ranges are fixed), every fifth
  // primitive of a call handed back; then with the workers beside it
  for (int workers : {0, -1}) {
    StandIn s3;
    s3.hand_back = 5;
    BuildParams prm3 = prm2;
    prm3.flood_host_workers = workers;
    prm3.flood_first_share = 0.3;
    prm3.flood_min_share = 16;
    Layout d3;
    CHECK(build_layout(V.data(), nv, Fp, nf, Sp, ns, prm3, &s3, on_tree, &s3, d3, err) == 0);
    CHECK(s3.flood_calls >= 1 && d3.flood_device > 0);
    if (workers == 0) CHECK(s3.flood_calls >= 3);
    CHECK(d3.flood_device + d3.flood_bounded + d3.flood_unbounded ==
          dev.flood_device + dev.flood_bounded + dev.flood_unbounded);
    CHECK(same(host, d3));
  }

  for (const char *stage : {"cells", "flooding", "packing"}) {
    setenv("P2M_INJECT_BAD_ALLOC", stage, 1);
    Layout L;
    bool thrown = false;
    try {
      build_layout(V.data(), nv, Fp, nf, Sp, ns, prm, nullptr, nullptr, nullptr, L, err);
    } catch (const std::bad_alloc &) {
      thrown = true;
    }
    CHECK(thrown);
  }
  // a failure of a host worker beside the device flooding: the build
  // throws once the device call has come back and every worker has ended
  {
    setenv("P2M_INJECT_BAD_ALLOC", "flooding", 1);
    StandIn s4;
    Layout L;
    bool thrown = false;
    try {
      build_layout(V.data(), nv, Fp, nf, Sp, ns, prm2, &s4, on_tree, &s4, L, err);
    } catch (const std::bad_alloc &) {
      thrown = true;
    }
    CHECK(thrown && s4.flood_calls == 1);
  }
  unsetenv("P2M_INJECT_BAD_ALLOC");
  std::printf("OK\n");
  return 0;
}
