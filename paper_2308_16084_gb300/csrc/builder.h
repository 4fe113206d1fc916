// builder.h -- host preprocessing of the P2M query layout (Alg. A.1).
//
// Produces everything the query kernels read: a bucketed KD tree over the
// vertices (perfect binary tree, child boxes in the parent), the CSR
// interception table in KD-tree row order with one Region box per entry,
// and per-primitive geometry records.  Runs on the host with std::thread;
// the Voronoi-cell certification can hand its nearest-vertex queries, and
// the flooding its primitives, to device kernels through the NearestService
// interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace p2m {

struct BuildParams {
  double domain_scale = 10.0;
  double domain_margin = 0.0;
  double delta_rel = 4e-6;
  int threads = 0;
  int leaf_size = 8;
  bool device_flood = false;  // flood on the nearest service when it offers that
  bool device_cells = false;  // Voronoi cells on the nearest service when it offers that
  bool device_pack = false;   // the table's packing on the nearest service when it offers that
  // the device flooding beside the host's: host workers beside the device
  // (< 0: the build's threads but one), the share of all primitives the
  // first device call takes (< 0: sized from the workers) and the fewest
  // primitives a later call takes
  int flood_host_workers = -1;
  double flood_first_share = -1.0;
  int64_t flood_min_share = 1 << 14;
};

// The Voronoi cells of every row (KD-tree position), clipped to D, for a
// device service: what the builder's cell stage takes (cell_core.h).
struct CellProblem {
  int64_t nv = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // the domain D
  double eps = 0, epsc = 0, delta = 0;
};

// What a device service returns: per row, gave_up[p] = 1 where the host
// must compute the cell itself, else its Voronoi neighbours
// nb[nb_off[p] .. nb_off[p+1]) (rows, in the order of its faces) and its
// widened cell (points pt[3 pt_off[p] ..), loops as in FloodProblem).
struct CellResult {
  std::vector<uint8_t> gave_up;
  std::vector<int64_t> nb_off;
  std::vector<int32_t> nb;
  std::vector<int64_t> pt_off;
  std::vector<double> pt;
  std::vector<int64_t> beg_off;
  std::vector<int32_t> beg;
  // over the rows it kept: the most certification rounds one of them took
  // and the corners they searched (the host's own counts over those rows)
  int64_t rounds = 0, queries = 0;
};

// The flooding inspection (Alg. 1) of a set of primitives, for a device
// service.  Host arrays; rows are KD-tree positions.
struct FloodProblem {
  int64_t nv = 0;  // rows
  int64_t n = 0;   // primitives
  // widened cells: the points of row p's cell are
  // cell_pt[cell_pt_off[p] .. cell_pt_off[p+1]) (3 doubles each); its nf
  // face loops start at the offsets cell_beg[cell_beg_off[p] ..
  // cell_beg_off[p+1]) relative to its first point (nf + 1 of them, the
  // last one the point count)
  const int64_t *cell_pt_off = nullptr;
  const double *cell_pt = nullptr;
  const int64_t *cell_beg_off = nullptr;
  const int32_t *cell_beg = nullptr;
  const double *pv = nullptr;      // nv * 3 vertex positions
  const int32_t *vid = nullptr;    // nv vertex ids
  const uint32_t *nb_off = nullptr;  // nv + 1, Voronoi neighbours (rows)
  const uint32_t *nb = nullptr;
  // primitive i: Space-perp half-spaces perp[perp_off[i] .. perp_off[i+1])
  // (n.x <= c as 4 doubles n, c; at most 16), the filter's geometry g[6i..]
  // (a, unit u; gtype 1 = line, 2 = plane), its seeds (2 for an edge, 3 for
  // a face: rows and vertex ids) and its typed id
  const int64_t *perp_off = nullptr;
  const double *perp = nullptr;
  const int32_t *gtype = nullptr;
  const double *g = nullptr;
  const int32_t *seed_row = nullptr;  // n * 3
  const int32_t *seed_vid = nullptr;  // n * 3
  const int32_t *tid = nullptr;
  double eps = 0, delta = 0, eta = 0;
};

// one interception-table entry: table row, typed id, Region box lo, hi
struct FloodRec {
  int32_t row, tid;
  float box[6];
};

struct Layout;

// a run of records for the packing service
struct PackPart {
  const FloodRec *rec;
  int64_t n;
};

// Device services of the builder: the exact search that certifies the
// Voronoi cells' corners, the whole cell stage and the flooding.  Each
// returns false where it is unavailable (the host then does the work).
struct NearestService {
  virtual ~NearestService() = default;
  // exact (double precision) certification search: for each x (3 doubles)
  // the nearest KD-tree position strictly closer than sqrt(r2), -1 if none,
  // -2 where the service gave up (the host searches); false = unavailable
  virtual bool within(const double *xyz, const double *r2, int64_t n, int64_t *out_pos) {
    (void)xyz, (void)r2, (void)n, (void)out_pos;
    return false;
  }
  // the flooding of every primitive of pb: the records of the primitives
  // it finished (in any order), gave_up[i] = 1 for those it did not (their
  // records are left out: the host floods them), and the vertices inspected
  // for the finished ones; false = unavailable (the host floods everything)
  virtual bool flood(const FloodProblem &pb, std::vector<FloodRec> &out,
                     std::vector<uint8_t> &gave_up, int64_t &inspections) {
    (void)pb, (void)out, (void)gave_up, (void)inspections;
    return false;
  }
  // the Voronoi cell of every row as the host builder computes it (the same
  // values bit for bit), with the rows it hands back marked
  virtual bool cells(const CellProblem &pb, CellResult &out) {
    (void)pb, (void)out;
    return false;
  }
  // the packing of the table from the records of parts[] (row >= 0, any
  // order) in the code frame qlo / qinv, as the host builder packs it (the
  // same words bit for bit): out's row_off, entries, chunk_off, chunks,
  // super_off, supers, the longest row and the count of entry codes outside
  // their chunk's frame
  virtual bool pack(int64_t nv, const std::vector<PackPart> &parts, const float qlo[3],
                    const float qinv[3], Layout &out, int64_t &max_list, int64_t &bad_boxes) {
    (void)nv, (void)parts, (void)qlo, (void)qinv, (void)out, (void)max_list, (void)bad_boxes;
    return false;
  }
};

// Device-ready arrays (all little-endian, float32 unless stated).
struct Layout {
  int64_t nv = 0, nf = 0, ne = 0;
  // domain D and the widening margin
  float dom[6] = {0, 0, 0, 0, 0, 0};
  float delta = 0.f;
  // KD tree: depth d, L = 2^d leaves; leaf j holds tree positions
  // [j*nv/L, (j+1)*nv/L).  Internal node i (heap order, 0..L-2) stores the
  // boxes of its two children in 12 floats:
  //   {c0.lo.x, c0.lo.y, c0.lo.z, c0.hi.x}, {c0.hi.y, c0.hi.z, c1.lo.x, c1.lo.y},
  //   {c1.lo.z, c1.hi.x, c1.hi.y, c1.hi.z}
  int kd_depth = 0;
  std::vector<float> kd_nodes;    // (L-1) * 12
  std::vector<float> kd_points;   // nv * 4: x, y, z, original vertex id (int bits)
  float kd_root[6] = {0, 0, 0, 0, 0, 0};
  std::vector<int32_t> pos_of_vertex;   // original id -> tree position (= table row)
  // Voronoi neighbours of every vertex, as tree positions (CSR by row): the
  // generators of the bisector faces of its exact cell clipped to D
  std::vector<uint32_t> nb_off;    // nv + 1
  std::vector<uint32_t> nb;
  std::vector<float> nbp;          // per neighbour: x, y, z, row bits (parallel to nb)
  // interception table, rows in tree order
  std::vector<uint32_t> row_off;   // nv + 1
  // Entries of each row are in spatial (Morton) order of their Region-box
  // centres and grouped into chunks of up to kChunk consecutive entries (a
  // one-level R-tree per list, Sec. 4.6).  Boxes are 15-bit integer codes
  // (quant.h):
  //   chunk c: {3 words of codes in the frame qframe (D widened by 4 delta),
  //             entry-frame exponents e.x | e.y << 8 | e.z << 16}
  //   entry j: {typed id, 3 words of codes in its chunk's entry frame};
  //            typed id = type << 30 | id (type 1 = edge, 2 = face)
  // Entry j of row r belongs to chunk chunk_off[r] + (j - row_off[r]) / kChunk.
  static constexpr int kChunk = 8;
  std::vector<uint32_t> entries;   // n_entries * 4
  std::vector<uint32_t> chunk_off; // nv + 1
  std::vector<uint32_t> chunks;    // n_chunks * 4
  // second level: super-chunk s of row r covers chunks
  // chunk_off[r] + kChunk*(s - super_off[r]) ... (up to kChunk of them); its
  // codes (same frame as the chunks) are the hull of their codes
  std::vector<uint32_t> super_off; // nv + 1
  std::vector<uint32_t> supers;    // n_supers * 4
  float qframe_lo[3] = {0, 0, 0}, qframe_inv[3] = {0, 0, 0};
  // geometry records
  //   edge e: {a.x, a.y, a.z, 1/|b-a|^2}, {b.x-a.x, b.y-a.y, b.z-a.z, 0}
  //   face f: {a, A}, {b-a, B}, {c-a, C} with the projection weights
  //           s = A (e1.w) - B (e2.w), t = C (e2.w) - B (e1.w), w = q - a
  std::vector<float> edge_rec;     // ne * 8
  std::vector<float> face_rec;     // nf * 12
  std::vector<int32_t> edges;      // ne * 2 canonical (min, max)
  std::vector<int32_t> tris;       // nf * 4 (a, b, c, 0) for the backward scatter
  // statistics
  int64_t n_entries = 0, max_list = 0, neighbour_pairs = 0, inspections = 0;
  int64_t cert_rounds = 0, cert_queries = 0, n_degenerate = 0;
  // primitives flooded on the device, by the host's bounded core and by its
  // unbounded code (the ones the core gave up)
  int64_t flood_device = 0, flood_bounded = 0, flood_unbounded = 0;
  // Voronoi cells made on the device and on the host; 1 if the table was
  // packed on the device
  int64_t cells_device = 0, cells_host = 0, pack_device = 0;
  double ms_total = 0, ms_cells = 0, ms_inspect = 0;
};

// Status codes mirror p2m_status.
// S: ns segments (vertex pairs) that are edges of no face, may be NULL.
int build_layout(const float *V, int64_t nv, const int32_t *F, int64_t nf, const int32_t *S,
                 int64_t ns, const BuildParams &prm, NearestService *nearest,
                 // called once the KD tree exists, before the cells need it
                 bool (*on_tree)(void *ctx, const Layout &), void *ctx, Layout &out,
                 std::string &err);

}  // namespace p2m
