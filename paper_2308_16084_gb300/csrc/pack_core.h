// pack_core.h -- the packing of the interception table as the host builder
// does it, one row at a time, for the host and for the device kernels
// (pack.cu).
//
// A row's records are put in spatial order (Morton code of the Region-box
// centre within the union of the row's centres, ties by typed id: a total
// order, as typed ids are distinct in a row), cut into chunks of kChunk
// entries, each chunk given the 15-bit codes of its entries' hull (two codes
// wider on each side) in the global frame and an entry frame of its own, and
// every entry its codes in its chunk's frame; every kChunk chunks share a
// super-chunk whose codes are their hull (quant.h).  Every float and double
// operation is the host builder's, compiled without fused multiply-adds on
// both sides, so the packed words are the host's bit for bit.
#pragma once

#include <cstdint>

#include "builder.h"
#include "quant.h"

namespace p2m {
namespace pk {

constexpr uint32_t kChunk = 8;  // entries per chunk, chunks per super-chunk

// the global code frame (quant.h): origin, scale and their derived step, base
struct Frame {
  float lo[3], inv[3], step[3], base[3];
};

P2M_HD float fmin_first(float a, float b) { return b < a ? b : a; }  // std::min
P2M_HD float fmax_first(float a, float b) { return a < b ? b : a; }  // std::max

P2M_HD uint32_t spread10(uint32_t v) {
  v &= 0x3ff;
  v = (v | (v << 16)) & 0x030000FF;
  v = (v | (v << 8)) & 0x0300F00F;
  v = (v | (v << 4)) & 0x030C30C3;
  v = (v | (v << 2)) & 0x09249249;
  return v;
}

// the union of a row's box centres: lo[3], hi[3] (both INFINITY-seeded as on
// the host; any order of the records gives the same bounds)
P2M_HD void centre_bounds_add(const FloodRec &r, float lo[3], float hi[3]) {
  for (int d = 0; d < 3; ++d) {
    const float c = 0.5f * (r.box[d] + r.box[3 + d]);
    lo[d] = fmin_first(lo[d], c);
    hi[d] = fmax_first(hi[d], c);
  }
}

// the sort key of a record: Morton code of its centre in the row's bounds,
// then its typed id
P2M_HD uint64_t row_key(const FloodRec &r, const float lo[3], const float hi[3]) {
  uint32_t k[3];
  for (int d = 0; d < 3; ++d) {
    const float ext = hi[d] - lo[d];
    const float u = ext > 0 ? (0.5f * (r.box[d] + r.box[3 + d]) - lo[d]) / ext : 0.f;
    k[d] = (uint32_t)fmin_first(1023.f, fmax_first(0.f, u * 1024.f));
  }
  const uint32_t m = spread10(k[0]) | (spread10(k[1]) << 1) | (spread10(k[2]) << 2);
  return (uint64_t)m << 32 | (uint32_t)r.tid;
}

// One chunk: the cnt records r[0 .. cnt) (in row order) into the chunk's
// four words cw and the entries' four words each (ew, 4 per entry), in the
// global code frame (qlo, qinv, qstep, qbase).  Returns the number of entry
// codes outside their chunk's frame (0 unless something is wrong).
P2M_HD int encode_chunk(const FloodRec *r, uint32_t cnt, const float qlo[3], const float qinv[3],
                        const float qstep[3], const float qbase[3], uint32_t *cw, uint32_t *ew) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t k = 0; k < cnt; ++k)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin_first(lo[d], r[k].box[d]);
      hi[d] = fmax_first(hi[d], r[k].box[3 + d]);
    }
  // chunk codes: the entries' hull, two codes wider on each side, so that an
  // entry test that passes implies a chunk test that passes
  uint32_t cl[3], ch[3];
  for (int d = 0; d < 3; ++d) {
    const uint32_t a = q_code(lo[d], qlo[d], qinv[d]);
    const uint32_t b = q_code(hi[d], qlo[d], qinv[d]);
    cl[d] = a >= 2 ? a - 2 : 0;
    ch[d] = b + 2 < kQMax ? b + 2 : kQMax;
  }
  q_words(cl, ch, cw);
  // entry frame: origin from the chunk codes, scale inv * 2^e with the
  // largest e that keeps the entries clear of the frame's top code
  float clo[3], cinv[3];
  uint32_t w3 = 0;
  for (int d = 0; d < 3; ++d) {
    clo[d] = q_chunk_lo(cl[d], qstep[d], qbase[d]);
    const double diff = (double)hi[d] - (double)clo[d];
    const double ext = diff < 0.0 ? 0.0 : diff;
    uint32_t e = 0;
    while (e < 60 && ext * (double)qinv[d] * ldexp(1.0, (int)e + 1) <= (double)(kQMax - 64)) ++e;
    w3 |= e << (8 * d);
  }
  cw[3] = w3;
  for (int d = 0; d < 3; ++d) cinv[d] = q_chunk_inv(qinv[d], w3, d);
  int bad = 0;
  for (uint32_t k = 0; k < cnt; ++k) {
    uint32_t *w = ew + 4 * k;
    w[0] = (uint32_t)r[k].tid;
    uint32_t el[3], eh[3];
    for (int d = 0; d < 3; ++d) {
      el[d] = q_code(r[k].box[d], clo[d], cinv[d]);
      eh[d] = q_code(r[k].box[3 + d], clo[d], cinv[d]);
      // inside the frame, never clamped: queries far outside fail
      if (el[d] < 1 || eh[d] >= kQMax) ++bad;
    }
    q_words(el, eh, w + 1);
  }
  return bad;
}

// one super-chunk: the hull of the codes of the chunks cw[0 .. n) (4 words
// each) into sw
P2M_HD void encode_super(const uint32_t *cw, uint32_t n, uint32_t *sw) {
  uint32_t sl[3] = {kQMax, kQMax, kQMax}, sh[3] = {0, 0, 0};
  for (uint32_t k = 0; k < n; ++k) {
    uint32_t cl[3], ch[3];
    q_unwords(cw + 4 * k, cl, ch);
    for (int d = 0; d < 3; ++d) {
      sl[d] = cl[d] < sl[d] ? cl[d] : sl[d];
      sh[d] = sh[d] < ch[d] ? ch[d] : sh[d];
    }
  }
  q_words(sl, sh, sw);
  sw[3] = 0;  // unused (the layout zero-fills it)
}

}  // namespace pk
}  // namespace p2m
