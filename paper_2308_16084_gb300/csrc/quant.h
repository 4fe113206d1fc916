// quant.h -- 15-bit integer codes of the Region boxes in the interception
// lists (the boxes of Sec. 4.6's filter, stored compactly).
//
// A frame is a float origin `lo` and scale `inv` per axis.  The code of a
// coordinate x in a frame is
//     c(x) = floor(clamp((x - lo) * inv, -1, K - 1)) + 1      in 0..K,
// K = 32767, evaluated with the same rounded float operations on the host
// and on the device, so the host builder knows the exact code every query
// will get.  c is monotone in x, so a box [a, b] stored as the codes
// [c(a), c(b)] admits every x in [a, b]: the filter stays conservative by
// construction, with no error analysis.
//
// Six codes pack into three words of two 15-bit lanes (bits 15 and 31
// clear).  Upper bounds are stored complemented (K - H), so that each of the
// six comparisons reads "query lane >= box lane"; the query's lanes carry a
// guard bit, and one subtraction per word then evaluates two comparisons:
// (0x8000 + a) - b keeps bit 15 exactly when a >= b, and never borrows from
// the next lane.
//   box words:   {L.x | L.y << 16, L.z | (K - H.x) << 16, (K - H.y) | (K - H.z) << 16}
//   query words: {c.x | c.y << 16, c.z | (K - c.x) << 16, (K - c.y) | (K - c.z) << 16}
//                (each | 0x80008000 on the device)
//
// Frames: super-chunk and chunk boxes use one frame around the domain
// (scale inv_g per axis).  The entries of a chunk use a frame derived from
// the chunk's own codes: origin fma(L_c, step_g, base_g) with step_g =
// 1 / inv_g and base_g = lo_g - step_g, scale inv_g * 2^e per axis, the
// exponents e (8 bits each) stored in the chunk's fourth word.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define P2M_HD __host__ __device__ __forceinline__
#else
#define P2M_HD inline
#endif

namespace p2m {

constexpr uint32_t kQMax = 32767;
constexpr uint32_t kQGuard = 0x80008000u;

P2M_HD uint32_t q_code(float x, float lo, float inv) {
#if defined(__CUDA_ARCH__)
  float t = __fmul_rn(__fsub_rn(x, lo), inv);
  t = fminf(fmaxf(t, -1.0f), (float)(kQMax - 1));
  return (uint32_t)(__float2int_rd(t) + 1);
#else
  volatile float d = x - lo;  // one rounding, as on the device
  float t = d * inv;
  t = std::fmin(std::fmax(t, -1.0f), (float)(kQMax - 1));
  return (uint32_t)((int)std::floor(t) + 1);
#endif
}

// the three words of six codes (lower bounds lo[3], upper bounds hi[3])
P2M_HD void q_words(const uint32_t *lo, const uint32_t *hi, uint32_t *w) {
  w[0] = lo[0] | lo[1] << 16;
  w[1] = lo[2] | (kQMax - hi[0]) << 16;
  w[2] = (kQMax - hi[1]) | (kQMax - hi[2]) << 16;
}

// the codes back from the words
P2M_HD void q_unwords(const uint32_t *w, uint32_t *lo, uint32_t *hi) {
  lo[0] = w[0] & 0xffffu;
  lo[1] = w[0] >> 16;
  lo[2] = w[1] & 0xffffu;
  hi[0] = kQMax - (w[1] >> 16);
  hi[1] = kQMax - (w[2] & 0xffffu);
  hi[2] = kQMax - (w[2] >> 16);
}

// step and base of a frame: step = 1 / inv, base = lo - step (float ops)
P2M_HD void q_frame_derive(const float *lo, const float *inv, float *step, float *base) {
  for (int d = 0; d < 3; ++d) {
#if defined(__CUDA_ARCH__)
    step[d] = __fdiv_rn(1.0f, inv[d]);
    base[d] = __fsub_rn(lo[d], step[d]);
#else
    volatile float s = 1.0f / inv[d];
    step[d] = s;
    volatile float b = lo[d] - s;
    base[d] = b;
#endif
  }
}

// 2^e as a float, 0 <= e <= 100
P2M_HD float q_pow2(uint32_t e) {
#if defined(__CUDA_ARCH__)
  return __int_as_float((int)((127u + e) << 23));
#else
  return std::ldexp(1.0f, (int)e);
#endif
}

// origin of the entry frame of a chunk on one axis: fma(L_c, step, base);
// on the device (float)L_c comes from a byte permute under the exponent of
// 2^23 and one subtraction (exact), not from a conversion instruction
P2M_HD float q_chunk_lo(uint32_t lc, float step, float base) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(__fsub_rn(__uint_as_float(0x4B000000u | lc), 8388608.0f), step, base);
#else
  return std::fma((float)lc, step, base);
#endif
}

// scale of the entry frame of a chunk on axis d: inv_g * 2^e (exact)
P2M_HD float q_chunk_inv(float inv_g, uint32_t w3, int d) {
  const uint32_t e = (w3 >> (8 * d)) & 0xffu;
#if defined(__CUDA_ARCH__)
  return __fmul_rn(inv_g, q_pow2(e));
#else
  return inv_g * q_pow2(e);
#endif
}

#if defined(__CUDACC__)
// the query's guarded words in a frame
__device__ __forceinline__ void q_query_words(float x, float y, float z, const float *lo,
                                              const float *inv, uint32_t *w) {
  const uint32_t cx = q_code(x, lo[0], inv[0]), cy = q_code(y, lo[1], inv[1]),
                 cz = q_code(z, lo[2], inv[2]);
  w[0] = (cx | cy << 16) | kQGuard;
  w[1] = (cz | (kQMax - cx) << 16) | kQGuard;
  w[2] = ((kQMax - cy) | (kQMax - cz) << 16) | kQGuard;
}

// all six comparisons of a query against a box
__device__ __forceinline__ bool q_pass(const uint32_t *q, uint32_t b0, uint32_t b1, uint32_t b2) {
  return (((q[0] - b0) & (q[1] - b1) & (q[2] - b2)) & kQGuard) == kQGuard;
}
#endif

}  // namespace p2m
