// quant.h -- 16-bit box coordinates of the interception lists.
//
// A coordinate x inside a frame [lo, hi] is stored as q in 0..65535 and
// read back as fma(q, step, lo), step = (hi - lo) / 65534.  The step is a
// little larger than (hi - lo) / 65535, so q = 65535 always reads back at
// or above hi despite float rounding.  The encoder (host) rounds every box
// outward and re-reads it with exactly the decoder's float operations, so a
// decoded box always contains the true one.  Chunk boxes use a fixed frame
// around the domain; entry boxes use the decoded box of their chunk.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define P2M_HD __host__ __device__ __forceinline__
#else
#define P2M_HD inline
#endif

namespace p2m {

constexpr float kQInv = 1.0f / 65534.0f;

P2M_HD float q_step(float lo, float hi) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(__fsub_rn(hi, lo), kQInv);
#else
  return (hi - lo) * kQInv;
#endif
}

P2M_HD float q_dec(uint32_t q, float lo, float step) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn((float)q, step, lo);
#else
  return std::fmaf((float)q, step, lo);
#endif
}

// largest q whose value is <= x (x >= lo)
inline uint32_t q_enc_lo(float x, float lo, float step) {
  if (!(step > 0.f)) return 0;
  double e = std::floor(((double)x - (double)lo) / (double)step);
  uint32_t q = (uint32_t)std::min(65535.0, std::max(0.0, e));
  while (q > 0 && q_dec(q, lo, step) > x) --q;
  while (q < 65535 && q_dec(q + 1, lo, step) <= x) ++q;
  return q;
}

// smallest q whose value is >= x (x <= the frame's hi)
inline uint32_t q_enc_hi(float x, float lo, float step) {
  if (!(step > 0.f)) return 0;
  double e = std::ceil(((double)x - (double)lo) / (double)step);
  uint32_t q = (uint32_t)std::min(65535.0, std::max(0.0, e));
  while (q < 65535 && q_dec(q, lo, step) < x) ++q;
  while (q > 0 && q_dec(q - 1, lo, step) >= x) --q;
  return q;
}

#if defined(__CUDA_ARCH__)
// (float)q of the low (h = 0) or high (h = 1) half of w without an
// int-to-float conversion: one byte permute places the 16 bits under the
// exponent of 2^23, so the word reads as 2^23 + q exactly, and subtracting
// 2^23 leaves q exactly.  Same value as the conversion, on the ALU and FMA
// pipes instead of the conversion unit.
template <int h>
__device__ __forceinline__ float q_half(uint32_t w) {
  return __fsub_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, h ? 0x7432u : 0x7410u)),
                   8388608.0f);
}

__device__ __forceinline__ float q_dec_f(float qf, float lo, float step) {
  return __fmaf_rn(qf, step, lo);
}
#endif

// a packed box: 6 x 16 bits in words w0..w2 (lo.x, lo.y | lo.z, hi.x | hi.y, hi.z)
P2M_HD void q_unpack(uint32_t w0, uint32_t w1, uint32_t w2, const float *lo, const float *step,
                     float *blo, float *bhi) {
#if defined(__CUDA_ARCH__)
  blo[0] = q_dec_f(q_half<0>(w0), lo[0], step[0]);
  blo[1] = q_dec_f(q_half<1>(w0), lo[1], step[1]);
  blo[2] = q_dec_f(q_half<0>(w1), lo[2], step[2]);
  bhi[0] = q_dec_f(q_half<1>(w1), lo[0], step[0]);
  bhi[1] = q_dec_f(q_half<0>(w2), lo[1], step[1]);
  bhi[2] = q_dec_f(q_half<1>(w2), lo[2], step[2]);
#else
  blo[0] = q_dec(w0 & 0xffffu, lo[0], step[0]);
  blo[1] = q_dec(w0 >> 16, lo[1], step[1]);
  blo[2] = q_dec(w1 & 0xffffu, lo[2], step[2]);
  bhi[0] = q_dec(w1 >> 16, lo[0], step[0]);
  bhi[1] = q_dec(w2 & 0xffffu, lo[1], step[1]);
  bhi[2] = q_dec(w2 >> 16, lo[2], step[2]);
#endif
}

}  // namespace p2m
