// Device helpers shared by the stand-alone epilogue and reduction kernels
// and the fused epilogue of the tensor-core kernels: number formats of the
// MMA copy of H, the stream-K slot arithmetic, and fixed-order summation.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>

#include "../../include/symnmf.h"
#include "symnmf_internal.h"

namespace symnmf {

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t *>(&b);
}
__device__ __forceinline__ float bf16_val(uint16_t u) {
  __nv_bfloat16 b = *reinterpret_cast<__nv_bfloat16 *>(&u);
  return __bfloat162float(b);
}
// tf32 value of x >= 0 with the 13 low mantissa bits cleared
__device__ __forceinline__ float tf32_trunc(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}
// x >= 0 rounded to the nearest tf32 value (ties away from zero)
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// OCP E4M3 code of x, round to nearest even, saturating at +-448
__device__ __forceinline__ uint8_t e4m3_bits(float x) {
  return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float e4m3_val(uint8_t u) {
  return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)u, __NV_E4M3)));
}
// smallest power of two d with amax / d <= 448 (1 for amax = 0 or not
// finite).  With amax = m 2^E, m in [0.5, 1): amax / 448 = (m / 1.75)
// 2^(E-8), so d = 2^(E-9) when m <= 0.875 and 2^(E-8) otherwise; frexpf
// is exact, so the decision is exact.
__device__ __forceinline__ float e4m3_tile_scale(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  int E;
  const float m = frexpf(amax, &E);
  int e = E - 9 + (m > 0.875f ? 1 : 0);
  if (e < -100) e = -100;
  return ldexpf(1.f, e);
}
// two-piece E4M3 form of h at tile factor d: h ~ d (hi + lo), hi the
// E4M3 value of h / d and lo that of the remainder h / d - hi (exact in
// FP32), both rounded to nearest even
__device__ __forceinline__ void e4m3_pieces(float h, float inv_d, uint8_t &hi, uint8_t &lo) {
  const float x = h * inv_d;
  hi = e4m3_bits(x);
  lo = e4m3_bits(x - e4m3_val(hi));
}

// CTA of a stream-K launch whose unit range [b W / G, (b+1) W / G) holds x
__device__ __forceinline__ int64_t sk_cta(int64_t x, int64_t W, int64_t G) {
  int64_t b = x * G / W;
  while (b + 1 < G && (b + 1) * W / G <= x) ++b;
  while (b > 0 && b * W / G > x) --b;
  return b;
}

// Partials of a product launch that ran without the fused epilogue: with
// the stream-K layout (skG > 0) CTAs b0..b1 hold row position p's partials
// in slots b + p; the SIMT layout has nsplit column shares per position.
// part_sum adds the partials of row r, column c in that fixed order.
__device__ __forceinline__ void part_range(int p, int skG, int ncols, int nlist, int64_t &b0,
                                           int64_t &b1) {
  b0 = b1 = 0;
  if (skG > 0) {
    const int64_t W = (int64_t)nlist * ncols;
    b0 = sk_cta((int64_t)p * ncols, W, skG);
    b1 = sk_cta((int64_t)p * ncols + ncols - 1, W, skG);
  }
}
template <int KP>
__device__ __forceinline__ float part_sum(const float *P, int nsplit, int skG, int ncols, int nlist,
                                          int p, int r, int c, int64_t b0, int64_t b1) {
  float v = 0.f;
  if (skG > 0) {
    for (int64_t b = b0; b <= b1; ++b) v += P[((b + p) * kTileRows + r) * KP + c];
  } else {
    for (int s = 0; s < nsplit; ++s) v += P[(((int64_t)s * nlist + p) * kTileRows + r) * KP + c];
  }
  return v;
}

// num / (sqrt(v) + eps), the AdaGrad / RMSprop step (Sec. 2.2), in
// straight-line code: PTX sqrt.approx.f32 (relative error at most 2^-23)
// and div.full.f32 (at most 2 ulp over the full range).  With no
// out-of-line special-case path the columns of a row overlap in flight.
__device__ __forceinline__ float adaptive_step(float num, float v, float eps) {
  float r, q;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
  asm("div.full.f32 %0, %1, %2;" : "=f"(q) : "f"(num), "f"(r + eps));
  return q;
}

// Row order of every Gram partial (H_tile^T H_tile over a 128-row tile):
// entry (c, d) is (s_0 + s_1) + (s_2 + s_3), s_g the FMA chain over the rows
// r = 4 i + g, i = 0..31 in order, starting from zero.  gram_entry forms it
// from a tile in shared memory; gram_quad_sum adds the four s_g held by the
// lanes 4 q + g of a quad (every lane of the quad gets the same bits).
template <int KP>
__device__ __forceinline__ float gram_entry(const float (*Hn)[KP + 1], int c, int d) {
  float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int i = 0; i < kTileRows / 4; ++i)
#pragma unroll
    for (int g = 0; g < 4; ++g) s[g] = fmaf(Hn[4 * i + g][c], Hn[4 * i + g][d], s[g]);
  return (s[0] + s[1]) + (s[2] + s[3]);
}
__device__ __forceinline__ float gram_quad_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// (hi, lo) += (hi, lo) of lane ^ o for non-overlapping float pairs: the
// high parts by Knuth's TwoSum (exact: s + err = a + b), the low parts and
// err added and renormalised by Fast2Sum.  Relative error near 2^-44; both
// lanes of the pair get the same bits.
__device__ __forceinline__ void ff_xor_add(float &hi, float &lo, int o) {
  const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
  const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
  const float s = __fadd_rn(hi, bh);
  const float v = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(bh, v));
  const float t = __fadd_rn(__fadd_rn(lo, bl), err);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// Sum, in index order, `count` (<= 32) values at base[i * stride]; every
// load is issued before the ordered additions.
template <typename T>
__device__ __forceinline__ double ordered_sum32(const T *base, int64_t stride, int count) {
  double v[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = (j < count) ? (double)base[(int64_t)j * stride] : 0.0;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 32; ++j) s += v[j];
  return s;
}

// Fixed-order sum over nthr threads (et = 0..nthr-1): xor tree inside each
// warp, then warp partials added in warp order.  scratch holds >= 33
// doubles; bar() synchronises the participating threads.
template <class Bar>
__device__ __forceinline__ double group_sum(double v, int et, int nthr, Bar bar, double *scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  bar();
  if ((et & 31) == 0) scratch[et >> 5] = v;
  bar();
  if (et == 0) {
    double r = 0.0;
    for (int i = 0; i < (nthr >> 5); ++i) r += scratch[i];
    scratch[32] = r;
  }
  bar();
  return scratch[32];
}

}  // namespace symnmf
