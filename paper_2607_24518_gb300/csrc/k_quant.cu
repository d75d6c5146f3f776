// FP8 E4M3 storage of S with one power-of-two scale per 128 x 128 tile
// (the setup step before the solver streams S; the paper runs FP32 only, so
// this storage format is this library's).  One CTA per tile: the tile is
// read once into registers, its largest magnitude fixes the scale, then the
// codes are written.  The FP64 sum of squares of the unquantised tile is
// written beside the scale so the caller can form ||S||_F^2 of the source.
#include <cuda_bf16.h>

#include "epi_common.cuh"
#include "symnmf_internal.h"

namespace symnmf {
namespace {

template <int SRC>
__device__ __forceinline__ float load_src(const void *p, int64_t i) {
  if constexpr (SRC == 0) {
    return __ldg(reinterpret_cast<const float *>(p) + i);
  } else {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
  }
}

// 256 threads: warp w covers rows 16 w .. 16 w + 15, lane l columns 4 l .. 4 l + 3
template <int SRC>
__global__ void __launch_bounds__(256) quantize_kernel(const void *src, int64_t rows, int64_t cols,
                                                       int64_t ld_src, uint8_t *q, int64_t ldq,
                                                       float *scales, int64_t ld_scales,
                                                       double *tile_sumsq) {
  __shared__ float wmax[8];
  __shared__ double wsum[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.y * kTileRows, c0 = (int64_t)blockIdx.x * kTileRows;
  float v[16][4];
  float m = 0.f;
  double ss = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int64_t r = r0 + warp * 16 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = c0 + lane * 4 + j;
      const float x = (r < rows && c < cols) ? load_src<SRC>(src, r * ld_src + c) : 0.f;
      v[i][j] = x;
      m = fmaxf(m, fabsf(x));
      ss = fma((double)x, (double)x, ss);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if (lane == 0) {
    wmax[warp] = m;
    wsum[warp] = ss;
  }
  __syncthreads();
  float amax = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) amax = fmaxf(amax, wmax[w]);
  const float sc = e4m3_tile_scale(amax), inv = 1.f / sc;
  if (threadIdx.x == 0) {
    scales[(int64_t)blockIdx.y * ld_scales + blockIdx.x] = sc;
    if (tile_sumsq) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += wsum[w];
      tile_sumsq[(int64_t)blockIdx.y * ld_scales + blockIdx.x] = t;
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int64_t r = r0 + warp * 16 + i;
    if (r >= rows) break;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = c0 + lane * 4 + j;
      if (c < cols) q[r * ldq + c] = e4m3_bits(v[i][j] * inv);
    }
  }
}

}  // namespace

cudaError_t launch_quantize_fp8(const void *src, int src_dtype, int64_t rows, int64_t cols,
                                int64_t ld_src, uint8_t *q, int64_t ldq, float *scales,
                                int64_t ld_scales, double *tile_sumsq, cudaStream_t s) {
  const dim3 grid((unsigned)((cols + kTileRows - 1) / kTileRows),
                  (unsigned)((rows + kTileRows - 1) / kTileRows));
  if (src_dtype == 0)
    quantize_kernel<0><<<grid, 256, 0, s>>>(src, rows, cols, ld_src, q, ldq, scales, ld_scales,
                                            tile_sumsq);
  else
    quantize_kernel<1><<<grid, 256, 0, s>>>(src, rows, cols, ld_src, q, ldq, scales, ld_scales,
                                            tile_sumsq);
  return cudaGetLastError();
}

}  // namespace symnmf
