// Per-restart check quantities for restarts concatenated along N (the k
// columns of H hold R independent solves of rank kb = k / R).  At a check
// the fused step has written the gradient g of H_t, and with the Gram of
// H_t block diagonal each restart's objective follows from two sums over
// its column block (Sec. 2.1: S H = H Gram - g / 4, so
// tr(H_r^T S H_r) = ||Gram_rr||^2 - sum H_r .* g_r / 4):
//   f_r = ||S||^2 - ||Gram_rr||^2 + sum(H_r .* g_r) / 2
// and its KKT measure from the projected gradient (Eq. 6) of the block;
// the sum of the block's accumulator drives Piecewise AdaGrad's cooldown.
#include "restart_stats.h"

namespace symnmf {
namespace {

constexpr int kMaxR = 8;  // k <= 64 and kb >= 8

constexpr int kQ = kRestartSums;

__global__ void __launch_bounds__(128) restart_tile_kernel(const float *H, const float *g,
                                                           const float *A, int64_t n, int k,
                                                           int kp, int R, double *part) {
  __shared__ double red[4][kQ * kMaxR];
  const int tile = blockIdx.x, r = threadIdx.x;
  const int64_t row = (int64_t)tile * 128 + r;
  const int kb = k / R;
  double s[kQ * kMaxR];
#pragma unroll
  for (int q = 0; q < kQ * kMaxR; ++q) s[q] = 0.0;
  if (row < n) {
    for (int c = 0; c < k; ++c) {
      const double h = (double)H[row * kp + c], gv = (double)g[row * kp + c];
      const double av = (double)A[row * kp + c];
      const double pg = h > 0.0 ? gv : (gv < 0.0 ? gv : 0.0);
      const int b = c / kb;
#pragma unroll
      for (int q = 0; q < kMaxR; ++q)
        if (q == b) {
          s[kQ * q] += h * gv;
          s[kQ * q + 1] += pg * pg;
          s[kQ * q + 2] += av;
        }
    }
  }
  // fixed order: xor tree per warp, warps in order
#pragma unroll
  for (int q = 0; q < kQ * kMaxR; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
  }
  if ((r & 31) == 0)
#pragma unroll
    for (int q = 0; q < kQ * kMaxR; ++q) red[r >> 5][q] = s[q];
  __syncthreads();
  if (r < kQ * R)
    part[(int64_t)tile * kQ * R + r] = red[0][r] + red[1][r] + red[2][r] + red[3][r];
}

__global__ void restart_sum_kernel(const double *part, int ntiles, int R, double *out) {
  const int q = threadIdx.x;
  if (q >= kQ * R) return;
  double v = 0.0;
  for (int t = 0; t < ntiles; ++t) v += part[(int64_t)t * kQ * R + q];
  out[q] = v;
}

}  // namespace

cudaError_t launch_restart_stats(const float *H, const float *g, const float *A, int64_t n, int k,
                                 int kp, int R, double *part, double *out, cudaStream_t s) {
  if (R < 1 || R > kMaxR || k % R != 0) return cudaErrorInvalidValue;
  const int ntiles = (int)((n + 127) / 128);
  restart_tile_kernel<<<ntiles, 128, 0, s>>>(H, g, A, n, k, kp, R, part);
  restart_sum_kernel<<<1, 32, 0, s>>>(part, ntiles, R, out);
  return cudaGetLastError();
}

}  // namespace symnmf
