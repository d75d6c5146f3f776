// Spherical K-means (Lloyd) on the rows of S (Sec. 6, "Clustering
// alternatives"): the rows s_i are normalised, x_i = s_i / ||s_i||, each
// cluster's centroid is the normalised sum of its members, and each row
// joins the cluster of largest cosine.  One Lloyd iteration is two passes
// of the streamed product with n x K operands (S symmetric):
//   C = S (D^-1 B)             columns c_k = sum_{i in C_k} x_i
//   P = S C                    P_ik = <s_i, c_k>
//   cos_ik = P_ik / (||s_i|| ||c_k||),  L'(i) = first argmax_k cos_ik,
//   J = sum_i (1 - max_k cos_ik).
// The kernels here are the small ones around the two product passes: row
// norms (once per matrix), the operand D^-1 B from the labels, the centroid
// gather with per-tile FP64 column sums of squares, the centroid norms, the
// assignment with per-tile FP64 objective partials, and the final
// fixed-order sum.  Every cross-tile sum is FP64 in tile order, so a run is
// bit-reproducible.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "../../include/symnmf.h"
#include "epi_common.cuh"
#include "symnmf_internal.h"

namespace symnmf {
namespace {

template <int DT>
__device__ __forceinline__ double s_at(const void *S, int64_t idx) {
  if constexpr (DT == 0) {
    return (double)reinterpret_cast<const float *>(S)[idx];
  } else if constexpr (DT == 1) {
    return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(S)[idx]);
  } else {
    __nv_fp8_e4m3 q;
    q.__x = reinterpret_cast<const __nv_fp8_storage_t *>(S)[idx];
    return (double)static_cast<float>(q);
  }
}

// ||s_i|| in FP64: one warp per row, lanes over columns, xor tree
template <int DT>
__global__ void __launch_bounds__(256) row_norms_kernel(const void *S, int64_t n, int64_t lds,
                                                        const float *scales, int64_t ld_scales,
                                                        double *rn) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double acc = 0.0;
  for (int64_t c = lane; c < n; c += 32) {
    double v = s_at<DT>(S, row * lds + c);
    if constexpr (DT == 2) v *= (double)scales[(row / kTileRows) * ld_scales + c / kTileRows];
    acc += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) rn[row] = sqrt(acc);
}

// operand D^-1 B: row i holds 1 / ||s_i|| in column labels[i]
template <int KP>
__global__ void km_operand_kernel(const int *labels, const double *rn, int64_t n, float *H,
                                  int64_t rows_alloc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows_alloc * KP) return;
  const int64_t r = e / KP;
  const int c = (int)(e % KP);
  float v = 0.f;
  if (r < n && labels[r] == c) v = (float)(1.0 / rn[r]);
  H[e] = v;
}

// centroid rows C_I = sum of the partials, and per-tile FP64 column sums of
// squares (column order, rows in order)
template <int KP>
__global__ void __launch_bounds__(256) km_centroid_kernel(KmArgs a) {
  __shared__ float Cs[kTileRows][KP + 1];
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int64_t r0 = (int64_t)tile * kTileRows;
  int64_t b0, b1;
  part_range(tile, a.skG, a.ncols, a.ntiles, b0, b1);
  for (int e = tid; e < kTileRows * KP; e += blockDim.x) {
    const int r = e / KP, c = e % KP;
    float v = 0.f;
    if (r0 + r < a.n && c < a.K)
      v = part_sum<KP>(a.P, a.nsplit, a.skG, a.ncols, a.ntiles, tile, r, c, b0, b1);
    Cs[r][c] = v;
    a.C[(r0 + r) * KP + c] = v;
  }
  __syncthreads();
  if (tid < KP) {
    double s = 0.0;
    for (int r = 0; r < kTileRows; ++r) {
      const double v = (double)Cs[r][tid];
      s += v * v;
    }
    a.colsq[(int64_t)tile * KP + tid] = s;
  }
}

// ||c_k||: fixed-order sum over tiles; inv_norm = 0 for an empty cluster
template <int KP>
__global__ void km_norms_kernel(KmArgs a) {
  const int c = threadIdx.x;
  if (c >= KP) return;
  double s = 0.0;
  for (int t = 0; t < a.ntiles; ++t) s += a.colsq[(int64_t)t * KP + c];
  const double nk = sqrt(s);
  a.inv_norm[c] = (c < a.K && nk > 0.0) ? (float)(1.0 / nk) : 0.f;
}

// assignment: one thread per row; first argmax over k < K of P_ik / ||c_k||
// (the row's 1 / ||s_i|| is common to all k); per-tile FP64 sums of
// 1 - cos and of the changed labels
template <int KP>
__global__ void __launch_bounds__(kTileRows) km_assign_kernel(KmArgs a) {
  __shared__ double red[40];
  const int tile = blockIdx.x, r = threadIdx.x;
  const int64_t row = (int64_t)tile * kTileRows + r;
  int64_t b0, b1;
  part_range(tile, a.skG, a.ncols, a.ntiles, b0, b1);
  double j = 0.0, ch = 0.0;
  if (row < a.n) {
    int best = 0;
    float bs = 0.f;
    for (int c = 0; c < a.K; ++c) {
      const float p = part_sum<KP>(a.P, a.nsplit, a.skG, a.ncols, a.ntiles, tile, r, c, b0, b1);
      const float sc = p * a.inv_norm[c];
      if (c == 0 || sc > bs) {
        bs = sc;
        best = c;
      }
    }
    const double cosv = (double)bs / a.rn[row];
    j = 1.0 - cosv;
    a.labels_out[row] = best;
    ch = (best != a.labels_in[row]) ? 1.0 : 0.0;
  }
  // fixed-order block sums: xor tree per warp, warps in order
  double v[2] = {j, ch};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  if ((r & 31) == 0) {
    red[(r >> 5) * 2 + 0] = v[0];
    red[(r >> 5) * 2 + 1] = v[1];
  }
  __syncthreads();
  if (r == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kTileRows / 32; ++w) {
      s0 += red[2 * w];
      s1 += red[2 * w + 1];
    }
    a.slots[(int64_t)tile * 2 + 0] = s0;
    a.slots[(int64_t)tile * 2 + 1] = s1;
  }
}

// J and the changed count: runs of tiles per thread, runs in order
__global__ void __launch_bounds__(256) km_final_kernel(KmArgs a) {
  __shared__ double red[2][8];
  const int tid = threadIdx.x;
  const int per = (a.ntiles + 255) / 256;
  double s0 = 0.0, s1 = 0.0;
  for (int t = tid * per; t < a.ntiles && t < (tid + 1) * per; ++t) {
    s0 += a.slots[(int64_t)t * 2];
    s1 += a.slots[(int64_t)t * 2 + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = s0;
    red[1][tid >> 5] = s1;
  }
  __syncthreads();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < 8; ++w) {
      t0 += red[0][w];
      t1 += red[1][w];
    }
    a.out[0] = t0;
    a.out[1] = t1;
  }
}

}  // namespace

#define KM_KP_SWITCH(kp, ...)                                \
  switch (kp) {                                              \
    case 8: { constexpr int KPV = 8; __VA_ARGS__; } break;   \
    case 16: { constexpr int KPV = 16; __VA_ARGS__; } break; \
    case 32: { constexpr int KPV = 32; __VA_ARGS__; } break; \
    case 64: { constexpr int KPV = 64; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;                   \
  }

cudaError_t launch_row_norms(const void *S, int64_t n, int64_t lds, int dtype, const float *scales,
                             int64_t ld_scales, double *rn, cudaStream_t s) {
  const unsigned blocks = (unsigned)((n + 7) / 8);
  switch (dtype) {
    case 0: row_norms_kernel<0><<<blocks, 256, 0, s>>>(S, n, lds, scales, ld_scales, rn); break;
    case 1: row_norms_kernel<1><<<blocks, 256, 0, s>>>(S, n, lds, scales, ld_scales, rn); break;
    case 2: row_norms_kernel<2><<<blocks, 256, 0, s>>>(S, n, lds, scales, ld_scales, rn); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_km_operand(const int *labels, const double *rn, int64_t n, int kp, float *H,
                              int64_t rows_alloc, cudaStream_t s) {
  const int64_t total = rows_alloc * kp;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  KM_KP_SWITCH(kp, km_operand_kernel<KPV><<<blocks, 256, 0, s>>>(labels, rn, n, H, rows_alloc));
  return cudaGetLastError();
}

cudaError_t launch_km_centroids(const KmArgs &a, int kp, cudaStream_t s) {
  KM_KP_SWITCH(kp, {
    km_centroid_kernel<KPV><<<a.ntiles, 256, 0, s>>>(a);
    km_norms_kernel<KPV><<<1, 64, 0, s>>>(a);
  });
  return cudaGetLastError();
}

cudaError_t launch_km_assign(const KmArgs &a, int kp, cudaStream_t s) {
  KM_KP_SWITCH(kp, km_assign_kernel<KPV><<<a.ntiles, kTileRows, 0, s>>>(a));
  km_final_kernel<<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace symnmf
