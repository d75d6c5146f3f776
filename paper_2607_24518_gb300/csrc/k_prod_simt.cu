// SIMT product P = S[rows, cols] * H[cols] (Sec. 2.1: the S H term of the
// gradient), FP32 FFMA with FP32 accumulation.  This is the exact-FP32
// path and the fallback for layouts the tensor-core kernel cannot take
// (S row pitch not a multiple of 16 bytes).  One CTA owns one 128-row tile
// and a contiguous share (split) of the column-tile list; partial sums go
// to out[split][row_pos] and are added in split order by the epilogue.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "symnmf_internal.h"

namespace symnmf {
namespace {

constexpr int BK = 32;

template <int DT>
__device__ __forceinline__ float load_s(const void *S, int64_t idx) {
  if constexpr (DT == 0) {
    return __ldg(reinterpret_cast<const float *>(S) + idx);
  } else if constexpr (DT == 1) {
    const __nv_bfloat16 *p = reinterpret_cast<const __nv_bfloat16 *>(S) + idx;
    return __bfloat162float(*p);
  } else {
    __nv_fp8_e4m3 q;
    q.__x = reinterpret_cast<const __nv_fp8_storage_t *>(S)[idx];
    return static_cast<float>(q);
  }
}

template <int DT, int KP>
__global__ void __launch_bounds__(256) prod_simt_kernel(ProdArgs a) {
  constexpr int CG = KP / 4;    // column groups of 4
  constexpr int RG = 256 / CG;  // row groups
  constexpr int TM = 128 / RG;  // rows per thread
  __shared__ float Ss[128][BK + 1];
  __shared__ __align__(16) float Hs[BK][KP];
  const int tid = threadIdx.x;
  const int pos = blockIdx.x;
  const int split = blockIdx.y;
  const int rt = a.row_list ? a.row_list[pos] : pos;
  const int64_t r0 = (int64_t)rt * kTileRows;
  const int per = (a.n_cols_list + a.nsplit - 1) / a.nsplit;
  const int cb = split * per;
  const int ce = min(a.n_cols_list, cb + per);
  const int cg = tid % CG, rg = tid / CG;
  float acc[TM][4];
#pragma unroll
  for (int i = 0; i < TM; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;

  for (int ci = cb; ci < ce; ++ci) {
    const int ct = a.col_list ? a.col_list[ci] : ci;
    const int64_t c0 = (int64_t)ct * kTileRows;
    float scale = 1.f;
    if constexpr (DT == 2) scale = a.scales[(int64_t)rt * a.ld_scales + ct];
    for (int kk = 0; kk < kTileRows; kk += BK) {
      for (int e = tid; e < 128 * BK; e += 256) {
        const int r = e / BK, c = e % BK;
        const int64_t gr = r0 + r, gc = c0 + kk + c;
        float v = 0.f;
        if (gr < a.n && gc < a.n) v = load_s<DT>(a.S, gr * a.lds + gc) * scale;
        Ss[r][c] = v;
      }
      for (int e = tid; e < BK * KP; e += 256) {
        const int r = e / KP, c = e % KP;
        const int64_t gr = c0 + kk + r;
        Hs[r][c] = (gr < a.n) ? a.H[gr * KP + c] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int x = 0; x < BK; ++x) {
        const float4 hv = *reinterpret_cast<const float4 *>(&Hs[x][cg * 4]);
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const float sv = Ss[rg + i * RG][x];
          acc[i][0] = fmaf(sv, hv.x, acc[i][0]);
          acc[i][1] = fmaf(sv, hv.y, acc[i][1]);
          acc[i][2] = fmaf(sv, hv.z, acc[i][2]);
          acc[i][3] = fmaf(sv, hv.w, acc[i][3]);
        }
      }
      __syncthreads();
    }
  }
  float *out = a.out + ((int64_t)split * a.n_rows_list + pos) * kTileRows * KP;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = rg + i * RG;
    *reinterpret_cast<float4 *>(&out[r * KP + cg * 4]) =
        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

template <int DT>
cudaError_t launch_dt(const ProdArgs &a, cudaStream_t s) {
  dim3 grid(a.n_rows_list, a.nsplit);
  switch (a.kp) {
    case 8: prod_simt_kernel<DT, 8><<<grid, 256, 0, s>>>(a); break;
    case 16: prod_simt_kernel<DT, 16><<<grid, 256, 0, s>>>(a); break;
    case 32: prod_simt_kernel<DT, 32><<<grid, 256, 0, s>>>(a); break;
    case 64: prod_simt_kernel<DT, 64><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prod_simt(const ProdArgs &a, cudaStream_t s) {
  if (a.n_rows_list <= 0 || a.n_cols_list <= 0) return cudaSuccess;
  switch (a.dtype) {
    case 0: return launch_dt<0>(a, s);
    case 1: return launch_dt<1>(a, s);
    case 2: return launch_dt<2>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace symnmf
