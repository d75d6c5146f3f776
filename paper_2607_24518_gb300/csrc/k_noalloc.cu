// Objective f = ||S||^2 - 2 tr(H^T S H) + ||H^T H||^2 (Eq. 2) for a caller's
// S and H without a handle and without allocating device memory.
//
// Some callers cannot allocate at the moment they need an objective: a
// monitor thread that must not stall a running solve (cudaMalloc / cudaFree
// can synchronise the device), a process whose memory is fully reserved by
// another allocator, or code that has promised its host application a fixed
// device footprint.  This entry point serves them.  Its scratch is one
// fixed array in device memory, created with the library's module, so a
// call only launches kernels.
//
// Three kernels: (1) one CTA per (row tile, column share) multiplies its
// share of S by H (FP32 FMA) and immediately dots the partial product rows
// with H_I, leaving one FP64 partial of tr per CTA; (2) one CTA per row
// tile writes the FP32 Gram partial H_I^T H_I; (3) one CTA adds the
// partials in a fixed order in FP64 and writes f.  Every scratch slot that
// (3) reads is written by (1) or (2) earlier in the same call, so nothing
// in the scratch has to start at zero, and two calls with the same inputs
// give the same bits.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <mutex>

#include "../../include/symnmf.h"
#include "symnmf_internal.h"

namespace symnmf {
namespace {

constexpr int kSplit = 8;   // column shares per row tile in kernel (1)
constexpr int BK = 32;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SYMNMF_NOALLOC_SCRATCH_BYTES];

template <int DT>
__device__ __forceinline__ float load_s(const void *S, int64_t idx) {
  if constexpr (DT == 0) {
    return __ldg(reinterpret_cast<const float *>(S) + idx);
  } else if constexpr (DT == 1) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(S)[idx]);
  } else {
    __nv_fp8_e4m3 q;
    q.__x = reinterpret_cast<const __nv_fp8_storage_t *>(S)[idx];
    return static_cast<float>(q);
  }
}

struct ObjArgs {
  const void *S;
  int64_t n, lds;
  const float *scales;
  int64_t ld_scales;
  const float *H;   // n x k, row pitch k
  int k;
  int ntiles;
  double normS2;
  double *tr_part;  // ntiles * kSplit
  float *gram_part; // ntiles * kp * kp
  double *f;
};

// fixed-order sum over the block: xor tree per warp, warps in order
__device__ __forceinline__ double block_sum_fixed(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  __syncthreads();
  return r;  // valid in thread 0
}

template <int DT, int KP>
__global__ void __launch_bounds__(256) tr_share_kernel(ObjArgs a) {
  constexpr int CG = KP / 4, RG = 256 / CG, TM = 128 / RG;
  __shared__ float Ss[128][BK + 1];
  __shared__ __align__(16) float Hs[BK][KP];
  __shared__ double red[8];
  const int tid = threadIdx.x, tile = blockIdx.x, split = blockIdx.y;
  const int64_t r0 = (int64_t)tile * kTileRows;
  const int per = (a.ntiles + kSplit - 1) / kSplit;
  const int cb = split * per, ce = min(a.ntiles, cb + per);
  const int cg = tid % CG, rg = tid / CG;
  float acc[TM][4];
#pragma unroll
  for (int i = 0; i < TM; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  for (int ct = cb; ct < ce; ++ct) {
    const int64_t c0 = (int64_t)ct * kTileRows;
    float scale = 1.f;
    if constexpr (DT == 2) scale = a.scales[(int64_t)tile * a.ld_scales + ct];
    for (int kk = 0; kk < kTileRows; kk += BK) {
      for (int e = tid; e < 128 * BK; e += 256) {
        const int r = e / BK, c = e % BK;
        const int64_t gr = r0 + r, gc = c0 + kk + c;
        Ss[r][c] = (gr < a.n && gc < a.n) ? load_s<DT>(a.S, gr * a.lds + gc) * scale : 0.f;
      }
      for (int e = tid; e < BK * KP; e += 256) {
        const int r = e / KP, c = e % KP;
        const int64_t gr = c0 + kk + r;
        Hs[r][c] = (gr < a.n && c < a.k) ? a.H[gr * a.k + c] : 0.f;
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
  // this share's part of sum_{r, c} H_rc (S H)_rc over the tile's rows
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gr = r0 + rg + i * RG;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = cg * 4 + j;
      if (gr < a.n && c < a.k) t = fmaf(a.H[gr * a.k + c], acc[i][j], t);
    }
  }
  const double s = block_sum_fixed((double)t, red);
  if (tid == 0) a.tr_part[(int64_t)tile * kSplit + split] = s;
}

template <int KP>
__global__ void __launch_bounds__(256) gram_tile_kernel(ObjArgs a) {
  __shared__ float Hn[kTileRows][KP + 1];
  const int tile = blockIdx.x;
  const int64_t r0 = (int64_t)tile * kTileRows;
  for (int e = threadIdx.x; e < kTileRows * KP; e += blockDim.x) {
    const int r = e / KP, c = e % KP;
    Hn[r][c] = (r0 + r < a.n && c < a.k) ? a.H[(r0 + r) * a.k + c] : 0.f;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < KP * KP; q += blockDim.x) {
    // rows r = 4 i + g in four FMA chains, added (s0 + s1) + (s2 + s3): the
    // row order of the solver's Gram partials
    const int c = q / KP, d = q % KP;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int i = 0; i < kTileRows / 4; ++i)
#pragma unroll
      for (int g = 0; g < 4; ++g) s[g] = fmaf(Hn[4 * i + g][c], Hn[4 * i + g][d], s[g]);
    a.gram_part[(int64_t)tile * KP * KP + q] = (s[0] + s[1]) + (s[2] + s[3]);
  }
}

template <int KP>
__global__ void __launch_bounds__(256) finish_kernel(ObjArgs a) {
  __shared__ double red[8];
  const int tid = threadIdx.x;
  // tr: thread tid adds a contiguous run of partials, runs added in order
  const int64_t m = (int64_t)a.ntiles * kSplit;
  const int64_t per = (m + 255) / 256;
  double tr = 0.0;
  for (int64_t i = tid * per; i < m && i < (tid + 1) * per; ++i) tr += a.tr_part[i];
  // ||H^T H||^2: each Gram entry summed over tiles in tile order
  double g2 = 0.0;
  for (int q = tid; q < KP * KP; q += 256) {
    double g = 0.0;
    for (int t = 0; t < a.ntiles; ++t) g += (double)a.gram_part[(int64_t)t * KP * KP + q];
    g2 += g * g;
  }
  const double trs = block_sum_fixed(tr, red);
  const double g2s = block_sum_fixed(g2, red);
  if (tid == 0) *a.f = a.normS2 - 2.0 * trs + g2s;
}

template <int DT, int KP>
cudaError_t launch_all(const ObjArgs &a, cudaStream_t s) {
  tr_share_kernel<DT, KP><<<dim3(a.ntiles, kSplit), 256, 0, s>>>(a);
  gram_tile_kernel<KP><<<a.ntiles, 256, 0, s>>>(a);
  finish_kernel<KP><<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DT>
cudaError_t launch_dt(const ObjArgs &a, int kp, cudaStream_t s) {
  switch (kp) {
    case 8: return launch_all<DT, 8>(a, s);
    case 16: return launch_all<DT, 16>(a, s);
    case 32: return launch_all<DT, 32>(a, s);
    case 64: return launch_all<DT, 64>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {};

// Load every kernel this entry point launches on the current device.  With
// lazy module loading each kernel would otherwise be loaded at its first
// launch, i.e. inside some later call, which may allocate and synchronise.
template <int DT>
cudaError_t preload_dt() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tr_share_kernel<DT, 8>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tr_share_kernel<DT, 16>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tr_share_kernel<DT, 32>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tr_share_kernel<DT, 64>);
  return e;
}
template <int KP>
cudaError_t preload_kp() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, gram_tile_kernel<KP>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, finish_kernel<KP>);
  return e;
}
cudaError_t preload_kernels() {
  cudaError_t e = preload_dt<0>();
  if (e == cudaSuccess) e = preload_dt<1>();
  if (e == cudaSuccess) e = preload_dt<2>();
  if (e == cudaSuccess) e = preload_kp<8>();
  if (e == cudaSuccess) e = preload_kp<16>();
  if (e == cudaSuccess) e = preload_kp<32>();
  if (e == cudaSuccess) e = preload_kp<64>();
  return e;
}

// Argument and size check of the entry point, host arithmetic only.  On OK
// *need is the scratch the call uses and *kp the padded rank.
int noalloc_validate(bool have_S, int64_t n, int64_t lds, int32_t dtype, bool have_scales,
                     int64_t ld_scales, bool have_H, int32_t k, bool have_f, size_t *need,
                     int *kp_out) {
  if (!have_S || !have_H || !have_f || n < 1 || lds < n || k < 1 || k > 64)
    return SYMNMF_ERR_INVALID;
  if (dtype != SYMNMF_F32 && dtype != SYMNMF_BF16 && dtype != SYMNMF_FP8E4M3)
    return SYMNMF_ERR_INVALID;
  const int64_t ntiles = (n + kTileRows - 1) / kTileRows;
  if (dtype == SYMNMF_FP8E4M3 && (!have_scales || ld_scales < ntiles)) return SYMNMF_ERR_INVALID;
  const int kp = k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : 64;
  // scratch: ntiles * kSplit FP64 tr partials, then (256-byte aligned)
  // ntiles * kp * kp FP32 Gram partials
  const size_t tr_bytes = ((size_t)ntiles * kSplit * sizeof(double) + 255) & ~(size_t)255;
  *need = tr_bytes + (size_t)ntiles * kp * kp * sizeof(float);
  *kp_out = kp;
  if (ntiles > 65535 || *need > (size_t)SYMNMF_NOALLOC_SCRATCH_BYTES) return SYMNMF_ERR_UNSUPPORTED;
  return SYMNMF_OK;
}

}  // namespace
}  // namespace symnmf

using namespace symnmf;

extern "C" int symnmf_objective_noalloc_check(int64_t n, int64_t lds, int32_t dtype,
                                              int32_t have_scales, int64_t ld_scales, int32_t k,
                                              size_t *need) {
  size_t bytes = 0;
  int kp = 0;
  const int st = noalloc_validate(true, n, lds, dtype, have_scales != 0, ld_scales, true, k, true,
                                  &bytes, &kp);
  if (need) *need = bytes;
  return st;
}

extern "C" int symnmf_objective_noalloc(const void *S, int64_t n, int64_t lds, int32_t dtype,
                                        const float *scales, int64_t ld_scales, const float *H,
                                        int32_t k, double normS2, double *f, void *stream) {
  size_t need = 0;
  int kp = 0;
  const int st = noalloc_validate(S != nullptr, n, lds, dtype, scales != nullptr, ld_scales,
                                  H != nullptr, k, f != nullptr, &need, &kp);
  if (st != SYMNMF_OK) return st;
  const int64_t ntiles = (n + kTileRows - 1) / kTileRows;
  const size_t tr_bytes = ((size_t)ntiles * kSplit * sizeof(double) + 255) & ~(size_t)255;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SYMNMF_ERR_CUDA;
  void *base = nullptr;
  {
    // first call on a device: look up that device's copy of the scratch
    // (this loads the library's module there, creating the array) and load
    // every kernel of this entry point, so later calls only launch
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess ||
          preload_kernels() != cudaSuccess) {
        cudaGetLastError();
        return SYMNMF_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  ObjArgs a{};
  a.S = S;
  a.n = n;
  a.lds = lds;
  a.scales = scales;
  a.ld_scales = ld_scales;
  a.H = H;
  a.k = k;
  a.ntiles = (int)ntiles;
  a.normS2 = normS2;
  a.tr_part = reinterpret_cast<double *>(base);
  a.gram_part = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(base) + tr_bytes);
  a.f = f;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  switch (dtype) {
    case SYMNMF_F32: e = launch_dt<0>(a, kp, s); break;
    case SYMNMF_BF16: e = launch_dt<1>(a, kp, s); break;
    default: e = launch_dt<2>(a, kp, s); break;
  }
  return e == cudaSuccess ? SYMNMF_OK : SYMNMF_ERR_CUDA;
}
