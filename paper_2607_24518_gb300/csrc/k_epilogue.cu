// Per-tile epilogue of one solver iteration and the fixed-order reductions.
//
// For each 128-row tile I the epilogue forms the gradient rows
//   g_I = 4 (H_I Gram_t - (S H)_I)                          (Sec. 2.1)
// or the Row-SVRG / Block-SVRG estimates (Sec. 5.1; appendix), applies the
// AdaGrad or RMSprop update with the max(0, .) projection (appendix,
// Family 3; Sec. 2.4 "Projected space") into the other H buffer, writes the
// bf16 hi/lo MMA copy of the new rows, and produces the per-tile partials
// tr_I = sum H_I * (S H)_I (Eq. 2), ||grad_proj||^2_I (Eq. 6), sum(G)_I, the
// NaN/Inf count and the Gram partial H'_I^T H'_I.  Within a tile sums are
// FP32 in a fixed order; across tiles they are FP64 in tile order
// (launch_reduce), so every result is bit-reproducible run to run.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "../../include/symnmf.h"
#include "epi_common.cuh"
#include "symnmf_internal.h"

namespace symnmf {
namespace {

__device__ __forceinline__ double block_sum(double v, double *sh) {
  // fixed-order: xor tree within the warp, then warp 0 adds warps in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) r += sh[i];
    sh[32] = r;
  }
  __syncthreads();
  return sh[32];
}

// writes the transposed MMA copy (format bt_fmt) and the Gram partial of
// the tile held in smem Hn[128][KP+1]; every thread of the block calls it
template <int KP>
__device__ void tile_tail(const float (*Hn)[KP + 1], int64_t r0, void *Bt, int bt_fmt, int64_t ldb,
                          float *gram_part, int tile) {
  const int tid = threadIdx.x;
  if (Bt && bt_fmt == 0) {
    uint16_t *B = reinterpret_cast<uint16_t *>(Bt);
    for (int e = tid; e < KP * kTileRows; e += blockDim.x) {
      const int c = e / kTileRows, r = e % kTileRows;
      const float v = Hn[r][c];
      const uint16_t hi = bf16_bits(v);
      const uint16_t lo = bf16_bits(v - bf16_val(hi));
      B[(int64_t)c * ldb + r0 + r] = hi;
      B[(int64_t)(KP + c) * ldb + r0 + r] = lo;
    }
  } else if (Bt && bt_fmt == 2) {
    // tile factor d from the tile's largest entry (H >= 0), then the pieces
    __shared__ float wmax[32];
    float m = 0.f;
    for (int e = tid; e < KP * kTileRows; e += blockDim.x) m = fmaxf(m, Hn[e % kTileRows][e / kTileRows]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) wmax[tid >> 5] = m;
    __syncthreads();
    float amax = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) amax = fmaxf(amax, wmax[w]);
    const float d = e4m3_tile_scale(amax), inv = 1.f / d;
    uint8_t *B = reinterpret_cast<uint8_t *>(Bt);
    for (int e = tid; e < KP * kTileRows; e += blockDim.x) {
      const int c = e / kTileRows, r = e % kTileRows;
      uint8_t hi, lo;
      e4m3_pieces(Hn[r][c], inv, hi, lo);
      B[(int64_t)c * ldb + r0 + r] = hi;
      B[(int64_t)(KP + c) * ldb + r0 + r] = lo;
    }
    if (tid == 0) bt_deq(Bt, KP, ldb)[tile] = d;
    __syncthreads();
  } else if (Bt) {
    float *B = reinterpret_cast<float *>(Bt);
    uint16_t *B16 = bt_b16(Bt, KP, ldb);
    for (int e = tid; e < KP * kTileRows; e += blockDim.x) {
      const int c = e / kTileRows, r = e % kTileRows;
      const float v = Hn[r][c];
      const float hi = tf32_trunc(v);
      B[(int64_t)c * ldb + r0 + r] = hi;
      B[(int64_t)(KP + c) * ldb + r0 + r] = tf32_round(v - hi);
      B16[(int64_t)c * ldb + r0 + r] = bf16_bits(v);
    }
  }
  if (gram_part) {
    for (int q = tid; q < KP * KP; q += blockDim.x)
      gram_part[(int64_t)tile * KP * KP + q] = gram_entry<KP>(Hn, q / KP, q % KP);
  }
}

template <int KP>
constexpr size_t epi_smem_bytes() {
  return (size_t)(2 * kTileRows * (KP + 1) + 2 * KP * (KP + 1)) * sizeof(float);
}

constexpr int kEpiThreads = 512;

template <int KP>
__global__ void __launch_bounds__(kEpiThreads) epilogue_kernel(EpiArgs a) {
  constexpr int EPT = kTileRows * KP / kEpiThreads;  // elements per thread
  extern __shared__ float smem_epi[];
  float(*Hs)[KP + 1] = reinterpret_cast<float(*)[KP + 1]>(smem_epi);
  float(*Hn)[KP + 1] = reinterpret_cast<float(*)[KP + 1]>(smem_epi + kTileRows * (KP + 1));
  float(*G1)[KP + 1] = reinterpret_cast<float(*)[KP + 1]>(smem_epi + 2 * kTileRows * (KP + 1));
  float(*G2)[KP + 1] =
      reinterpret_cast<float(*)[KP + 1]>(smem_epi + 2 * kTileRows * (KP + 1) + KP * (KP + 1));
  __shared__ double red[40];
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int64_t r0 = (int64_t)tile * kTileRows;
  const int rows = (int)((a.n - r0) < kTileRows ? (a.n - r0) : kTileRows);
  const float *__restrict__ Hg = a.H;
  for (int e = tid; e < kTileRows * KP; e += kEpiThreads) {
    const int r = e / KP, c = e % KP;
    Hs[r][c] = (r < rows) ? Hg[(r0 + r) * KP + c] : 0.f;
  }
  const bool block = (a.mode == MODE_BLOCK);
  const float *g1src = block ? a.gramJ : a.gram;
  for (int e = tid; e < KP * KP; e += kEpiThreads) {
    G1[e / KP][e % KP] = g1src[e];
    if (block) G2[e / KP][e % KP] = a.gramI[e];
  }
  int p1 = -1, p2 = -1, p3 = -1;
  if (a.mode == MODE_FULL || a.mode == MODE_GRAD_ONLY) {
    p1 = tile;
  } else {
    p1 = a.pos1[tile];
    if (block) {
      p2 = a.pos2[tile];
      p3 = a.pos3[tile];
    }
  }
  // block mode: a list whose column list was empty holds no partials
  const bool has1 = p1 >= 0 && (!block || a.ncols1 > 0);
  const bool has2 = p2 >= 0 && a.ncols2 > 0;
  const bool has3 = p3 >= 0 && a.ncols3 > 0;
  int64_t b10 = 0, b11 = 0, b20 = 0, b21 = 0, b30 = 0, b31 = 0;
  if (has1 && a.skG1 > 0) {
    const int64_t W = (int64_t)a.n1 * a.ncols1;
    b10 = sk_cta((int64_t)p1 * a.ncols1, W, a.skG1);
    b11 = sk_cta((int64_t)p1 * a.ncols1 + a.ncols1 - 1, W, a.skG1);
  }
  if (has2 && a.skG2 > 0) {
    const int64_t W = (int64_t)a.n2 * a.ncols2;
    b20 = sk_cta((int64_t)p2 * a.ncols2, W, a.skG2);
    b21 = sk_cta((int64_t)p2 * a.ncols2 + a.ncols2 - 1, W, a.skG2);
  }
  if (has3 && a.skG3 > 0) {
    const int64_t W = (int64_t)a.n3 * a.ncols3;
    b30 = sk_cta((int64_t)p3 * a.ncols3, W, a.skG3);
    b31 = sk_cta((int64_t)p3 * a.ncols3 + a.ncols3 - 1, W, a.skG3);
  }

  // phase 1: issue every global load of this thread's elements
  float pv[EPT], qv[EPT], av[EPT], mv[EPT], uv[EPT];
  const bool rms = (a.method == SYMNMF_RMSPROP);
  const bool admm = (a.method == SYMNMF_ADMM);
#pragma unroll
  for (int i = 0; i < EPT; ++i) {
    const int e = tid + i * kEpiThreads;
    const int r = e / KP, c = e % KP;
    const bool valid = (r < rows) && (c < a.k);
    const int64_t gi = (r0 + r) * KP + c;
    pv[i] = (valid && has1)
                ? part_sum<KP>(a.P, a.nsplit, a.skG1, a.ncols1, a.n1, p1, r, c, b10, b11)
                : 0.f;
    qv[i] = (valid && has2)
                ? part_sum<KP>(a.Q, a.nsplit2, a.skG2, a.ncols2, a.n2, p2, r, c, b20, b21)
                : 0.f;
    if (valid && has3) {
      const float rv = part_sum<KP>(a.R, a.nsplit3, a.skG3, a.ncols3, a.n3, p3, r, c, b30, b31);
      pv[i] = (p1 >= 0) ? rv + pv[i] : 0.f;
      qv[i] = (p2 >= 0) ? rv + qv[i] : 0.f;
    }
    uv[i] = (valid && p1 < 0 && p2 < 0) ? a.mu[gi] : 0.f;
    av[i] = (valid && a.update) ? a.A[gi] : 0.f;
    mv[i] = (valid && a.update && rms) ? a.M[gi] : 0.f;
  }
  __syncthreads();

  // phase 2: gradient, update, projection
  float tr = 0.f, kkt2 = 0.f, sumA = 0.f;
  int nonfin = 0;
#pragma unroll
  for (int i = 0; i < EPT; ++i) {
    const int e = tid + i * kEpiThreads;
    const int r = e / KP, c = e % KP;
    float hn = 0.f;
    if (r < rows && c < a.k) {
      const int64_t gi = (r0 + r) * KP + c;
      const float h = Hs[r][c];
      float g;
      if (p1 >= 0 || p2 >= 0) {
        g = 0.f;
        if (p1 >= 0) {
          float hg = 0.f;
#pragma unroll
          for (int d = 0; d < KP; ++d) hg = fmaf(Hs[r][d], G1[d][c], hg);
          g = a.coef * (hg - pv[i]);
          tr = fmaf(h, pv[i], tr);
        }
        if (p2 >= 0) {
          float hg = 0.f;
#pragma unroll
          for (int d = 0; d < KP; ++d) hg = fmaf(Hs[r][d], G2[d][c], hg);
          g += a.coef * (hg - qv[i]);
        }
      } else {
        g = uv[i];
      }
      const float pg = (h > 0.f) ? g : fminf(0.f, g);
      kkt2 = fmaf(pg, pg, kkt2);
      if (!isfinite(g)) ++nonfin;
      if (a.gout) a.gout[gi] = g;
      if (a.gcaller) a.gcaller[(r0 + r) * a.k + c] = g;
      if (a.store_mu) a.mu[gi] = g;
      if (a.update && admm) {
        // ADMM right-hand-side row 2 (S W) + rho (W - U), finished below
        hn = 2.f * pv[i] + a.rho * (h - av[i]);
      } else if (a.update) {
        float x;
        if (rms) {
          const float v = a.alpha * av[i] + (1.f - a.alpha) * (g * g);
          a.A[gi] = v;
          const float m = a.mom * mv[i] + adaptive_step(a.eta * g, v, a.eps);
          a.M[gi] = m;
          x = h - m;
          sumA += v;
        } else {
          const float acc = av[i] + g * g;
          a.A[gi] = acc;
          x = h - adaptive_step(a.eta * g, acc, a.eps);
          sumA += acc;
        }
        hn = (x > 0.f) ? x : 0.f;
        a.Hn[gi] = hn;
      } else {
        hn = h;
      }
    }
    Hn[r][c] = hn;
  }
  __syncthreads();
  if (a.update && admm) {
    // H = rhs (2 W^T W + rho I)^-1, W' = [H + U]_+, U' = U + H - W'
    // (appendix, Family 6)
    float xv[EPT];
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * kEpiThreads;
      const int r = e / KP, c = e % KP;
      float x = 0.f;
      if (r < rows && c < a.k) {
#pragma unroll 8
        for (int d = 0; d < KP; ++d) x = fmaf(Hn[r][d], a.minv[d * KP + c], x);
        x += av[i];
      }
      xv[i] = x;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * kEpiThreads;
      const int r = e / KP, c = e % KP;
      float w = 0.f;
      if (r < rows && c < a.k) {
        const int64_t gi = (r0 + r) * KP + c;
        w = (xv[i] > 0.f) ? xv[i] : 0.f;
        const float u = xv[i] - w;
        a.A[gi] = u;
        a.Hn[gi] = w;
        sumA += u;
      }
      Hn[r][c] = w;
    }
    __syncthreads();
  }
  if (a.update) tile_tail<KP>(Hn, r0, a.Btn, a.bt_fmt, a.ldb, a.gram_part, tile);
  const double s_tr = block_sum((double)tr, red);
  const double s_kkt = block_sum((double)kkt2, red);
  const double s_a = block_sum((double)sumA, red);
  const double s_nf = block_sum((double)nonfin, red);
  if (tid == 0 && a.slots) {
    double *sl = a.slots + (int64_t)tile * kSlotStride;
    sl[0] = s_tr;
    sl[1] = s_kkt;
    sl[2] = s_a;
    sl[3] = s_nf;
  }


}

template <int KP>
__global__ void __launch_bounds__(256) prepare_kernel(const float *H, int64_t n, void *Bt,
                                                      int bt_fmt, int64_t ldb, float *gram_part) {
  __shared__ float Hn[kTileRows][KP + 1];
  const int tile = blockIdx.x;
  const int64_t r0 = (int64_t)tile * kTileRows;
  const int rows = (int)((n - r0) < kTileRows ? (n - r0) : kTileRows);
  for (int e = threadIdx.x; e < kTileRows * KP; e += blockDim.x) {
    const int r = e / KP, c = e % KP;
    Hn[r][c] = (r < rows) ? H[(r0 + r) * KP + c] : 0.f;
  }
  __syncthreads();
  tile_tail<KP>(Hn, r0, Bt, bt_fmt, ldb, gram_part, tile);
}

// Fixed-order FP64 reduction of an iteration's per-tile results (the 4
// scalar slots and the kp x kp Gram partial of every tile).  Grid (entry
// blocks of 128 values, chunks of 32 tiles): level 1 sums a chunk's tiles in
// tile order; the last CTA of an entry block to arrive sums the chunks in
// chunk order, so the result does not depend on timing.  Entry block 0 also
// forms the iteration record f = ||S||^2 - 2 tr + ||Gram_t||^2 (Eq. 2).
template <int KP>
__global__ void __launch_bounds__(128) reduce_iter_kernel(ReduceArgs a) {
  // let the next step kernel start streaming now: only its epilogue warps
  // read what this kernel writes, and they wait for it (griddepcontrol.wait)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ double red[40];
  __shared__ double sc[4];
  __shared__ int last;
  const int stride = 4 + KP * KP;
  const int eb = blockIdx.x, tc = blockIdx.y, nTC = gridDim.y;
  const int e = eb * 128 + threadIdx.x;
  const int t0 = tc * 32;
  const int cnt = (a.ntiles - t0) < 32 ? (a.ntiles - t0) : 32;
  const bool gram = (a.gram_part != nullptr);
  if (e < stride) {
    double v = 0.0;
    if (e < 4) {
      if (a.slots) v = ordered_sum32(a.slots + (int64_t)t0 * kSlotStride + e, kSlotStride, cnt);
    } else if (gram) {
      v = ordered_sum32(a.gram_part + (int64_t)t0 * KP * KP + (e - 4), KP * KP, cnt);
    }
    a.lvl1[(int64_t)tc * stride + e] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int old = atomicAdd(&a.counters[eb], 1);
    last = (old == nTC - 1);
    if (last) a.counters[eb] = 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  if (e < stride) {
    for (int g0 = 0; g0 < nTC; g0 += 32) {
      const int c2 = (nTC - g0) < 32 ? (nTC - g0) : 32;
      s += ordered_sum32(a.lvl1 + (int64_t)g0 * stride + e, stride, c2);
    }
    if (e >= 4 && gram) {
      // restarts concatenated along N: only the diagonal kb x kb blocks
      if (a.kb > 0 && (e - 4) / KP / a.kb != (e - 4) % KP / a.kb) s = 0.0;
      a.gram64_next[e - 4] = s;
      a.gram32_next[e - 4] = (float)s;
    }
  }
  if (eb != 0) return;
  if (threadIdx.x < 4) sc[threadIdx.x] = s;
  double g2 = 0.0;
  if (a.gram64_cur)
    for (int i = threadIdx.x; i < KP * KP; i += blockDim.x) g2 += a.gram64_cur[i] * a.gram64_cur[i];
  g2 = block_sum(g2, red);
  if (threadIdx.x == 0 && a.rec && a.slots) {
    DevRecord rc;
    rc.t = a.t;
    rc.tr = sc[0];
    rc.gram2 = g2;
    rc.f = a.normS2 - 2.0 * sc[0] + g2;
    rc.E = rc.f / a.normS2;
    rc.kkt = sqrt(sc[1]) / ((double)a.n * (double)a.k);
    rc.sumA = sc[2];
    rc.nonfinite = (int)sc[3];
    rc.full = a.full;
    *a.rec = rc;
  }
}

template <int KP>
__global__ void __launch_bounds__(256) gram_subset_kernel(const float *gram_part, const int *l1,
                                                          int n1, const int *l2, int n2,
                                                          float *o1, float *o2, int kb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= KP * KP) return;
  const int *l = blockIdx.y == 0 ? l1 : l2;
  const int m = blockIdx.y == 0 ? n1 : n2;
  float *o = blockIdx.y == 0 ? o1 : o2;
  double s = 0.0;
  for (int i = 0; i < m; ++i) s += (double)gram_part[(int64_t)l[i] * KP * KP + e];
  if (kb > 0 && e / KP / kb != e % KP / kb) s = 0.0;
  o[e] = (float)s;
}

template <int DT>
__device__ __forceinline__ double s_value(const void *S, int64_t idx, double scale) {
  if constexpr (DT == 0) {
    return (double)reinterpret_cast<const float *>(S)[idx];
  } else if constexpr (DT == 1) {
    return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(S)[idx]);
  } else {
    __nv_fp8_e4m3 q;
    q.__x = reinterpret_cast<const __nv_fp8_storage_t *>(S)[idx];
    return (double)static_cast<float>(q) * scale;
  }
}

template <int DT>
__global__ void __launch_bounds__(256) norm_s2_kernel(const void *S, int64_t n, int64_t lds,
                                                      const float *scales, int64_t ld_scales,
                                                      double *partials) {
  __shared__ double red[40];
  double acc = 0.0;
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      const double sc = (DT == 2) ? (double)scales[(r / kTileRows) * ld_scales + c / kTileRows] : 1.0;
      const double v = s_value<DT>(S, r * lds + c, sc);
      acc += v * v;
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void sum_array_kernel(const double *x, int m, int stride, int off, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += x[(int64_t)i * stride + off];
    *out = s;
  }
}

// caller row-major n x k -> n x kp over all tile rows (pads zeroed)
__global__ void pack_kernel(const float *src, float *dst, int64_t n, int k, int kp) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tiles = (n + kTileRows - 1) / kTileRows;
  if (e >= tiles * kTileRows * kp) return;
  const int64_t r = e / kp;
  const int c = (int)(e % kp);
  dst[e] = (c < k && r < n) ? src[r * k + c] : 0.f;
}

__global__ void unpack_kernel(const float *src, float *dst, int64_t n, int k, int kp) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t r = e / k;
  const int c = (int)(e % k);
  dst[e] = src[r * kp + c];
}

// radix select of the lower median of g^2 over columns c0 .. c0 + kw - 1
// (FP32 bit patterns of non-negative floats order like unsigned integers);
// three passes of 11, 11, 10 bits
__global__ void __launch_bounds__(256) hist_kernel(const float *g, int64_t n, int c0, int kw,
                                                   int kp, int shift, int nbits,
                                                   const unsigned *sel, unsigned *hist) {
  __shared__ unsigned sh[2048];
  const int nb = 1 << nbits;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const unsigned mask = sel[0], val = sel[1];
  const int64_t total = n * kw;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / kw;
    const int c = c0 + (int)(e % kw);
    const float x = g[r * kp + c];
    const float x2 = x * x;
    const unsigned u = __float_as_uint(x2);
    if ((u & mask) == val) atomicAdd(&sh[(u >> shift) & (nb - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__global__ void select_kernel(unsigned *hist, int shift, int nbits, unsigned *sel, float *out,
                              int last) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nb = 1 << nbits;
  unsigned rank = sel[2];
  unsigned cum = 0;
  int b = 0;
  for (; b < nb; ++b) {
    if (cum + hist[b] > rank) break;
    cum += hist[b];
  }
  if (b >= nb) b = nb - 1;
  sel[2] = rank - cum;
  sel[0] |= (unsigned)(nb - 1) << shift;
  sel[1] |= (unsigned)b << shift;
  for (int i = 0; i < nb; ++i) hist[i] = 0u;
  if (last) *out = __uint_as_float(sel[1]);
}

__global__ void init_sel_kernel(unsigned *sel, unsigned rank, unsigned *hist) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sel[0] = 0u;
    sel[1] = 0u;
    sel[2] = rank;
  }
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) hist[i] = 0u;
}

// A = c max(g^2, median) on columns c0 .. c0 + kw - 1; slot 2 of each tile
// gets the tile's sum of the reset entries
template <int KP>
__global__ void __launch_bounds__(256) reset_kernel(float *A, const float *g, const float *med,
                                                    float c, int64_t n, int c0, int kw,
                                                    double *slots) {
  __shared__ double red[40];
  const int tile = blockIdx.x;
  const int64_t r0 = (int64_t)tile * kTileRows;
  const int rows = (int)((n - r0) < kTileRows ? (n - r0) : kTileRows);
  const float m = *med;
  float s = 0.f;
  for (int e = threadIdx.x; e < kTileRows * KP; e += blockDim.x) {
    const int r = e / KP, cc = e % KP;
    if (r < rows && cc >= c0 && cc < c0 + kw) {
      const int64_t gi = (r0 + r) * KP + cc;
      const float x = g[gi];
      const float v = c * fmaxf(x * x, m);
      A[gi] = v;
      s += v;
    }
  }
  const double tot = block_sum((double)s, red);
  if (threadIdx.x == 0) slots[(int64_t)tile * kSlotStride + 2] = tot;
}

// ADMM (appendix, Family 6): the H-update solves H (2 W^T W + rho I) =
// 2 S W + rho (W - U) row by row; every row shares the kp x kp matrix, so
// its inverse is formed once per iteration here and the step's epilogue
// multiplies each right-hand-side row by it.  M = 2 G + rho I is formed in
// FP64 from the FP64 Gram of W = H_t, rounded to FP32 and inverted by
// Gauss-Jordan elimination in place without pivoting (M is symmetric
// positive definite, rho > 0): pivot p maps a_pp -> 1/a_pp,
// a_pj -> a_pj/a_pp, a_ip -> -a_ip/a_pp and a_ij -> a_ij - a_ip a_pj/a_pp.
// Two shared buffers alternate so one barrier per pivot suffices.  Entries
// past k hold the identity, so the padded block of the inverse is the
// identity and the padded columns of H stay zero.
template <int KP>
__global__ void __launch_bounds__(256) admm_minv_kernel(const double *gram64, int k, double rho,
                                                        float *minv) {
  // the next step kernel may start streaming S now; its epilogue warps wait
  // for this grid (griddepcontrol.wait) before they read minv
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // gram64 is written by the preceding reduction kernel
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ float X[2][KP][KP + 1];
  for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) {
    const int i = e / KP, j = e % KP;
    float v = (i == j) ? 1.f : 0.f;
    if (i < k && j < k) v = (float)(2.0 * gram64[e] + (i == j ? rho : 0.0));
    X[0][i][j] = v;
  }
  __syncthreads();
  for (int p = 0; p < KP; ++p) {
    const float(*src)[KP + 1] = X[p & 1];
    float(*dst)[KP + 1] = X[(p + 1) & 1];
    const float d = 1.f / src[p][p];
    for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) {
      const int i = e / KP, j = e % KP;
      float v;
      if (i == p) {
        v = (j == p) ? d : src[p][j] * d;
      } else {
        const float f = src[i][p] * d;
        v = (j == p) ? -f : fmaf(-f, src[p][j], src[i][j]);
      }
      dst[i][j] = v;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) minv[e] = X[KP & 1][e / KP][e % KP];
}

}  // namespace

#define KP_SWITCH(kp, ...)                              \
  switch (kp) {                                         \
    case 8: { constexpr int KPV = 8; __VA_ARGS__; } break;   \
    case 16: { constexpr int KPV = 16; __VA_ARGS__; } break; \
    case 32: { constexpr int KPV = 32; __VA_ARGS__; } break; \
    case 64: { constexpr int KPV = 64; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;              \
  }

cudaError_t launch_epilogue(const EpiArgs &a, cudaStream_t s) {
  KP_SWITCH(a.kp, {
    constexpr size_t bytes = epi_smem_bytes<KPV>();
    cudaError_t e = cudaFuncSetAttribute(epilogue_kernel<KPV>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    epilogue_kernel<KPV><<<a.ntiles, kEpiThreads, bytes, s>>>(a);
  });
  return cudaGetLastError();
}

cudaError_t launch_admm_minv(const double *gram64, int k, int kp, double rho, float *minv,
                             cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  KP_SWITCH(kp, return cudaLaunchKernelEx(&cfg, admm_minv_kernel<KPV>, gram64, k, rho, minv));
  return cudaErrorInvalidValue;
}

cudaError_t launch_prepare_tiles(const float *H, int64_t n, int k, int kp, void *Bt, int bt_fmt,
                                 int64_t ldb, float *gram_part, cudaStream_t s) {
  (void)k;
  const int ntiles = (int)((n + kTileRows - 1) / kTileRows);
  KP_SWITCH(kp, prepare_kernel<KPV><<<ntiles, 256, 0, s>>>(H, n, Bt, bt_fmt, ldb, gram_part));
  return cudaGetLastError();
}

cudaError_t launch_reduce_iter(const ReduceArgs &a, int kp, cudaStream_t s) {
  const int stride = 4 + (a.gram_part ? kp * kp : 0);
  dim3 grid((stride + 127) / 128, (a.ntiles + 31) / 32);
  KP_SWITCH(kp, reduce_iter_kernel<KPV><<<grid, 128, 0, s>>>(a));
  return cudaGetLastError();
}

cudaError_t launch_gram_subset(const float *gram_part, int kp, const int *l1, int n1,
                               const int *l2, int n2, float *o1, float *o2, int kb, cudaStream_t s) {
  dim3 grid((kp * kp + 255) / 256, 2);
  KP_SWITCH(kp, gram_subset_kernel<KPV><<<grid, 256, 0, s>>>(gram_part, l1, n1, l2, n2, o1, o2, kb));
  return cudaGetLastError();
}

cudaError_t launch_norm_s2(const void *S, int64_t n, int64_t lds, int dtype, const float *scales,
                           int64_t ld_scales, double *partials, int nparts, double *out,
                           cudaStream_t s) {
  switch (dtype) {
    case 0: norm_s2_kernel<0><<<nparts, 256, 0, s>>>(S, n, lds, scales, ld_scales, partials); break;
    case 1: norm_s2_kernel<1><<<nparts, 256, 0, s>>>(S, n, lds, scales, ld_scales, partials); break;
    case 2: norm_s2_kernel<2><<<nparts, 256, 0, s>>>(S, n, lds, scales, ld_scales, partials); break;
    default: return cudaErrorInvalidValue;
  }
  sum_array_kernel<<<1, 32, 0, s>>>(partials, nparts, 1, 0, out);
  return cudaGetLastError();
}

cudaError_t launch_pack(const float *src, float *dst, int64_t n, int k, int kp, cudaStream_t s) {
  const int64_t tot = (n + kTileRows - 1) / kTileRows * kTileRows * kp;
  pack_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, dst, n, k, kp);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const float *src, float *dst, int64_t n, int k, int kp, cudaStream_t s) {
  const int64_t tot = n * k;
  unpack_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, dst, n, k, kp);
  return cudaGetLastError();
}

cudaError_t launch_median_g2(const float *g, int64_t n, int c0, int kw, int kp, unsigned *hist,
                             unsigned *sel, float *out, cudaStream_t s) {
  const int64_t total = n * kw;
  const unsigned rank = (unsigned)((total - 1) / 2);
  init_sel_kernel<<<1, 256, 0, s>>>(sel, rank, hist);
  const int grid = (int)std::min<int64_t>(1024, (total + 255) / 256);
  const int shifts[3] = {21, 10, 0};
  const int bits[3] = {11, 11, 10};
  for (int p = 0; p < 3; ++p) {
    hist_kernel<<<grid, 256, 0, s>>>(g, n, c0, kw, kp, shifts[p], bits[p], sel, hist);
    select_kernel<<<1, 1, 0, s>>>(hist, shifts[p], bits[p], sel, out, p == 2);
  }
  return cudaGetLastError();
}

cudaError_t launch_reset(float *A, const float *g, const float *med, float c, int64_t n, int c0,
                         int kw, int kp, double *slots, cudaStream_t s) {
  const int ntiles = (int)((n + kTileRows - 1) / kTileRows);
  KP_SWITCH(kp, reset_kernel<KPV><<<ntiles, 256, 0, s>>>(A, g, med, c, n, c0, kw, slots));
  return cudaGetLastError();
}

cudaError_t launch_sum_slot(const double *slots, int ntiles, int which, double *out,
                            cudaStream_t s) {
  sum_array_kernel<<<1, 32, 0, s>>>(slots, ntiles, kSlotStride, which, out);
  return cudaGetLastError();
}

}  // namespace symnmf
