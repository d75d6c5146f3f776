// Dependence matrix on the GPU (Sec. 3: the absolute correlation matrix and
// the empirical TPDM), the step before the solver.  Both are unit-diagonal
// normalisations of a Gram matrix of the n variables over T observations:
//   S_ij = |G_ij| / sqrt(G_ii G_jj),   G = Y^T Y,
// with Y the observations with centred columns (correlation) or the
// exceedance angles Omega (TPDM; the n / n_exc factor cancels).
//
// Kernels:
//   dep_stats   column means (centring) and d_i = sum_t c_ti^2 of the
//               FP32 centred values c_ti, FP64
//   dep_split   transposes Y into P = [hi | lo] (n x 2 Tp, FP32 holding
//               tf32 values): hi = c with the 13 low mantissa bits cleared,
//               lo = (c - hi) rounded to tf32; Tp = T rounded up to 32
//   dep_gemm    persistent, one CTA per SM over the list of 128 x 256
//               tiles of G, on tcgen05 (kind::tf32, M = 128, N = 256, two
//               accumulators in tensor memory taken in turn, so a tile's
//               epilogue overlaps the next tile's MMAs): each stage holds a
//               16-column chunk of A_hi, A_lo, B_hi and B_lo (64-byte
//               swizzle, fetched from P by TMA) and feeds the three products
//               hi hi, lo hi and hi lo (the dropped lo lo term is below
//               2^-21 relative), so every staged byte serves two products;
//               the epilogue
//               normalises, clamps to [0, 1], writes 1 on the diagonal and
//               stores S as FP32, BF16 (round to nearest) or E4M3 with one
//               power-of-two scale per 128 x 128 tile, plus the CTA's FP64
//               sum of squares (FP8: of the values before quantisation).
//               Only 128 x 128 tiles on or above the diagonal are computed;
//               each one above it is also stored transposed, so S is
//               exactly symmetric and the tensor work is halved
//   dep_sum     fixed-order FP64 sum of the CTA partials -> ||S||^2
// Every mbarrier wait is bounded (2 s); on expiry the CTA records an error
// code, drains its own copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "../../include/symnmf.h"
#include "epi_common.cuh"
#include "symnmf_internal.h"
#include "tc_ptx.cuh"

#include <algorithm>
#include <vector>

namespace symnmf {
namespace {

using namespace tc;

constexpr int kDepStages = 4;
constexpr int kDepKC = 16;                             // tf32 per staged row (64 bytes)
constexpr uint32_t kDepA = 128 * 64;                   // 128 rows x 16 tf32
constexpr uint32_t kDepB = 256 * 64;                   // 256 rows x 16 tf32
constexpr uint32_t kDepStage = 2 * kDepA + 2 * kDepB;  // A_hi, A_lo, B_hi, B_lo: 48 KB
constexpr size_t kDepSmem = 1024 + (size_t)kDepStages * kDepStage + 256 + 256 * 4 + 64 * 8;
constexpr int kDepThreads = 192;  // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue

__global__ void __launch_bounds__(256) dep_stats_kernel(const float *Y, int64_t T, int64_t n,
                                                        int64_t ldy, int center, float *mean32,
                                                        double *inv_d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double m = 0.0;
  if (center) {
    for (int64_t t = 0; t < T; ++t) m += (double)Y[t * ldy + i];
    m /= (double)T;
  }
  const float mf = (float)m;
  double d = 0.0;
  for (int64_t t = 0; t < T; ++t) {
    const float c = Y[t * ldy + i] - mf;
    d += (double)c * (double)c;
  }
  mean32[i] = mf;
  inv_d[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
}

// 32 x 32 tiles through shared memory; block (32, 8)
__global__ void dep_split_kernel(const float *Y, int64_t T, int64_t n, int64_t ldy,
                                 const float *mean32, int Tp, float *P) {
  __shared__ float tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t t = t0 + r, i = i0 + tx;
    float c = 0.f;
    if (t < T && i < n) c = Y[t * ldy + i] - mean32[i];
    tile[r][tx] = c;
  }
  __syncthreads();
  const int64_t pitch = 2 * (int64_t)Tp;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, t = t0 + tx;
    if (i < n) {
      const float c = tile[tx][r];
      const float hi = tf32_trunc(c);
      P[i * pitch + t] = hi;
      P[i * pitch + Tp + t] = tf32_round(c - hi);
    }
  }
}

struct DepArgs {
  int64_t n;
  int Tp;
  int natoms;       // Tp / 16 staged chunks per tile
  int ntiles;       // entries of the tile list
  const int *tiles; // (ib << 16 | jb) per 128 x 256 tile on or above the diagonal
  const double *inv_d;
  void *S;
  int64_t lds;
  int out;          // 0 FP32, 1 BF16, 2 E4M3
  float *scales;
  int64_t ld_scales;
  double *sq;       // per CTA
  int *err;
  int exact_sq;     // F32 / BF16: run sums of squares as float-float pairs
};

__device__ __forceinline__ void dep_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Persistent: CTA b takes tiles b, b + G, b + 2G, ... of the list.  Two
// accumulators of 256 TMEM columns alternate between tiles, so the
// epilogue of one tile overlaps the MMAs of the next.
__global__ void __launch_bounds__(kDepThreads, 1)
    dep_gemm_kernel(const __grid_constant__ CUtensorMap mP, const DepArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kDepStages * kDepStage);
  uint64_t *empty = full + kDepStages;
  uint64_t *accf = empty + kDepStages;  // 2: accumulator ready for the epilogue
  uint64_t *acce = accf + 2;            // 2: accumulator free for the MMAs
  uint32_t *holder = reinterpret_cast<uint32_t *>(acce + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(holder + 1);
  int *consumed = const_cast<int *>(abort_flag) + 1;
  float *invj = reinterpret_cast<float *>(smem + kDepStages * kDepStage + 256);
  double *red = reinterpret_cast<double *>(invj + 256);  // 64 doubles

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x;
  const int my_tiles = (a.ntiles - (int)blockIdx.x + G - 1) / G;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDepStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);
    }
    *abort_flag = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(holder, 512);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *holder;
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mP)) : "memory");
      int c = 0;  // atoms issued over all tiles
      bool stop = false;
      for (int lt = 0; lt < my_tiles && !stop; ++lt) {
        const int tl = a.tiles[blockIdx.x + lt * G];
        const int ib = tl >> 16, jb = tl & 0xFFFF;
        for (int at = 0; at < a.natoms; ++at, ++c) {
          const int s = c % kDepStages;
          if (c >= kDepStages &&
              !mbar_wait(&empty[s], (uint32_t)((c / kDepStages - 1) & 1), abort_flag)) {
            set_err(a.err, 31);
            *abort_flag = 1;
            stop = true;
            break;
          }
          const int o = at * kDepKC;
          uint8_t *st = smem + (size_t)s * kDepStage;
          uint8_t *sb = st + 2 * kDepA;
          mbar_expect_tx(&full[s], kDepStage);
          tma_load_2d(st, &mP, &full[s], o, ib * 128);                    // A_hi
          tma_load_2d(st + kDepA, &mP, &full[s], a.Tp + o, ib * 128);     // A_lo
          tma_load_2d(sb, &mP, &full[s], o, jb * 256);                    // B_hi
          tma_load_2d(sb + kDepB / 2, &mP, &full[s], o, jb * 256 + 128);
          tma_load_2d(sb + kDepB, &mP, &full[s], a.Tp + o, jb * 256);     // B_lo
          tma_load_2d(sb + kDepB + kDepB / 2, &mP, &full[s], a.Tp + o, jb * 256 + 128);
          ++issued;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(128, 256);
      int c = 0, done = 0;
      bool stop = false;
      for (int lt = 0; lt < my_tiles && !stop; ++lt) {
        const int b = lt & 1;
        if (lt >= 2 && !mbar_wait(&acce[b], (uint32_t)((lt / 2 - 1) & 1), abort_flag)) {
          set_err(a.err, 34);
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t tacc = tbase + (uint32_t)(b * 256);
        for (int at = 0; at < a.natoms; ++at, ++c) {
          const int s = c % kDepStages;
          if (!mbar_wait(&full[s], (uint32_t)((c / kDepStages) & 1), abort_flag)) {
            set_err(a.err, 32);
            *abort_flag = 1;
            stop = true;
            break;
          }
          fence_after();
          const uint32_t ah = smem_u32(smem + (size_t)s * kDepStage), al = ah + kDepA;
          const uint32_t bh = ah + 2 * kDepA, bl = bh + kDepB;
#pragma unroll
          for (int ks = 0; ks < kDepKC / 8; ++ks) {  // K = 8 tf32 (32 bytes) per MMA
            const uint32_t o = (uint32_t)ks * 32u;
            mma_tf32_ss(tacc, sdesc64(ah + o), sdesc64(bh + o), idesc, (at > 0 || ks > 0) ? 1u : 0u);
            mma_tf32_ss(tacc, sdesc64(al + o), sdesc64(bh + o), idesc, 1u);
            mma_tf32_ss(tacc, sdesc64(ah + o), sdesc64(bl + o), idesc, 1u);
          }
          mma_commit(&empty[s]);
          done = c + 1;
        }
        mma_commit(&accf[b]);
      }
      *consumed = done;
    }
  } else {
    // epilogue: thread row r of each tile, 256 columns = the 128-column
    // tiles jt = 2 jb and 2 jb + 1.  Only the upper triangle is computed:
    // a tile with jt > ib is stored and mirrored to (jt, ib) (lane = row,
    // so the mirrored stores of a warp are 32 consecutive entries of one
    // row); in a tile with jt == ib the entries j >= i are stored and those
    // with j > i mirrored; jt < ib is left to its mirror.  Every stored
    // pair S_ij, S_ji is one accumulator value, so S is exactly symmetric.
    const int q = warp & 3, r = q * 32 + lane, et = threadIdx.x - 64;
    double sq = 0.0;
    for (int lt = 0; lt < my_tiles; ++lt) {
      const int b = lt & 1;
      const int tl = a.tiles[blockIdx.x + lt * G];
      const int ib = tl >> 16, jb = tl & 0xFFFF;
      const int64_t i = (int64_t)ib * 128 + r;
      const bool vrow = i < a.n;
      const float inv_i = vrow ? (float)a.inv_d[i] : 0.f;
      const uint32_t trow = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256);
      const int64_t j0 = (int64_t)jb * 256;
      int mode[2];  // 0 skip, 1 store (diagonal tile), 2 store and mirror
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jt = 2 * jb + h;
        mode[h] = ((int64_t)jt * 128 >= a.n || jt < ib) ? 0 : (jt == ib ? 1 : 2);
      }
      dep_bar();  // every thread is done with the previous tile's invj
      for (int c = et; c < 256; c += 128) {
        const int64_t j = j0 + c;
        invj[c] = j < a.n ? (float)a.inv_d[j] : 0.f;
      }
      dep_bar();
      const bool ok = warp_wait_idle(&accf[b], (uint32_t)((lt / 2) & 1), abort_flag);
      if (!ok) {
        if (lane == 0) {
          set_err(a.err, 33);
          *abort_flag = 1;
        }
        break;
      }
      fence_after();
      auto sval = [&](uint32_t bits, int c) -> float {
        const int64_t j = j0 + c;
        if (!vrow || j >= a.n) return 0.f;
        if (j == i) return 1.f;
        return fminf(1.f, fabsf(__uint_as_float(bits)) * inv_i * invj[c]);
      };
      // how many stored entries the value of column c stands for (0, 1, 2)
      auto wgt = [&](int md, int c) -> float {
        const int64_t j = j0 + c;
        if (md == 2) return 2.f;
        return j > i ? 2.f : (j == i ? 1.f : 0.f);
      };
      // the accumulator goes back to the MMAs once the last read is done
      auto release = [&]() {
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[b]);
      };
      if (a.out == 2) {
        float amax[2] = {0.f, 0.f};
        for (int c0 = 0; c0 < 256; c0 += 32) {
          const int md = mode[c0 >> 7];
          if (!md) continue;
          uint32_t x[32];
#pragma unroll
          for (int u = 0; u < 4; ++u) tmem_ld8_nw(trow + c0 + 8 * u, x, 8 * u);
          tmem_wait_ld_all(x);
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (wgt(md, c0 + u) > 0.f) amax[c0 >> 7] = fmaxf(amax[c0 >> 7], sval(x[u], c0 + u));
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
            amax[h] = fmaxf(amax[h], __shfl_xor_sync(0xffffffffu, amax[h], o));
        float *fr = reinterpret_cast<float *>(red);
        if (lane == 0) {
          fr[q * 2 + 0] = amax[0];
          fr[q * 2 + 1] = amax[1];
        }
        dep_bar();
        float dsc[2], inv_dsc[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float m = fmaxf(fmaxf(fr[h], fr[2 + h]), fmaxf(fr[4 + h], fr[6 + h]));
          dsc[h] = e4m3_tile_scale(m);
          inv_dsc[h] = 1.f / dsc[h];
        }
        dep_bar();
        if (et < 2 && mode[et]) {
          const int64_t jt = (int64_t)jb * 2 + et;
          a.scales[(int64_t)ib * a.ld_scales + jt] = dsc[et];
          if (mode[et] == 2) a.scales[jt * a.ld_scales + ib] = dsc[et];
        }
        uint8_t *S8 = reinterpret_cast<uint8_t *>(a.S);
        for (int c0 = 0; c0 < 256; c0 += 32) {
          const int md = mode[c0 >> 7];
          if (!md) continue;
          uint32_t x[32];
#pragma unroll
          for (int u = 0; u < 4; ++u) tmem_ld8_nw(trow + c0 + 8 * u, x, 8 * u);
          tmem_wait_ld_all(x);
          const float isc = inv_dsc[c0 >> 7];
          uint32_t w[8];
          float part = 0.f;
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const float v = sval(x[u], c0 + u);
            part = fmaf(wgt(md, c0 + u) * v, v, part);
            const uint32_t code = e4m3_bits(v * isc);
            if ((u & 3) == 0) w[u >> 2] = 0u;
            w[u >> 2] |= code << (8 * (u & 3));
          }
          sq += (double)part;
          if (!vrow) continue;
          uint8_t *Srow = S8 + i * a.lds;
          if (md == 2 && j0 + c0 + 32 <= a.n) {
            uint4 *dst = reinterpret_cast<uint4 *>(Srow + j0 + c0);
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
          } else {
            for (int u = 0; u < 32 && j0 + c0 + u < a.n; ++u)
              if (md == 2 || j0 + c0 + u >= i)
                Srow[j0 + c0 + u] = (uint8_t)(w[u >> 2] >> (8 * (u & 3)));
          }
          for (int u = 0; u < 32 && j0 + c0 + u < a.n; ++u)
            if (md == 2 || j0 + c0 + u > i)
              S8[(j0 + c0 + u) * a.lds + i] = (uint8_t)(w[u >> 2] >> (8 * (u & 3)));
        }
        release();
      } else {
        for (int c0 = 0; c0 < 256; c0 += 32) {
          const int md = mode[c0 >> 7];
          if (!md) continue;
          uint32_t x[32];
#pragma unroll
          for (int u = 0; u < 4; ++u) tmem_ld8_nw(trow + c0 + 8 * u, x, 8 * u);
          tmem_wait_ld_all(x);
          float v[32];
          float ph = 0.f, pl = 0.f;
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            float s = sval(x[u], c0 + u);
            if (a.out == 1) s = __bfloat162float(__float2bfloat16_rn(s));
            v[u] = s;
          }
          if (a.exact_sq) {
            // the stored values' squares summed as a float-float pair
            // (products split exactly by an FMA, Knuth's TwoSum on the high
            // parts): the run's sum is exact to about 2^-44 before it joins
            // the FP64 total, so ||S||^2 from here stands in for a pass over
            // the stored matrix
#pragma unroll
            for (int u = 0; u < 32; ++u) {
              const float ws = wgt(md, c0 + u) * v[u];  // weight 0, 1 or 2: exact
              const float pr = __fmul_rn(ws, v[u]), pe = fmaf(ws, v[u], -pr);
              const float t = __fadd_rn(ph, pr), bv = __fsub_rn(t, ph);
              pl = __fadd_rn(pl, __fadd_rn(__fadd_rn(__fsub_rn(ph, __fsub_rn(t, bv)),
                                                     __fsub_rn(pr, bv)), pe));
              ph = t;
            }
          } else {
#pragma unroll
            for (int u = 0; u < 32; ++u) ph = fmaf(wgt(md, c0 + u) * v[u], v[u], ph);
          }
          sq += (double)ph + (double)pl;
          if (!vrow) continue;
          const bool whole = md == 2 && j0 + c0 + 32 <= a.n;
          if (a.out == 0) {
            float *S32 = reinterpret_cast<float *>(a.S);
            float *Srow = S32 + i * a.lds + j0 + c0;
            if (whole) {
#pragma unroll
              for (int u = 0; u < 8; ++u)
                reinterpret_cast<float4 *>(Srow)[u] =
                    make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            } else {
              for (int u = 0; u < 32 && j0 + c0 + u < a.n; ++u)
                if (md == 2 || j0 + c0 + u >= i) Srow[u] = v[u];
            }
#pragma unroll
            for (int u = 0; u < 32; ++u)
              if (j0 + c0 + u < a.n && (md == 2 || j0 + c0 + u > i))
                S32[(j0 + c0 + u) * a.lds + i] = v[u];
          } else {
            uint16_t *S16 = reinterpret_cast<uint16_t *>(a.S);
            uint16_t *Srow = S16 + i * a.lds + j0 + c0;
            if (whole) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                uint32_t p[4];
#pragma unroll
                for (int z = 0; z < 4; ++z)
                  p[z] = (uint32_t)bf16_bits(v[8 * u + 2 * z]) |
                         ((uint32_t)bf16_bits(v[8 * u + 2 * z + 1]) << 16);
                reinterpret_cast<uint4 *>(Srow)[u] = make_uint4(p[0], p[1], p[2], p[3]);
              }
            } else {
              for (int u = 0; u < 32 && j0 + c0 + u < a.n; ++u)
                if (md == 2 || j0 + c0 + u >= i) Srow[u] = bf16_bits(v[u]);
            }
#pragma unroll
            for (int u = 0; u < 32; ++u)
              if (j0 + c0 + u < a.n && (md == 2 || j0 + c0 + u > i))
                S16[(j0 + c0 + u) * a.lds + i] = bf16_bits(v[u]);
          }
        }
        release();
      }
    }
    // the CTA's sum of squares: xor tree per warp, warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    dep_bar();
    if (lane == 0) red[8 + q] = sq;
    dep_bar();
    if (et == 0) a.sq[blockIdx.x] = red[8] + red[9] + red[10] + red[11];
  }
  fence_before();
  __syncthreads();
  if (warp == 0 && lane == 0 && *abort_flag) {
    // copies issued but never consumed (bounded)
    for (int c = *consumed; c < issued; ++c) {
      int dummy = 0;
      mbar_wait(&full[c % kDepStages], (uint32_t)((c / kDepStages) & 1),
                reinterpret_cast<volatile int *>(&dummy), 100000000ull);
    }
  }
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// fixed-order FP64 sum: contiguous runs per thread, runs in order
__global__ void __launch_bounds__(256) dep_sum_kernel(const double *x, int64_t m, double *out) {
  __shared__ double red[8];
  const int tid = threadIdx.x;
  const int64_t per = (m + 255) / 256;
  double s = 0.0;
  for (int64_t k = tid * per; k < m && k < (tid + 1) * per; ++k) s += x[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *out = t;
  }
}

}  // namespace

cudaError_t launch_dependence(const float *Y, int64_t T, int64_t n, int64_t ldy, int center,
                              int out, void *S, int64_t lds, float *scales, int64_t ld_scales,
                              double *normS2, int *err, cudaStream_t s, bool exact_norm) {
  const int Tp = (int)((T + 31) / 32 * 32);
  const int nib = (int)((n + 127) / 128), njb = (int)((n + 255) / 256);
  if (nib >= 65536 || njb >= 65536) return cudaErrorInvalidValue;
  // the 128 x 256 tiles on or above the diagonal (2 jb + 1 >= ib), in groups
  // of 16 row tiles that sweep the column blocks together, so the operand
  // rows they share stay in L2
  std::vector<int> tiles;
  constexpr int kGroup = 16;
  for (int g0 = 0; g0 < nib; g0 += kGroup)
    for (int jb = 0; jb < njb; ++jb)
      for (int ib = g0; ib < nib && ib < g0 + kGroup; ++ib)
        if (2 * jb + 1 >= ib) tiles.push_back((ib << 16) | jb);
  const int ntiles = (int)tiles.size();
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int G = std::max(1, std::min(sms, ntiles));
  float *P = nullptr, *mean32 = nullptr;
  double *inv_d = nullptr, *sq = nullptr;
  int *dtiles = nullptr;
  e = cudaMallocAsync((void **)&P, sizeof(float) * (size_t)n * 2 * Tp, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&mean32, sizeof(float) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&inv_d, sizeof(double) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&sq, sizeof(double) * (size_t)G, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&dtiles, sizeof(int) * (size_t)ntiles, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dtiles, tiles.data(), sizeof(int) * (size_t)ntiles,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    dep_stats_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Y, T, n, ldy, center, mean32,
                                                                  inv_d);
    dep_split_kernel<<<dim3((unsigned)(Tp / 32), (unsigned)((n + 31) / 32)), dim3(32, 8), 0, s>>>(
        Y, T, n, ldy, mean32, Tp, P);
    CUtensorMap mP;
    if (!make_map_2d(&mP, P, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (uint64_t)2 * Tp, (uint64_t)n,
                     (uint64_t)2 * Tp * 4, kDepKC, 128, 64)) {
      e = cudaErrorInvalidValue;
    } else {
      e = cudaFuncSetAttribute(dep_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kDepSmem);
    }
    if (e == cudaSuccess) {
      DepArgs a{};
      a.n = n;
      a.Tp = Tp;
      a.natoms = Tp / kDepKC;
      a.ntiles = ntiles;
      a.tiles = dtiles;
      a.inv_d = inv_d;
      a.S = S;
      a.lds = lds;
      a.out = out;
      a.scales = scales;
      a.ld_scales = ld_scales;
      a.sq = sq;
      a.err = err;
      a.exact_sq = exact_norm ? 1 : 0;
      dep_gemm_kernel<<<(unsigned)G, kDepThreads, kDepSmem, s>>>(mP, a);
      if (normS2) dep_sum_kernel<<<1, 256, 0, s>>>(sq, G, normS2);
      e = cudaGetLastError();
    }
  }
  // the tile list must outlive the asynchronous copy
  if (dtiles) {
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
  }
  for (void *p : {(void *)P, (void *)mean32, (void *)inv_d, (void *)sq, (void *)dtiles})
    if (p) cudaFreeAsync(p, s);
  return e;
}

}  // namespace symnmf
