// Tensor-core product P = S[rows, cols] * H[cols] for BF16-stored S on
// sm_103a (the S H term of the gradient, Sec. 2.1; the dominant cost of
// every iteration, Sec. 4.3).
//
// Design (one CTA per SM, persistent, warp-specialised):
//   warp 0     TMA producer: streams 128 x 128 tiles of S (two 128-byte
//              swizzle atoms) and the matching 128-column slice of the
//              bf16 hi/lo copy of H^T into a ring of shared-memory stages
//   warp 1     MMA issuer: one thread issues tcgen05.mma kind::f16
//              (M = 128, N = 2 kp: the hi and lo halves of H side by side,
//              K = 16 per instruction) into a double-buffered TMEM
//              accumulator and frees stages with tcgen05.commit
//   warps 2-5  epilogue: tcgen05.ld the 128 x N accumulator, add the hi and
//              lo halves (so H enters with ~16 significant bits), write the
//              FP32 partial of its (row tile, column range) segment
// Work is the row-major list of (row tile, column tile) units, split into
// equal contiguous ranges, one per CTA (stream-K), so every SM streams the
// same number of S bytes whatever n is.  A CTA's range covers whole row
// tiles plus at most one partial tile at each end; partial segment of CTA
// b for row tile p goes to slot b + p (unique, see stream_k_slot), and the
// epilogue kernel adds a tile's slots in CTA order, so the result is
// deterministic.
//
// Every wait on an mbarrier is bounded (2 s of %globaltimer); on expiry the
// CTA records an error code, stops all roles, drains its own copies and
// MMAs with bounded waits, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "symnmf_internal.h"

namespace symnmf {
namespace {

constexpr int kThreads = 192;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kAtomBytes = 128 * 128;   // 128 rows x 128 bytes

struct TcArgs {
  int64_t W;             // units = n_rows_list * n_cols_list
  int G;                 // CTAs
  int n_cols;
  const int *row_list;
  const int *col_list;
  float *out;
  int *err;
  int stages;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false on timeout or when another role has aborted
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint64_t limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(holder)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// 8 columns of hi and 8 of lo for this thread's TMEM lane, then wait
__device__ __forceinline__ void tmem_ld_pair(uint32_t ta, uint32_t tb, uint32_t (&x)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]),
                 "=r"(x[6]), "=r"(x[7])
               : "r"(ta));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]),
                 "=r"(x[14]), "=r"(x[15])
               : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]),
                 "+r"(x[6]), "+r"(x[7]), "+r"(x[8]), "+r"(x[9]), "+r"(x[10]), "+r"(x[11]),
                 "+r"(x[12]), "+r"(x[13]), "+r"(x[14]), "+r"(x[15])
               :
               : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int KP>
struct Cfg {
  static constexpr int N = 2 * KP;
  static constexpr uint32_t A_BYTES = 2 * kAtomBytes;      // 128 rows x 128 bf16
  static constexpr uint32_t B_BYTES = 2 * N * 128;         // N rows x 128 bf16
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t TMEM_COLS = (2 * N <= 32) ? 32 : (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : 256;
  static constexpr int STAGES = (int)std::min<uint32_t>(8u, (200u * 1024u) / STAGE);
  static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024 + 256;
};

__device__ __forceinline__ void set_err(int *err, int code) {
  if (err) atomicCAS(err, 0, code);
}

template <int KP>
__global__ void __launch_bounds__(kThreads, 1)
    prod_tc_bf16_kernel(const __grid_constant__ CUtensorMap mapS,
                        const __grid_constant__ CUtensorMap mapB, TcArgs a) {
  using C = Cfg<KP>;
  constexpr int N = C::N;
  constexpr int STAGES = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * C::STAGE);
  uint64_t *empty = full + STAGES;
  uint64_t *tfull = empty + STAGES;
  uint64_t *tempty = tfull + 2;
  uint64_t *drain = tempty + 2;
  uint32_t *holder = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(holder + 1);
  int *consumed = const_cast<int *>(abort_flag) + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(holder, C::TMEM_COLS);
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *holder;

  const int b = blockIdx.x;
  const int64_t L0 = (int64_t)b * a.W / a.G;
  const int64_t L1 = (int64_t)(b + 1) * a.W / a.G;
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapS)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t L = L0; L < L1; ++L) {
        const int tp = (int)(L / a.n_cols), ci = (int)(L % a.n_cols);
        const int rt = a.row_list ? a.row_list[tp] : tp;
        const int ct = a.col_list ? a.col_list[ci] : ci;
        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) {
          set_err(a.err, 1);
          *abort_flag = 1;
          break;
        }
        uint8_t *sa = smem + stage * C::STAGE;
        uint8_t *sb = sa + C::A_BYTES;
        mbar_expect_tx(&full[stage], C::STAGE);
        tma_load_2d(sa, &mapS, &full[stage], ct * 128, rt * 128);
        tma_load_2d(sa + kAtomBytes, &mapS, &full[stage], ct * 128 + 64, rt * 128);
        tma_load_2d(sb, &mapB, &full[stage], ct * 128, 0);
        tma_load_2d(sb + N * 128, &mapB, &full[stage], ct * 128 + 64, 0);
        ++issued;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t tphase[2] = {0u, 0u};
      constexpr uint32_t idesc = idesc_bf16(128, N);
      int done = 0;
      for (int64_t L = L0; L < L1; ++L) {
        const int ci = (int)(L % a.n_cols);
        const bool seg_start = (L == L0) || (ci == 0);
        const bool seg_end = (L == L1 - 1) || (ci == a.n_cols - 1);
        if (seg_start) {
          if (!mbar_wait(&tempty[acc], tphase[acc] ^ 1, abort_flag)) {
            set_err(a.err, 2);
            *abort_flag = 1;
            break;
          }
          fence_after();
        }
        if (!mbar_wait(&full[stage], phase, abort_flag)) {
          set_err(a.err, 3);
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t sa = smem_u32(smem + stage * C::STAGE);
        const uint32_t sb = sa + C::A_BYTES;
        const uint32_t d = tmem_base + (uint32_t)(acc * N);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t aoff = (uint32_t)(j >> 2) * kAtomBytes + (uint32_t)(j & 3) * 32u;
          const uint32_t boff = (uint32_t)(j >> 2) * (uint32_t)(N * 128) + (uint32_t)(j & 3) * 32u;
          mma_bf16(d, sdesc(sa + aoff), sdesc(sb + boff), idesc, (seg_start && j == 0) ? 0u : 1u);
        }
        mma_commit(&empty[stage]);
        ++done;
        if (seg_end) {
          mma_commit(&tfull[acc]);
          tphase[acc] ^= 1;
          acc ^= 1;
        }
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      *consumed = done;
      // wait until every MMA issued by this thread has completed
      mma_commit(drain);
      if (!mbar_wait(drain, 0, abort_flag, 100000000ull) && !*abort_flag) set_err(a.err, 4);
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int acc = 0;
    uint32_t tphase[2] = {0u, 0u};
    int64_t L = L0;
    while (L < L1) {
      const int tp = (int)(L / a.n_cols);
      const int64_t tile_end = (int64_t)(tp + 1) * a.n_cols;
      const int64_t seg_end = L1 < tile_end ? L1 : tile_end;
      // one lane waits, the warp follows together (tcgen05.ld is .sync.aligned)
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&tfull[acc], tphase[acc], abort_flag) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          set_err(a.err, 5);
          *abort_flag = 1;
        }
        break;
      }
      fence_after();
      float *dst = a.out + ((int64_t)(b + tp) * 128 + row) * KP;
      const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * N);
#pragma unroll
      for (int c0 = 0; c0 < KP; c0 += 8) {
        uint32_t x[16];
        tmem_ld_pair(lane_base + c0, lane_base + KP + c0, x);
        float4 o0, o1;
        o0.x = __uint_as_float(x[0]) + __uint_as_float(x[8]);
        o0.y = __uint_as_float(x[1]) + __uint_as_float(x[9]);
        o0.z = __uint_as_float(x[2]) + __uint_as_float(x[10]);
        o0.w = __uint_as_float(x[3]) + __uint_as_float(x[11]);
        o1.x = __uint_as_float(x[4]) + __uint_as_float(x[12]);
        o1.y = __uint_as_float(x[5]) + __uint_as_float(x[13]);
        o1.z = __uint_as_float(x[6]) + __uint_as_float(x[14]);
        o1.w = __uint_as_float(x[7]) + __uint_as_float(x[15]);
        reinterpret_cast<float4 *>(dst + c0)[0] = o0;
        reinterpret_cast<float4 *>(dst + c0)[1] = o1;
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      tphase[acc] ^= 1;
      acc ^= 1;
      L = seg_end;
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && *abort_flag) {
    // drain TMA copies that were issued but never consumed (bounded)
    int stage = *consumed % STAGES;
    uint32_t phase = (uint32_t)((*consumed / STAGES) & 1);
    for (int i = *consumed; i < issued; ++i) {
      int dummy = 0;
      mbar_wait(&full[stage], phase, reinterpret_cast<volatile int *>(&dummy), 100000000ull);
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1;
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem_base, C::TMEM_COLS);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map_2d(CUtensorMap *m, const void *base, CUtensorMapDataType dt, uint64_t inner,
                 uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KP>
cudaError_t launch_kp(const ProdArgs &p, cudaStream_t s, int G, TcArgs ta) {
  using C = Cfg<KP>;
  CUtensorMap mS, mB;
  if (!make_map_2d(&mS, p.S, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (uint64_t)p.n, (uint64_t)p.n,
                   (uint64_t)p.lds * 2, 64, 128))
    return cudaErrorInvalidValue;
  if (!make_map_2d(&mB, p.Bt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (uint64_t)p.ldb, (uint64_t)(2 * KP),
                   (uint64_t)p.ldb * 2, 64, 2 * KP))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(prod_tc_bf16_kernel<KP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (e != cudaSuccess) return e;
  ta.stages = C::STAGES;
  prod_tc_bf16_kernel<KP><<<G, kThreads, C::SMEM, s>>>(mS, mB, ta);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(int dtype, int kp) {
  return dtype == 1 && (kp == 8 || kp == 16 || kp == 32 || kp == 64) && encode_fn() != nullptr;
}

int stream_k_ctas(int64_t units, int num_sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(units, num_sms));
}

cudaError_t launch_prod_tc(const ProdArgs &a, cudaStream_t s, int num_sms, int *G_out, int *err) {
  if (a.n_rows_list <= 0 || a.n_cols_list <= 0) return cudaSuccess;
  TcArgs ta{};
  ta.W = (int64_t)a.n_rows_list * a.n_cols_list;
  ta.G = stream_k_ctas(ta.W, num_sms);
  ta.n_cols = a.n_cols_list;
  ta.row_list = a.row_list;
  ta.col_list = a.col_list;
  ta.out = a.out;
  ta.err = err;
  *G_out = ta.G;
  switch (a.kp) {
    case 8: return launch_kp<8>(a, s, ta.G, ta);
    case 16: return launch_kp<16>(a, s, ta.G, ta);
    case 32: return launch_kp<32>(a, s, ta.G, ta);
    case 64: return launch_kp<64>(a, s, ta.G, ta);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace symnmf
