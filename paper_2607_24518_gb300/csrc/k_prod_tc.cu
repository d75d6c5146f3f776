// Tensor-core solver step on sm_103a: the streamed product S H (the S H term
// of the gradient, Sec. 2.1, the dominant cost of every iteration, Sec. 4.3)
// with the iteration's epilogue fused into the same kernel.
//
// One persistent CTA per SM, warp-specialised:
//   warp 0      TMA producer: streams 128-row tiles of S (128-byte swizzled
//               atoms) and the matching slice of the hi/lo MMA copy of H^T
//               into a ring of shared-memory stages
//   warp 1      MMA issuer: one thread issues tcgen05.mma into a double-
//               buffered 128 x 2kp TMEM accumulator (columns [0,kp) multiply
//               H_hi, [kp,2kp) multiply H_lo) and frees stages with
//               tcgen05.commit
//   warps 2-9   epilogue, two threads per tile row (half the columns each):
//               (tcgen05.ld), P = acc_hi + acc_lo, and for a finished tile
//               runs the whole per-row update: g = 4 (H Gram_t - P), the
//               AdaGrad / RMSprop / ADMM step with the max(0, .) projection
//               into the other H buffer, the MMA copy of the new rows, and
//               the tile partials tr = sum H * P, ||grad_proj||^2, sum(G),
//               NaN count and the Gram partial H'^T H'
//   warps 10-13 folders: fold each accumulator chain into FP32 registers and
//               hand a finished tile segment's P over; with FP32 storage
//               they also convert the staged S rows, see below; with FP8
//               storage they apply the per-unit scale of S when folding
// Storage types:
//   BF16  kind::f16, A = S straight from shared memory, B = [H_hi | H_lo]
//         in bf16 (H enters with about 16 significant bits)
//   FP32  error-compensated TF32 (after Ootomo & Yokota, IJHPCA 2022):
//         kind::tf32 reads the staged FP32 S tile straight from shared
//         memory and uses its 19 high bits, i.e. S_hi = S with the 13 low
//         mantissa bits cleared, against B = [H_hi | H_lo] in tf32; the
//         converter warps form S_lo = S - S_hi (exact) and store it in
//         tensor memory, where a second MMA reads it as its A operand: for
//         kp <= 32 rounded to bf16 against a bf16 copy of H (kind::f16),
//         otherwise rounded to tf32 against H_hi (kind::tf32).  What is
//         left out is S_lo H_lo (relative 2^-21) and the rounding of the
//         lo parts
//   FP8   kind::f8f6f4 on the E4M3 codes of S against H as two E4M3 pieces
//         per entry at a power-of-two factor d per 128-row tile,
//         H ~ d (hi + lo); from kp = 16 up the two pieces go through two
//         MMAs of N = kp into one accumulator; S's tile scale over d is
//         applied per unit when the folders fold
// Work: the row-major list of (row tile, 128-column tile) units is split
// into equal contiguous ranges, one per CTA (stream-K), so every SM streams
// the same number of S bytes.  A tile whose units span several CTAs is
// finished by the last of them to arrive (per-tile counter): the others
// leave their FP32 partial in slot (cta + tile); the finisher adds the
// slots in CTA order, so results do not depend on timing.  Finished tiles
// leave per-tile FP64 scalars and FP32 Gram partials; the reduction kernel
// that follows (reduce_iter_kernel in k_epilogue.cu, overlapped with the
// next step by programmatic dependent launch) sums them across tiles in a
// fixed order into the Gram of H_{t+1} and the iteration record.
// Launches over row / column lists (sampled iterations) only write the
// partial slots; the stand-alone epilogue kernel consumes them.
//
// Every mbarrier wait is bounded (2 s of %globaltimer): on expiry the CTA
// records an error code, stops all roles, drains its own copies and MMAs
// with bounded waits, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "epi_common.cuh"
#include "symnmf_internal.h"
#include "tc_ptx.cuh"

namespace symnmf {
namespace {

using namespace tc;

struct TcArgs {
  int64_t W;             // units = n_rows_list * n_cols_list
  int G;                 // CTAs
  int R;                 // row positions (tiles of 128 rows)
  int n_cols;
  const int *row_list;
  const int *col_list;
  float *out;            // partial slots
  int *err;
  int fused;             // run the per-tile epilogue in the kernel
  int *tile_cnt;         // per-tile arrival counters (fused)
  const float *sS;       // FP8: tile scales of S (row pitch ld_sS)
  int64_t ld_sS;
  const float *deq;      // FP8: tile factors d of the MMA copy of H
};

template <int DT, int KP>
struct Cfg {
  static constexpr bool F32 = (DT == 0);
  static constexpr bool F8 = (DT == 2);
  // FP32 with kp <= 32: the S_lo H product runs as kind::f16 on a bf16
  // S_lo (in TMEM) and a bf16 copy of H (N2 rows, zero past kp)
  static constexpr bool SLO16 = F32 && KP <= 32;
  static constexpr int N2 = SLO16 ? (KP < 16 ? 16 : KP) : 0;
  static constexpr int N = 2 * KP;  // rows of the staged B: [H_hi | H_lo]
  // FP8 from kp = 16: S H_hi and S H_lo accumulate into one accumulator
  // (two MMAs of N = kp); kp = 8 keeps one MMA of N = 16 (M = 128 needs N
  // a multiple of 16) and adds the two parts when folding
  static constexpr bool JOIN = F8 && KP >= 16;
  static constexpr int NA = JOIN ? KP : N;  // accumulator columns of the main product
  static constexpr int ATOM_COLS = F32 ? 32 : F8 ? 128 : 64;  // elements per 128-byte row
  static constexpr int APS = (KP == 64 || F8) ? 1 : 2;    // swizzle atoms per stage
  static constexpr int SPU = 128 / (APS * ATOM_COLS);    // stages per 128-column unit
  static constexpr int KSL = 4 * APS;                    // MMA k-slices per stage
  static constexpr uint32_t A_BYTES = APS * kAtomBytes;
  static constexpr uint32_t B_ATOM = N * 128;
  static constexpr uint32_t B_BYTES = APS * B_ATOM;
  static constexpr uint32_t B2_BYTES = SLO16 ? (uint32_t)N2 * 128u : 0u;
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES + B2_BYTES;
  // stages per accumulator chain: the tensor core's FP32 accumulation is
  // kept to at most 8 chained MMAs per accumulator, the rest is summed in
  // FP32 registers
  static constexpr int FOLD = F32 ? 1 : SPU;
  // accumulator columns per part read before one wait when folding
  static constexpr int FOLD_CW = F32 ? 8 : (KP == 64 ? 16 : 32);
  // the epilogue's H tile (kp = 64: and a second tile-shaped buffer for
  // H_t Gram_t and then g, which 32 columns per thread cannot keep in
  // registers); the Gram of H_t is read from global memory (L1)
  static constexpr uint32_t EPI_FLOATS = 128 * (KP + 1) * (KP == 64 ? 2 : 1);
  // + FP8: a ring of 256 unit scales after the epilogue scratch
  static constexpr uint32_t EPI_BYTES = EPI_FLOATS * 4 + 512 + (F8 ? 1024 : 0);
  static constexpr uint32_t BAR_BYTES = 512;
  static constexpr uint32_t BUDGET = 232448u - 1024u - BAR_BYTES - EPI_BYTES;
  // fewer stages than fit measured faster at kp = 64 (every storage type)
  // and with FP8 at kp = 32: about 120-130 KB in flight per SM; more only
  // lengthens the round trips
  static constexpr int STAGE_CAP = KP == 64 ? 4 : (F8 && KP == 32) ? 5 : 8;
  static constexpr int STAGES = (BUDGET / STAGE) < (uint32_t)STAGE_CAP ? (int)(BUDGET / STAGE) : STAGE_CAP;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + BAR_BYTES + EPI_BYTES;
  // MMA issuing threads (warps 1 and 14).  One thread issues a tcgen05.mma
  // about every 60 SM cycles at best, so a skinny-N stream of S is bounded
  // by the issuer unless the chains are split between two of them.
  static constexpr int NISSUE = 2;
  // 16 warps: TMA, MMA, 8 epilogue, 4 folder, second MMA, spare
  static constexpr int THREADS = 512;
  // FP32: TMEM columns of one S_lo buffer, number of S_lo buffers, width
  // of the separate S_lo H accumulator (0: shared with the main one)
  // (SLO16: one bf16 S_lo buffer of 32 columns per ring stage, so a
  // stage's release also frees its S_lo buffer)
  static constexpr uint32_t ABUF = SLO16 ? 32u : F32 ? 32u * APS : 0u;
  static constexpr int NABUF = SLO16 ? STAGES : F32 ? 2 : 1;
  static constexpr int NL = SLO16 ? N2 : 0;
  static constexpr uint32_t ACC0 = F32 ? NABUF * ABUF : 0u;
  static constexpr uint32_t ACCW = NA + NL;               // columns per accumulator buffer
  static constexpr uint32_t PB0 = ACC0 + 2 * ACCW;        // double-buffered P rows
  // kp = 64: the folders keep the running sum of a tile segment in tensor
  // memory (PA) instead of 64 registers per thread, which the 128-register
  // budget of a 16-warp CTA cannot hold next to a fold's loads
  static constexpr bool PTMEM = (KP == 64);
  static constexpr uint32_t PA0 = PB0 + 2 * KP;
  // columns of the running sum kept in registers (kp = 64 with FP32
  // storage: half of them, which measured faster there; BF16 and FP8 keep
  // all of them in PA)
  static constexpr int NPR = !PTMEM ? KP : F32 ? KP / 2 : 0;
  static constexpr uint32_t TMEM_NEED = PA0 + (uint32_t)(KP - NPR);
  static constexpr uint32_t TMEM_COLS = TMEM_NEED <= 32 ? 32 : TMEM_NEED <= 64 ? 64 : TMEM_NEED <= 128 ? 128 : TMEM_NEED <= 256 ? 256 : 512;
  static_assert(STAGES >= 2, "shared memory ring too small");
  static_assert(TMEM_NEED <= 512, "tensor memory budget exceeded");
};

// The units of CTA b are its stream-K share [b W / G, (b+1) W / G) of the
// row-major unit list (W = R n_cols), so every CTA streams the same number
// of units.  A share is made of pieces: the part of its first row
// position, whole row positions, the part of its last row position.  A
// fused step streams its longest piece last (ties: the last one) and the
// rest before it, so every CTA finishes at most one row position at the
// end of its stream, and any other row position it finishes is complete
// with at least half of its share still to stream: the two CTAs sharing a
// row position never both keep their part of it for last.  The two
// segments are the two contiguous ranges in streaming order.  Without the
// fused epilogue the order does not matter and segment 0 is the share.
struct Segs {
  int64_t lo[2], hi[2];
};
__device__ __forceinline__ int64_t sk_start(const TcArgs &a, int b, int64_t W) {
  return (int64_t)b * W / a.G;
}
// CTA holding unit u
__device__ __forceinline__ int64_t sk_owner(const TcArgs &a, int64_t u, int64_t W) {
  return sk_cta(u, W, a.G);
}
__device__ __forceinline__ Segs cta_segments(const TcArgs &a, int b) {
  const int64_t W = (int64_t)a.R * a.n_cols;
  const int64_t lo = sk_start(a, b, W), hi = sk_start(a, b + 1, W);
  Segs s;
  s.lo[0] = lo;
  s.hi[0] = hi;
  s.lo[1] = s.hi[1] = lo;
  if (!a.fused || hi <= lo) return s;
  int64_t mid = (hi - 1) / a.n_cols * a.n_cols;  // start of the last row position
  if (mid <= lo) return s;                      // one piece
  const int64_t l = hi - mid;                   // last piece
  const int64_t f = (lo / a.n_cols + 1) * a.n_cols - lo;  // first piece
  const bool whole_rows = (mid - lo - f) > 0;
  if (l >= f && (!whole_rows || l >= a.n_cols)) {
    s.hi[0] = mid;                              // the last piece goes last
    s.lo[1] = mid;
    s.hi[1] = hi;
  } else {
    s.lo[0] = mid;                              // the last piece first, then
    s.lo[1] = lo;                               // the first piece and whole rows
    s.hi[1] = mid;
  }
  return s;
}
// column position visited for unit L
__device__ __forceinline__ int unit_col(const TcArgs &a, int64_t L) {
  return (int)(L % a.n_cols);
}
// Element (r, c) of partial slot s of a fused step.  Its slots are written
// and read by the epilogue warps of the same kernel only and are column-
// major, so the 32 rows of a warp's load or store of one column are one
// 128-byte line.  (Slots of a launch without the fused epilogue keep the
// row-major layout of part_sum.)
template <int KP>
__device__ __forceinline__ int64_t fslot(int64_t s, int c, int r) {
  return (s * KP + c) * 128 + r;
}

// ------------------------------------------------------------------ epilogue
// The kp x kp Gram partial as an 8 x 8 grid of B x B blocks, one per quad
// of the 256 epilogue threads
template <int KP>
struct GramBlk {
  static constexpr int B = KP / 8;
  static constexpr int BP = B == 8 ? 2 : B;  // block rows summed per pass
};

// Per-tile update for the thread's row (row = tile row, et = index among the
// 128 epilogue threads); p holds the row of S H for H_t, summed in FP32 in
// a fixed order.  Everything the iteration produces for this tile is
// written here; the cross-tile sums are left to the reduction kernel.
// columns owned by each of the two epilogue threads of a row (kp = 8: the
// first thread owns all of them, the second only joins the barriers)
template <int KP>
struct Own {
  static constexpr int KH = KP >= 16 ? KP / 2 : KP;
  static constexpr int HW = KH <= 16 ? KH : 16;  // columns whose state is held at once
  // kp = 64: H_t Gram_t, then g (or ADMM's x), live in the shared-memory
  // buffer Gx rather than in 32 registers per thread
  static constexpr bool GX = (KP == 64);
  static constexpr int HG = GX ? 1 : KH;
};
// the thread's H_t Gram_t for the 8 owned columns from c (row hrow of Hs,
// columns cb + c ..), summed over d in order
template <int KP>
__device__ __forceinline__ void hgram8(const float *hrow, const float *Gs, int cb, int c,
                                       float (&h8)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) h8[j] = 0.f;
#pragma unroll 4
  for (int d = 0; d < KP; ++d) {
    const float hv = hrow[d];
    const float4 *gr = reinterpret_cast<const float4 *>(Gs + d * KP + cb + c);
    const float4 g0 = __ldg(gr), g1 = __ldg(gr + 1);
    h8[0] = fmaf(hv, g0.x, h8[0]);
    h8[1] = fmaf(hv, g0.y, h8[1]);
    h8[2] = fmaf(hv, g0.z, h8[2]);
    h8[3] = fmaf(hv, g0.w, h8[3]);
    h8[4] = fmaf(hv, g1.x, h8[4]);
    h8[5] = fmaf(hv, g1.y, h8[5]);
    h8[6] = fmaf(hv, g1.z, h8[6]);
    h8[7] = fmaf(hv, g1.w, h8[7]);
  }
}

// Rows [0, rows) of a tile held in Hs (row stride KP + 1) to dst (row
// stride KP) by the 256 epilogue threads: each warp store covers whole
// rows of dst, so the tile leaves in full 128-byte lines.
template <int KP>
__device__ __forceinline__ void store_rows(const float *Hs, float *dst, int rows, int et) {
  constexpr int C4 = KP / 4;
#pragma unroll 2
  for (int i = et; i < rows * C4; i += 256) {
    const int r = i / C4, c = (i - r * C4) * 4;
    const float *sp = Hs + r * (KP + 1) + c;
    *reinterpret_cast<float4 *>(dst + (int64_t)r * KP + c) = make_float4(sp[0], sp[1], sp[2], sp[3]);
  }
}

// What a tile's epilogue needs before its S H rows exist: H_t of the tile in
// Hs (both column halves), the thread's optimizer state (the first HW
// owned columns) and its share of H_t Gram_t.  Ends with the tile's H_t in
// Hs for every thread.  The rows are read in whole 128-byte lines by the
// 256 threads together and reach each row's threads through Hs: a load of
// one row per thread would cost one memory request per 16 bytes, and while
// the stream saturates HBM those requests slow the CTA's own TMA copies.
template <int KP>
__device__ __forceinline__ void stage_rows(float *Hs, const float4 (&v)[KP / 8], int et) {
  constexpr int C4 = KP / 4;
#pragma unroll
  for (int i = 0; i < KP / 8; ++i) {
    const int idx = et + 256 * i, r = idx / C4, c = (idx - r * C4) * 4;
    float *d = Hs + r * (KP + 1) + c;
    d[0] = v[i].x;
    d[1] = v[i].y;
    d[2] = v[i].z;
    d[3] = v[i].w;
  }
}
template <int KP>
__device__ __forceinline__ void load_rows(float4 (&v)[KP / 8], const float *src, int rows, int et) {
  constexpr int C4 = KP / 4;
#pragma unroll
  for (int i = 0; i < KP / 8; ++i) {
    const int idx = et + 256 * i;
    v[i] = (idx < rows * C4) ? __ldcg(reinterpret_cast<const float4 *>(src) + idx)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}
template <int DT, int KP>
__device__ __forceinline__ void tile_prep(const EpiArgs &e, int tp, float *Hs, float *Gx,
                                          const float *Gs, int row, int half, int et,
                                          float (&hg)[Own<KP>::HG],
                                          float (&av)[Own<KP>::HW], float (&mv)[Own<KP>::HW]) {
  constexpr int KH = Own<KP>::KH;
  constexpr int HW = Own<KP>::HW;
  const bool works = (KP >= 16) || half == 0;
  const int cb = (KP >= 16) ? half * KH : 0;
  const int64_t r0 = (int64_t)tp * 128;
  const int rows = (int)((e.n - r0) < 128 ? (e.n - r0) : 128);
  const bool rms = (e.method == SYMNMF_RMSPROP);
  float *hrow = Hs + row * (KP + 1);
  // the thread's state columns of A (and M) through Hs, then H_t
  auto take = [&](float (&dst)[HW]) {
#pragma unroll
    for (int j = 0; j < HW; ++j) dst[j] = works ? hrow[cb + j] : 0.f;
  };
  float4 v[KP / 8];
#pragma unroll
  for (int j = 0; j < HW; ++j) av[j] = mv[j] = 0.f;
  if constexpr (DT == 0) {
    // FP32 storage: the folders read the staged S rows from shared memory
    // to split them, and extra shared-memory traffic here slows that more
    // than the row loads below slow the stream
    const bool vrow = works && row < rows;
    const int64_t base = (r0 + row) * KP + cb;
#pragma unroll
    for (int c4 = 0; c4 < HW / 4; ++c4) {
      float4 u = make_float4(0.f, 0.f, 0.f, 0.f), w = u;
      if (vrow && e.update) {
        u = reinterpret_cast<const float4 *>(e.A + base)[c4];
        if (rms) w = reinterpret_cast<const float4 *>(e.M + base)[c4];
      }
      av[4 * c4 + 0] = u.x; av[4 * c4 + 1] = u.y; av[4 * c4 + 2] = u.z; av[4 * c4 + 3] = u.w;
      mv[4 * c4 + 0] = w.x; mv[4 * c4 + 1] = w.y; mv[4 * c4 + 2] = w.z; mv[4 * c4 + 3] = w.w;
    }
    if (works) {
      const float4 *src = reinterpret_cast<const float4 *>(e.H + base);
#pragma unroll
      for (int c4 = 0; c4 < KH / 4; ++c4) {
        const float4 u = (row < rows) ? src[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
        hrow[cb + 4 * c4 + 0] = u.x;
        hrow[cb + 4 * c4 + 1] = u.y;
        hrow[cb + 4 * c4 + 2] = u.z;
        hrow[cb + 4 * c4 + 3] = u.w;
      }
    }
    epi_bar();  // both halves of each H_t row are in Hs
  } else {
  if (e.update) {
    load_rows<KP>(v, e.A + r0 * KP, rows, et);
    stage_rows<KP>(Hs, v, et);
    epi_bar();
    take(av);
    epi_bar();
    if (rms) {
      load_rows<KP>(v, e.M + r0 * KP, rows, et);
      stage_rows<KP>(Hs, v, et);
      epi_bar();
      take(mv);
      epi_bar();
    }
  }
  load_rows<KP>(v, e.H + r0 * KP, rows, et);
  stage_rows<KP>(Hs, v, et);
  epi_bar();  // both halves of each H_t row are in Hs
  }
  // (H_t Gram_t) for the owned columns, right to left (Sec. 2.1)
  if constexpr (Own<KP>::GX) {
    float *gx = Gx + row * (KP + 1) + cb;
#pragma unroll 1
    for (int c = 0; c < KH; c += 8) {
      float h8[8];
      hgram8<KP>(hrow, Gs, cb, c, h8);
#pragma unroll
      for (int j = 0; j < 8; ++j) gx[c + j] = h8[j];
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < Own<KP>::HG; ++j) hg[j] = 0.f;
#pragma unroll 2
  for (int d = 0; d < KP; ++d) {
    const float hv = hrow[d];
    const float4 *gr = reinterpret_cast<const float4 *>(Gs + d * KP + cb);
#pragma unroll
    for (int c4 = 0; c4 < Own<KP>::HG / 4; ++c4) {
      const float4 gv = __ldg(gr + c4);
      hg[4 * c4 + 0] = fmaf(hv, gv.x, hg[4 * c4 + 0]);
      hg[4 * c4 + 1] = fmaf(hv, gv.y, hg[4 * c4 + 1]);
      hg[4 * c4 + 2] = fmaf(hv, gv.z, hg[4 * c4 + 2]);
      hg[4 * c4 + 3] = fmaf(hv, gv.w, hg[4 * c4 + 3]);
    }
  }
}

// The rest of tile tp's epilogue once p holds the thread's S H values (the
// rows of S H_t, summed in FP32 in a fixed order) and tile_prep has run for
// tp: g = coef (H Gram_t - S H), the update and projection into the other H
// buffer, the MMA copy of the new rows, and the tile partials.  Everything
// the iteration produces for this tile is written here; the cross-tile sums
// are left to the reduction kernel.
template <int DT, int KP>
__device__ __forceinline__ void tile_finish(const EpiArgs &e, int tp, float (&p)[Own<KP>::KH],
                                            const float (&hg)[Own<KP>::HG],
                                            float (&av)[Own<KP>::HW], float (&mv)[Own<KP>::HW],
                                            float *Hs, float *Gx, double *scratch, int et,
                                            int row, int half) {
  constexpr int KH = Own<KP>::KH;
  constexpr int HW = Own<KP>::HW;
  const bool works = (KP >= 16) || half == 0;
  const int cb = (KP >= 16) ? half * KH : 0;  // first owned column
  const int64_t r0 = (int64_t)tp * 128;
  const int rows = (int)((e.n - r0) < 128 ? (e.n - r0) : 128);
  const bool vrow = works && row < rows;
  const bool rms = (e.method == SYMNMF_RMSPROP);
  const int64_t base = (r0 + row) * KP + cb;
  float *hrow = Hs + row * (KP + 1);
  auto load_state = [&](int c0) {
#pragma unroll
    for (int c4 = 0; c4 < HW / 4; ++c4) {
      float4 u = make_float4(0.f, 0.f, 0.f, 0.f), w = u;
      if (vrow && e.update) {
        u = reinterpret_cast<const float4 *>(e.A + base + c0)[c4];
        if (rms) w = reinterpret_cast<const float4 *>(e.M + base + c0)[c4];
      }
      av[4 * c4 + 0] = u.x; av[4 * c4 + 1] = u.y; av[4 * c4 + 2] = u.z; av[4 * c4 + 3] = u.w;
      mv[4 * c4 + 0] = w.x; mv[4 * c4 + 1] = w.y; mv[4 * c4 + 2] = w.z; mv[4 * c4 + 3] = w.w;
    }
  };
  // tr(H^T S H) share of the row (Eq. 2) and g = coef ((H Gram_t) - S H)
  float tr = 0.f, kkt2 = 0.f, sumA = 0.f, nonfin = 0.f, hmax = 0.f;
  // ADMM (appendix, Family 6): the handle's H is W and its A buffer the
  // scaled dual U; U of the owned columns is in av when all of them fit
  const bool admm = (e.method == SYMNMF_ADMM);
  auto dual = [&](int j) -> float {
    if constexpr (KH == HW) return av[j];
    else return (vrow && e.update) ? e.A[base + j] : 0.f;
  };
  // H_t Gram_t of column j: in registers, or (kp = 64) in Gx
  float *gxrow = Gx + row * (KP + 1) + cb;
  auto hg_of = [&](int j) -> float {
    if constexpr (Own<KP>::GX) return gxrow[j];
    else return hg[j];
  };
  if (!admm) {
#pragma unroll
    for (int j = 0; j < KH; ++j) {
      float g = 0.f;
      const float hgj = hg_of(j);
      if (cb + j < e.k) {
        tr = fmaf(hrow[cb + j], p[j], tr);
        g = e.coef * (hgj - p[j]);
        const float pg = (hrow[cb + j] > 0.f) ? g : fminf(0.f, g);
        kkt2 = fmaf(pg, pg, kkt2);
        if (!isfinite(g)) nonfin += 1.f;
      }
      if constexpr (Own<KP>::GX) gxrow[j] = g;
      else p[j] = g;
    }
  } else {
    // g goes out at once (checks only); p becomes the right-hand side
    // 2 (S W) + rho (W - U) of the ADMM H-update
#pragma unroll
    for (int c4 = 0; c4 < KH / 4; ++c4) {
      float gg[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = 4 * c4 + jj;
        float g = 0.f, r = 0.f;
        const float hgj = hg_of(j);
        if (cb + j < e.k) {
          const float h = hrow[cb + j];
          tr = fmaf(h, p[j], tr);
          g = e.coef * (hgj - p[j]);
          const float pg = (h > 0.f) ? g : fminf(0.f, g);
          kkt2 = fmaf(pg, pg, kkt2);
          if (!isfinite(g)) nonfin += 1.f;
          r = 2.f * p[j] + e.rho * (h - dual(j));
        }
        gg[jj] = g;
        p[j] = r;
      }
      if (e.gout && vrow)
        reinterpret_cast<float4 *>(e.gout + base)[c4] = make_float4(gg[0], gg[1], gg[2], gg[3]);
    }
  }
  if (!vrow) tr = kkt2 = nonfin = 0.f;
  epi_bar();  // every thread has read H_t from Hs
  if (admm && e.update) {
    // x = rhs (2 W^T W + rho I)^-1 + U for the owned columns (H = rhs
    // Minv); the right-hand-side rows go through Hs
    if (works) {
#pragma unroll
      for (int j = 0; j < KH; ++j) hrow[cb + j] = p[j];
    }
    epi_bar();  // every right-hand-side row is complete
    if (works) {
#pragma unroll
      for (int j = 0; j < KH; ++j) p[j] = dual(j);
#pragma unroll 4
      for (int d = 0; d < KP; ++d) {
        const float rv = hrow[d];
        const float4 *mr = reinterpret_cast<const float4 *>(e.minv + d * KP + cb);
#pragma unroll
        for (int c4 = 0; c4 < KH / 4; ++c4) {
          const float4 m = mr[c4];
          p[4 * c4 + 0] = fmaf(rv, m.x, p[4 * c4 + 0]);
          p[4 * c4 + 1] = fmaf(rv, m.y, p[4 * c4 + 1]);
          p[4 * c4 + 2] = fmaf(rv, m.z, p[4 * c4 + 2]);
          p[4 * c4 + 3] = fmaf(rv, m.w, p[4 * c4 + 3]);
        }
      }
    }
    epi_bar();  // every thread has read the right-hand sides from Hs
  }
  if constexpr (Own<KP>::GX) {
    if (admm) {
#pragma unroll
      for (int j = 0; j < KH; ++j) gxrow[j] = p[j];  // x (update) or the rhs
    }
  }
  // g (ADMM: x) of owned column c
  auto gv = [&](int c) -> float {
    if constexpr (Own<KP>::GX) return gxrow[c];
    else return p[c];
  };
  // update and projection, HW columns at a time (one pass below kp = 64;
  // at kp = 64 the two passes stay a loop, which keeps the state of one
  // in registers at a time)
#pragma unroll 1
  for (int hc = 0; hc < KH; hc += HW) {
    if (hc > 0) load_state(hc);
#pragma unroll
    for (int cc = hc; cc < hc + HW; cc += 8) {
      float hn[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = cb + cc + j, s = cc - hc + j;
        const float h = hrow[c];
        const float g = gv(cc + j);
        hn[j] = h;
        if (e.update) {
          if (c < e.k && vrow) {
            float x;
            if (admm) {
              // W' = [x]_+, U' = x - W' = U + H - W'
              x = gv(cc + j);
              av[s] = x - ((x > 0.f) ? x : 0.f);
              sumA += av[s];
            } else if (rms) {
              const float v = e.alpha * av[s] + (1.f - e.alpha) * (g * g);
              av[s] = v;
              const float m = e.mom * mv[s] + adaptive_step(e.eta * g, v, e.eps);
              mv[s] = m;
              x = h - m;
              sumA += v;
            } else {
              const float acc = av[s] + g * g;
              av[s] = acc;
              x = h - adaptive_step(e.eta * g, acc, e.eps);
              sumA += acc;
            }
            hn[j] = (x > 0.f) ? x : 0.f;
          } else {
            hn[j] = 0.f;
          }
        }
      }
      const int s0 = cc - hc;
      if (vrow) {
        const float4 p0 = make_float4(gv(cc), gv(cc + 1), gv(cc + 2), gv(cc + 3));
        const float4 p1 = make_float4(gv(cc + 4), gv(cc + 5), gv(cc + 6), gv(cc + 7));
        if (e.gout && !admm) {
          float4 *g4 = reinterpret_cast<float4 *>(e.gout + base + cc);
          g4[0] = p0;
          g4[1] = p1;
        }
        if (e.store_mu) {
          float4 *m4 = reinterpret_cast<float4 *>(e.mu + base + cc);
          m4[0] = p0;
          m4[1] = p1;
        }
        if (e.gcaller && !admm) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (cb + cc + j < e.k) e.gcaller[(r0 + row) * e.k + cb + cc + j] = gv(cc + j);
        }
        // H_{t+1} leaves through Hs below, and so does the optimizer
        // state when all of the thread's columns are in registers at once
        if (e.update && KH != HW) {
          float4 *a4 = reinterpret_cast<float4 *>(e.A + base + cc);
          a4[0] = make_float4(av[s0], av[s0 + 1], av[s0 + 2], av[s0 + 3]);
          a4[1] = make_float4(av[s0 + 4], av[s0 + 5], av[s0 + 6], av[s0 + 7]);
          if (rms) {
            float4 *v4 = reinterpret_cast<float4 *>(e.M + base + cc);
            v4[0] = make_float4(mv[s0], mv[s0 + 1], mv[s0 + 2], mv[s0 + 3]);
            v4[1] = make_float4(mv[s0 + 4], mv[s0 + 5], mv[s0 + 6], mv[s0 + 7]);
          }
        }
      }
      if (e.update && works) {
#pragma unroll
        for (int j = 0; j < 8; ++j) hrow[cb + cc + j] = hn[j];
        if constexpr (DT == 2) {
#pragma unroll
          for (int j = 0; j < 8; ++j) hmax = fmaxf(hmax, hn[j]);
        } else if (e.Btn) {
          if (e.bt_fmt == 0) {
            uint16_t *B = reinterpret_cast<uint16_t *>(e.Btn);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const uint16_t hi = bf16_bits(hn[j]);
              B[(int64_t)(cb + cc + j) * e.ldb + r0 + row] = hi;
              B[(int64_t)(KP + cb + cc + j) * e.ldb + r0 + row] = bf16_bits(hn[j] - bf16_val(hi));
            }
          } else {
            float *B = reinterpret_cast<float *>(e.Btn);
            uint16_t *B16 = bt_b16(e.Btn, KP, e.ldb);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float hi = tf32_trunc(hn[j]);
              B[(int64_t)(cb + cc + j) * e.ldb + r0 + row] = hi;
              B[(int64_t)(KP + cb + cc + j) * e.ldb + r0 + row] = tf32_round(hn[j] - hi);
              B16[(int64_t)(cb + cc + j) * e.ldb + r0 + row] = bf16_bits(hn[j]);
            }
          }
        }
      }
    }
  }
  epi_bar();  // Hs holds the tile of H_{t+1}
  if (e.update) store_rows<KP>(Hs, e.Hn + r0 * KP, rows, et);
  if (e.update && e.gram_part) {
    // Each lane quad sums one B x B block of the 8 x 8 block grid in the
    // Gram row order (gram_quad_sum); a warp holds 2 x 4 blocks so that
    // its loads from Hs hit distinct banks.
    using GB = GramBlk<KP>;
    constexpr int B = GB::B, BP = GB::BP;
    const int g = et & 3, bl = (et >> 2) & 7, wq = et >> 5;
    const int c0 = (2 * (wq >> 1) + (bl >> 2)) * B;
    const int d0 = (4 * (wq & 1) + (bl & 3)) * B;
    float *gp = e.gram_part + (int64_t)tp * KP * KP;
#pragma unroll 1
    for (int cp = c0; cp < c0 + B; cp += BP) {  // BP block rows per pass
      float acc[BP][B];
#pragma unroll
      for (int i = 0; i < BP; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) acc[i][j] = 0.f;
#pragma unroll 4
      for (int i = 0; i < 32; ++i) {
        const float *hr = Hs + (4 * i + g) * (KP + 1);
        float x[BP], y[B];
#pragma unroll
        for (int ii = 0; ii < BP; ++ii) x[ii] = hr[cp + ii];
#pragma unroll
        for (int jj = 0; jj < B; ++jj) y[jj] = hr[d0 + jj];
#pragma unroll
        for (int ii = 0; ii < BP; ++ii)
#pragma unroll
          for (int jj = 0; jj < B; ++jj) acc[ii][jj] = fmaf(x[ii], y[jj], acc[ii][jj]);
      }
#pragma unroll
      for (int ii = 0; ii < BP; ++ii) {
#pragma unroll
        for (int jj = 0; jj < B; ++jj) acc[ii][jj] = gram_quad_sum(acc[ii][jj]);
        if ((ii * 4) / BP == g) {  // the quad's lanes share the stores
#pragma unroll
          for (int jj = 0; jj < B; ++jj) gp[(cp + ii) * KP + d0 + jj] = acc[ii][jj];
        }
      }
    }
  }
  // tile scalars: warp xor trees in float-float form (FP64 adds are slow on
  // this part), the warp sums exact in double, then warps added in order
  float fh[3] = {tr, kkt2, sumA}, fl[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 3; ++i) ff_xor_add(fh[i], fl[i], o);
  double v4[4];
#pragma unroll
  for (int i = 0; i < 3; ++i) v4[i] = (double)fh[i] + (double)fl[i];
  v4[3] = (double)__reduce_add_sync(0xffffffffu, (unsigned)nonfin);
  if constexpr (DT == 2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    if ((et & 31) == 0) scratch[32 + (et >> 5)] = (double)hmax;
  }
  if ((et & 31) == 0)
#pragma unroll
    for (int i = 0; i < 4; ++i) scratch[(et >> 5) * 4 + i] = v4[i];
  epi_bar();
  if (et < 4 && e.slots) {
    double sv = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sv += scratch[4 * w + et];
    e.slots[(int64_t)tp * kSlotStride + et] = sv;
  }
  if constexpr (DT == 2) {
    // E4M3 pieces of the tile of H_{t+1} at the tile's power-of-two factor
    if (e.update && e.Btn) {
      float amax = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) amax = fmaxf(amax, (float)scratch[32 + w]);
      const float d = e4m3_tile_scale(amax), inv = 1.f / d;
      if (works) {
        uint8_t *B = reinterpret_cast<uint8_t *>(e.Btn);
#pragma unroll 4
        for (int j = 0; j < KH; ++j) {
          uint8_t hi, lo;
          e4m3_pieces(hrow[cb + j], inv, hi, lo);
          B[(int64_t)(cb + j) * e.ldb + r0 + row] = hi;
          B[(int64_t)(KP + cb + j) * e.ldb + r0 + row] = lo;
        }
      }
      if (et == 0) bt_deq(e.Btn, KP, e.ldb)[tp] = d;
    }
  }
  if constexpr (KH == HW) {
    if (e.update) {
      // the new optimizer state goes out through Hs as well
      epi_bar();  // every read of H_{t+1} from Hs is done
      if (works) {
#pragma unroll
        for (int j = 0; j < KH; ++j) hrow[cb + j] = av[j];
      }
      epi_bar();
      store_rows<KP>(Hs, e.A + r0 * KP, rows, et);
      if (rms) {
        epi_bar();
        if (works) {
#pragma unroll
          for (int j = 0; j < KH; ++j) hrow[cb + j] = mv[j];
        }
        epi_bar();
        store_rows<KP>(Hs, e.M + r0 * KP, rows, et);
      }
    }
  }
  epi_bar();
}

// Shared-memory handshake between the folder and epilogue warps: the folders
// hand over one finished P row block per tile segment through the TMEM P
// buffer pb (double-buffered); sflag carries the epilogue's decisions
// between its threads.
struct Hand {
  uint64_t *pfull, *pempty;
  volatile int *sflag;
};

// Epilogue warps 2-5: one thread per tile row.
template <int DT, int KP>
__device__ void epilogue_role(const TcArgs &a, const EpiArgs &e, uint32_t tmem_base, float *Hs,
                              double *scratch, const Hand &hd,
                              volatile int *abort_flag, const Segs &sg) {
  using C = Cfg<DT, KP>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;
  const int row = q * 32 + lane;
  const int et = (warp - 2) * 32 + lane;  // 0..255
  const int half = (warp - 2) >> 2;       // column half owned
  float *Gx = Hs + 128 * (KP + 1);        // kp = 64 only (Own<KP>::GX)
  if (!a.fused) return;
  // the Gram of H_t and the tile slots belong to the preceding reduction
  // kernel, which may still run (programmatic dependent launch).  The Gram
  // is read from global memory: its next writer is the reduction kernel
  // that follows this step, which starts only after this grid completes.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const float *Gs = e.gram;
  constexpr int KH = Own<KP>::KH;
  constexpr int HW = Own<KP>::HW;
  float hg[Own<KP>::HG], av[HW], mv[HW];
  // The tile segments in streaming order; the epilogue prepares the next
  // one while it is idle, whether or not this CTA will finish it (the
  // last CTA of a tile to arrive does), so a finish starts with its tile's
  // rows and state already loaded.
  auto tile_from = [&](int si, int64_t L) -> int {  // tile of the segment starting at (si, L)
    if (si == 0 && L >= sg.hi[0]) {
      si = 1;
      L = sg.lo[1];
    }
    return (L < sg.hi[si]) ? (int)(L / a.n_cols) : -1;
  };
  // (FP8 storage, where the stream is shortest; otherwise only the tile of
  // the CTA's last unit, which this CTA finishes in practice, is prepared
  // ahead: the registers held across the wait cost the others more)
  constexpr bool kPrepNext = (DT == 2);
  int prepared = -1, final_tp = -1;
  if (sg.hi[0] > sg.lo[0])
    final_tp = (int)(((sg.hi[1] > sg.lo[1] ? sg.hi[1] : sg.hi[0]) - 1) / a.n_cols);
  // (kp = 64 too: its H_t Gram_t waits in Gx, not in registers)
  constexpr bool kPrepAhead = (KH == HW) || Own<KP>::GX;
  if constexpr (kPrepAhead) {
    const int t0 = kPrepNext ? tile_from(0, sg.lo[0]) : final_tp;
    if (t0 >= 0) {
      prepared = t0;
      tile_prep<DT, KP>(e, prepared, Hs, Gx, Gs, row, half, et, hg, av, mv);
    }
  }
  // Parts of tile tp left by other CTAs (fused slots, column-major): the
  // thread's KH columns from cb, for its row.  add_parts adds the parts of
  // CTAs b0..b1 but `self` to p in CTA order (p holds this CTA's part,
  // first in the order); sum_parts forms the CTA-order sum of all of them
  // with p standing for this CTA's part at its place.
  // (kp = 64: 8 columns at a time, fewer live registers; the additions of
  // each column keep CTA order either way)
  constexpr int PC = Own<KP>::GX ? 8 : KH;
  auto load_pc = [&](float (&v)[PC], int64_t bb, int tp, int c) {
#pragma unroll
    for (int j = 0; j < PC; ++j) v[j] = __ldcg(a.out + fslot<KP>(bb + tp, c + j, row));
  };
  auto add_parts = [&](float (&pp)[KH], int64_t b0, int64_t b1, int64_t self, int tp, int cb) {
#pragma unroll
    for (int c0 = 0; c0 < KH; c0 += PC) {
      for (int64_t bb = b0; bb <= b1; ++bb) {
        if (bb == self) continue;
        float v[PC];
        load_pc(v, bb, tp, cb + c0);
#pragma unroll
        for (int j = 0; j < PC; ++j) pp[c0 + j] += v[j];
      }
    }
  };
  auto sum_parts = [&](float (&pp)[KH], int64_t b0, int64_t b1, int64_t self, int tp, int cb) {
#pragma unroll
    for (int c0 = 0; c0 < KH; c0 += PC) {
      float acc[PC];
      if (b0 == self) {
#pragma unroll
        for (int j = 0; j < PC; ++j) acc[j] = pp[c0 + j];
      } else {
        load_pc(acc, b0, tp, cb + c0);
      }
      for (int64_t bb = b0 + 1; bb <= b1; ++bb) {
        if (bb == self) {
#pragma unroll
          for (int j = 0; j < PC; ++j) acc[j] += pp[c0 + j];
        } else {
          float v[PC];
          load_pc(v, bb, tp, cb + c0);
#pragma unroll
          for (int j = 0; j < PC; ++j) acc[j] += v[j];
        }
      }
#pragma unroll
      for (int j = 0; j < PC; ++j) pp[c0 + j] = acc[j];
    }
  };
  const int b = blockIdx.x;
  // holders of the row positions of the share's first and last unit (any
  // other row position of the share is held by this CTA alone), found
  // once while idle (each is a 64-bit division loop) and kept in shared
  // memory: {tile, first holder, last holder} twice, after the scratch
  // sums of tile_finish
  // (kp = 64 with BF16 / FP8 storage computes them per segment: there the
  // extra live state measured slower than the divisions in the tail)
  constexpr bool kOwnersAhead = (KP < 64 || DT == 0);
  int64_t *own = reinterpret_cast<int64_t *>(scratch + 48);
  if (kOwnersAhead && et == 0) {
    const int64_t WR = (int64_t)a.R * a.n_cols;
    const bool two = sg.hi[1] > sg.lo[1];
    const int64_t ulo = two ? (sg.lo[0] < sg.lo[1] ? sg.lo[0] : sg.lo[1]) : sg.lo[0];
    const int64_t uhi = two ? (sg.hi[0] > sg.hi[1] ? sg.hi[0] : sg.hi[1]) : sg.hi[0];
    const int64_t t2[2] = {ulo / a.n_cols, (uhi > ulo ? uhi - 1 : ulo) / a.n_cols};
    for (int i = 0; i < 2; ++i) {
      own[3 * i] = t2[i];
      own[3 * i + 1] = sk_owner(a, t2[i] * a.n_cols, WR);
      own[3 * i + 2] = sk_owner(a, t2[i] * a.n_cols + a.n_cols - 1, WR);
    }
  }
  epi_bar();
  int pb = 0;
  uint32_t pph = 0u;  // bit b: parity of P buffer b
  for (int si = 0; si < 2; ++si)
  for (int64_t L = sg.lo[si], L1 = sg.hi[si]; L < L1;) {
    const int tp = (int)(L / a.n_cols);
    const int64_t tile_end = (int64_t)(tp + 1) * a.n_cols;
    L = L1 < tile_end ? L1 : tile_end;
    if (!warp_wait_idle(&hd.pfull[pb], (pph >> pb) & 1u, abort_flag)) {
      if (lane == 0) {
        set_err(a.err, 6);
        *abort_flag = 1;
      }
      return;
    }
    fence_after();
    // this CTA's part of tile tp, the thread's KH columns
    float p[KH];
    {
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + C::PB0 +
                          (uint32_t)(pb * KP + ((KP >= 16) ? half * KH : 0));
#pragma unroll
      for (int cc = 0; cc < KH; cc += 8) {
        uint32_t x[8];
        tmem_ld8(tb + cc, x);
#pragma unroll
        for (int j = 0; j < 8; ++j) p[cc + j] = __uint_as_float(x[j]);
      }
    }
    fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&hd.pempty[pb]);
    pph ^= 1u << pb;
    pb ^= 1;
    // A row position held by several CTAs is finished by the last of them
    // to arrive (per-tile counter), adding the parts in CTA order.  The
    // first or second holder (own part first: own + s_b0 equals s_b0 + own
    // exactly) finishes without leaving its part when all the others have
    // already arrived; any other arrival stores its part in slot (cta +
    // tile), fenced, and counts itself in.
    int epi = 1;
    const int cb = (KP >= 16) ? half * KH : 0;
    const bool owns = (KP >= 16) || half == 0;
    int64_t b0 = b, b1 = b;
    if constexpr (kOwnersAhead) {
      if (tp == own[0]) {
        b0 = own[1];
        b1 = own[2];
      } else if (tp == own[3]) {
        b0 = own[4];
        b1 = own[5];
      }
    } else {
      const int64_t WR = (int64_t)a.R * a.n_cols;
      b0 = sk_owner(a, (int64_t)tp * a.n_cols, WR);
      b1 = sk_owner(a, (int64_t)tp * a.n_cols + a.n_cols - 1, WR);
    }
    if (b0 < b1) {
      epi = 0;
      if (b - b0 <= 1) {
        if (et == 0) {
          const int arrived = *reinterpret_cast<volatile int *>(&a.tile_cnt[tp]);
          const int last = (arrived == (int)(b1 - b0));
          if (last) a.tile_cnt[tp] = 0;
          *hd.sflag = last;
        }
        epi_bar();
        if (*hd.sflag) epi = 1;
        epi_bar();  // sflag is read before it is reused
      }
      if (epi) {
        __threadfence();
        if (owns) add_parts(p, b0, b1, b, tp, cb);  // own part first
      } else {
        if (owns) {
#pragma unroll
          for (int j = 0; j < KH; ++j) a.out[fslot<KP>(b + tp, cb + j, row)] = p[j];
        }
        __threadfence();
        epi_bar();
        if (et == 0) {
          const int old = atomicAdd(&a.tile_cnt[tp], 1);
          const int last = (old == (int)(b1 - b0));
          if (last) a.tile_cnt[tp] = 0;
          *hd.sflag = last;
        }
        epi_bar();
        if (*hd.sflag) {
          epi = 1;
          __threadfence();
          // every part, this CTA's own at its place in CTA order
          if (owns) sum_parts(p, b0, b1, b, tp, cb);
        }
        epi_bar();  // sflag is read before it is reused
      }
    }
    if (epi) {
      if (tp != prepared) {
        epi_bar();  // no thread still reads Hs of an earlier tile
        tile_prep<DT, KP>(e, tp, Hs, Gx, Gs, row, half, et, hg, av, mv);
      }
      prepared = -1;
      tile_finish<DT, KP>(e, tp, p, hg, av, mv, Hs, Gx, scratch, et, row, half);
    }
    if constexpr (kPrepAhead) {
      // prepare the next segment's tile while the stream goes on
      const int nx = kPrepNext ? tile_from(si, L) : (epi && tp != final_tp) ? final_tp : -1;
      if (nx >= 0 && nx != prepared) {
        epi_bar();  // no thread still reads Hs
        prepared = nx;
        tile_prep<DT, KP>(e, prepared, Hs, Gx, Gs, row, half, et, hg, av, mv);
      }
    }
  }
}

// Folder warps 6-9: fold each accumulator chain (<= 16 MMAs) into FP32
// registers, one thread per tile row, and hand the tile segment's P over.
// With FP32 storage the same warps first convert each staged S row into
// its tf32 hi / lo parts in TMEM (the MMA's A operand).
template <int DT, int KP>
__device__ void folder_role(const TcArgs &a, uint32_t tmem_base, uint8_t *smem, uint64_t *full,
                            uint64_t *empty, uint64_t *afull, uint64_t *aempty, uint64_t *tfull,
                            uint64_t *tempty, const Hand &hd,
                            volatile int *abort_flag, const Segs &sg, int b, float *sring) {
  using C = Cfg<DT, KP>;
  constexpr int STAGES = C::STAGES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;
  const int row = q * 32 + lane;
  const int ft = (warp - 10) * 32 + lane;
  const uint32_t lane_off = (uint32_t)(q * 32) << 16;
  constexpr int NP = C::NPR;  // columns [0, NP) of the sum in registers, the rest in PA
  constexpr int NPA = NP > 0 ? NP : 1;
  float p[NPA];
#pragma unroll
  for (int c = 0; c < NPA; ++c) p[c] = 0.f;
  bool pa_first = true;                   // PTMEM: the next fold starts PA (columns [NP, kp))
  const uint32_t tpa = tmem_base + lane_off + C::PA0;
  int acc = 0, pb = 0;
  uint32_t tph = 0u, pph = 0u;  // bit i: parity of accumulator / P buffer i
  bool ok = true;

  auto fail = [&](int code) {
    if (lane == 0) {
      set_err(a.err, code);
      *abort_flag = 1;
    }
    ok = false;
  };
  // A fused step hands every finished tile segment's P over to the
  // epilogue warps through TMEM P buffer pb; they finish the tile or leave
  // the partial for another CTA, so no store, fence or counter waits in
  // the folders' path.  Without the fused epilogue the folders store the
  // segment's partial themselves (row-major slot b + tp).
  auto handoff = [&]() {
    if (!warp_wait_idle(&hd.pempty[pb], ((pph >> pb) & 1u) ^ 1u, abort_flag)) {
      fail(7);
      return;
    }
    fence_after();
    const uint32_t tb = tmem_base + lane_off + C::PB0 + (uint32_t)(pb * KP);
    if constexpr (C::PTMEM) {
#pragma unroll
      for (int cc = NP; cc < KP; cc += 16) {
        uint32_t x[16];
        tmem_ld8_nw(tpa + (cc - NP), x, 0);
        tmem_ld8_nw(tpa + (cc - NP) + 8, x, 8);
        tmem_wait_ld_all(x);
        tmem_st16(tb + cc, x);
      }
    }
    {
#pragma unroll
      for (int cc = 0; cc < NP; cc += 8) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = p[cc + j];
        tmem_st8(tb + cc, v);
      }
    }
    tmem_wait_st();
    fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&hd.pfull[pb]);
    pph ^= 1u << pb;
    pb ^= 1;
  };
  auto finish_segment = [&](int tp) {
    if (a.fused) {
      handoff();
    } else {
      float *dst = a.out + ((int64_t)(b + tp) * 128 + row) * KP;
      if constexpr (C::PTMEM) {
#pragma unroll
        for (int cc = NP; cc < KP; cc += 16) {
          uint32_t x[16];
          tmem_ld8_nw(tpa + (cc - NP), x, 0);
          tmem_ld8_nw(tpa + (cc - NP) + 8, x, 8);
          tmem_wait_ld_all(x);
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4)
            reinterpret_cast<float4 *>(dst + cc)[c4] =
                make_float4(__uint_as_float(x[4 * c4]), __uint_as_float(x[4 * c4 + 1]),
                            __uint_as_float(x[4 * c4 + 2]), __uint_as_float(x[4 * c4 + 3]));
        }
      }
#pragma unroll
      for (int cc = 0; cc < NP; cc += 4)
        reinterpret_cast<float4 *>(dst + cc)[0] = make_float4(p[cc], p[cc + 1], p[cc + 2], p[cc + 3]);
    }
#pragma unroll
    for (int c = 0; c < NP; ++c) p[c] = 0.f;
    pa_first = true;
  };
  // fold accumulator chain f (stage-sized chunks [f FOLD, (f+1) FOLD))
  // FP8: the scale of each unit (S tile scale over the H tile factor) comes
  // from a shared ring of 2 x 128 entries in this CTA's unit order.  The
  // 128 folder threads load block j + 2 together at the end of block j and
  // store it 128 folds later, so no fold waits on these loads.
  const int64_t len0 = sg.hi[0] - sg.lo[0];
  const int64_t nunits = len0 + (sg.hi[1] - sg.lo[1]);
  auto scale_of = [&](int64_t i) -> float {
    if (i >= nunits) return 1.f;
    const int si = i < len0 ? 0 : 1;
    const int64_t u = i < len0 ? sg.lo[0] + i : sg.lo[1] + (i - len0);
    const int tp = (int)(u / a.n_cols), ci = unit_col(a, u);
    const int rt = a.row_list ? a.row_list[tp] : tp;
    const int ct = a.col_list ? a.col_list[ci] : ci;
    return __ldg(a.sS + (int64_t)rt * a.ld_sS + ct) * __ldg(a.deq + ct);
  };
  int64_t fcount = 0;  // units folded so far
  int fold_si = -1;     // segment of the last fold, and the end of its tile row
  int64_t tile_end = 0;
  float pre = 1.f;     // this thread's entry of the block two ahead
  if constexpr (C::F8) {
    sring[ft] = scale_of(ft);
    fold_bar();
    pre = scale_of(128 + ft);
  }
  // fold accumulator chain f (stage-sized chunks [f FOLD, (f+1) FOLD)) of
  // segment si, which ends at unit Lhi
  auto fold = [&](int64_t f, int64_t Lhi, int si) {
    float sc = 1.f;
    if constexpr (C::F8) {  // one unit per chain, in this CTA's order
      sc = sring[fcount & 255];
      if ((fcount & 127) == 127) {
        sring[(((fcount >> 7) + 1) & 1) * 128 + ft] = pre;
        fold_bar();
        pre = scale_of(((fcount >> 7) + 2) * 128 + ft);
      }
      ++fcount;
    }
    if (!warp_wait(&tfull[acc], (tph >> acc) & 1u, abort_flag)) {
      fail(5);
      return;
    }
    fence_after();
    const uint32_t tb = tmem_base + lane_off + C::ACC0 + (uint32_t)acc * C::ACCW;
    // CW columns of each accumulator part per round: all of a round's
    // loads are in flight before its one wait
    constexpr int NPART = (C::JOIN ? 1 : 2) + (C::NL > 0 ? 1 : 0);
    constexpr int CW = (KP < C::FOLD_CW) ? KP : C::FOLD_CW;
    if constexpr (C::PTMEM) {
      // columns [0, NP): p += this chain, 16 columns per round
#pragma unroll
      for (int cc = 0; cc < NP; cc += 16) {
        uint32_t x[NPART * 16];
#pragma unroll
        for (int u = 0; u < 16; u += 8) {
          tmem_ld8_nw(tb + cc + u, x, u);
          if constexpr (!C::JOIN) tmem_ld8_nw(tb + KP + cc + u, x, 16 + u);
          if constexpr (C::NL > 0) tmem_ld8_nw(tb + C::N + cc + u, x, 32 + u);
        }
        tmem_wait_ld_all(x);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float v;
          if constexpr (C::JOIN) {
            v = __uint_as_float(x[j]) * sc;
          } else if constexpr (C::F8) {
            v = (__uint_as_float(x[j]) + __uint_as_float(x[16 + j])) * sc;
          } else {
            v = __uint_as_float(x[j]) + __uint_as_float(x[16 + j]);
          }
          if constexpr (C::NL > 0) v += __uint_as_float(x[32 + j]);
          p[cc + j] += v;
        }
      }
      // columns [NP, kp): PA = (pa_first ? 0 : PA) + this chain
#pragma unroll
      for (int cc = NP; cc < KP; cc += 16) {
        uint32_t x[(NPART + 1) * 16];
#pragma unroll
        for (int u = 0; u < 16; u += 8) {
          tmem_ld8_nw(tb + cc + u, x, u);
          if constexpr (!C::JOIN) tmem_ld8_nw(tb + KP + cc + u, x, 16 + u);
          if constexpr (C::NL > 0) tmem_ld8_nw(tb + C::N + cc + u, x, 32 + u);
          if (!pa_first) tmem_ld8_nw(tpa + (cc - NP) + u, x, NPART * 16 + u);
        }
        tmem_wait_ld_all(x);
        uint32_t o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float v;
          if constexpr (C::JOIN) {
            v = __uint_as_float(x[j]) * sc;
          } else if constexpr (C::F8) {
            v = (__uint_as_float(x[j]) + __uint_as_float(x[16 + j])) * sc;
          } else {
            v = __uint_as_float(x[j]) + __uint_as_float(x[16 + j]);
          }
          if constexpr (C::NL > 0) v += __uint_as_float(x[32 + j]);
          o[j] = __float_as_uint(pa_first ? v : __uint_as_float(x[NPART * 16 + j]) + v);
        }
        tmem_st16(tpa + (cc - NP), o);
      }
      tmem_wait_st();
      pa_first = false;
    } else
#pragma unroll
    for (int cc = 0; cc < KP; cc += CW) {
      uint32_t x[NPART * CW];
#pragma unroll
      for (int u = 0; u < CW; u += 8) {
        tmem_ld8_nw(tb + cc + u, x, u);                 // [H_hi] part (FP8 from kp = 16: the sum)
        if constexpr (!C::JOIN)
          tmem_ld8_nw(tb + KP + cc + u, x, CW + u);     // [H_lo] part
        if constexpr (C::NL > 0)                        // S_lo bf16(H)
          tmem_ld8_nw(tb + C::N + cc + u, x, 2 * CW + u);
      }
      tmem_wait_ld_all(x);
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        float v;
        if constexpr (C::JOIN) {
          v = __uint_as_float(x[j]) * sc;
        } else if constexpr (C::F8) {
          v = (__uint_as_float(x[j]) + __uint_as_float(x[CW + j])) * sc;
        } else {
          v = __uint_as_float(x[j]) + __uint_as_float(x[CW + j]);
        }
        if constexpr (C::NL > 0) v += __uint_as_float(x[2 * CW + j]);
        p[cc + j] += v;
      }
    }
    fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&tempty[acc]);
    tph ^= 1u << acc;
    acc ^= 1;
    const int64_t cend = (f + 1) * C::FOLD;
    if (cend % C::SPU == 0) {
      const int64_t u = cend / C::SPU - 1;  // unit just completed
      // end of the current tile row, stepped rather than divided per unit
      if (si != fold_si) {
        fold_si = si;
        tile_end = (u / a.n_cols + 1) * a.n_cols;
      }
      if (u + 1 == Lhi || u + 1 == tile_end) finish_segment((int)(u / a.n_cols));
      if (u + 1 == tile_end) tile_end += a.n_cols;
    }
  };

  if constexpr (C::F32) {
    int stage = 0;
    uint32_t phase = 0;
    uint32_t eph[4] = {0u, 0u, 0u, 0u};
    int64_t prev = -1, prev_hi = 0;  // chunk waiting to be folded
    int prev_si = 0;
    int64_t run = 0;                  // chunks converted so far
    for (int si = 0; si < 2 && ok; ++si)
    for (int64_t c = sg.lo[si] * C::SPU; c < sg.hi[si] * C::SPU && ok; ++c, ++run) {
      const int ab = C::SLO16 ? stage : (int)(run % C::NABUF);
      if (!warp_wait(&full[stage], phase, abort_flag) ||
          (!C::SLO16 && !warp_wait(&aempty[ab], eph[ab] ^ 1, abort_flag))) {
        fail(15);
        break;
      }
      fence_after();
      const uint8_t *sa = smem + stage * C::STAGE;
      if constexpr (C::SLO16) {
        // S_lo = S - tf32_trunc(S) (exact), rounded to bf16, two per column
#pragma unroll
        for (int at = 0; at < C::APS; ++at) {
          const uint8_t *rowp = sa + at * kAtomBytes + row * 128;
          uint32_t pk[16];
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {  // 16-byte chunk of the 128-byte row
            const float4 v = *reinterpret_cast<const float4 *>(rowp + ((ch ^ (row & 7)) << 4));
            const __nv_bfloat162 l01 =
                __floats2bfloat162_rn(v.x - tf32_trunc(v.x), v.y - tf32_trunc(v.y));
            const __nv_bfloat162 l23 =
                __floats2bfloat162_rn(v.z - tf32_trunc(v.z), v.w - tf32_trunc(v.w));
            pk[2 * ch] = *reinterpret_cast<const uint32_t *>(&l01);
            pk[2 * ch + 1] = *reinterpret_cast<const uint32_t *>(&l23);
          }
          tmem_st16(tmem_base + lane_off + (uint32_t)ab * C::ABUF + (uint32_t)at * 16u, pk);
        }
      } else
#pragma unroll
      for (int at = 0; at < C::APS; ++at) {
        const uint8_t *rowp = sa + at * kAtomBytes + row * 128;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {  // 16 columns at a time
          uint32_t lo[16];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int ch = 4 * hh + j;  // 16-byte chunk of the 128-byte row
            const float4 v = *reinterpret_cast<const float4 *>(rowp + ((ch ^ (row & 7)) << 4));
            const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
              lo[4 * j + u] = __float_as_uint(tf32_round(x[u] - tf32_trunc(x[u])));
          }
          tmem_st16(tmem_base + lane_off + (uint32_t)ab * C::ABUF + (uint32_t)at * 32u +
                        (uint32_t)hh * 16u,
                    lo);
        }
      }
      tmem_wait_st();
      fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&empty[stage]);
        mbar_arrive(&afull[ab]);
      }
      if constexpr (!C::SLO16) eph[ab] ^= 1;
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1;
      }
      if (prev >= 0) fold(prev, prev_hi, prev_si);  // FOLD == 1: one chain per stage
      prev = c;
      prev_hi = sg.hi[si];
      prev_si = si;
    }
    if (ok && prev >= 0) fold(prev, prev_hi, prev_si);
  } else {
    for (int si = 0; si < 2; ++si)
      for (int64_t f = sg.lo[si] * C::SPU / C::FOLD; f < sg.hi[si] * C::SPU / C::FOLD && ok; ++f)
        fold(f, sg.hi[si], si);
  }
}

// MMA issuer `who` of NISSUE: issues the accumulator chains c with
// c % NISSUE == who (chain c covers the CTA's stages [c FOLD, (c+1) FOLD)
// and accumulates into buffer c % 2), commits each stage to its ring slot's
// empty barrier and each finished chain to tfull.  The loop keeps its ring
// position, phases and accumulator parities in registers and advances the
// shared-memory descriptors by constant offsets: the issue rate of a single
// thread bounds the stream.  On return *consumed holds the first stage this
// issuer did not finish (the CTA's stage count when it finished all).
template <int DT, int KP>
__device__ __noinline__ void mma_role(const TcArgs &a, const Segs &sg, uint8_t *smem, uint32_t tmem_base,
                         uint64_t *full, uint64_t *empty, uint64_t *afull, uint64_t *aempty,
                         uint64_t *tfull, uint64_t *tempty, uint64_t *drain, int *consumed,
                         volatile int *abort_flag, int who) {
  using C = Cfg<DT, KP>;
  constexpr int STAGES = C::STAGES;
  constexpr int N = C::N;
  constexpr int FOLD = C::FOLD;
  constexpr uint32_t idesc =
      C::F32 ? idesc_tf32(128, N) : C::F8 ? idesc_e4m3(128, C::NA) : idesc_bf16(128, N);
  constexpr uint64_t kLoD = (uint64_t)(KP * 128) >> 4;  // H_lo rows of the staged B
  // descriptor units are 16 bytes; stage, atom and 32-byte K-slice offsets
  constexpr uint64_t kStageD = C::STAGE >> 4, kAtomD = kAtomBytes >> 4, kBAtomD = C::B_ATOM >> 4;
  const uint64_t ad_base = sdesc(smem_u32(smem));
  const int64_t nst = (sg.hi[0] - sg.lo[0] + sg.hi[1] - sg.lo[1]) * C::SPU;
  const int64_t nchain = nst / FOLD;
  int stage = 0;
  uint32_t phase = 0, tph = 0;  // tph bit i: parity of accumulator i
  int64_t g = 0;                // CTA stage index of `stage`
  bool ok = true;
  for (int64_t c = 0; c < nchain && ok; ++c) {
    if ((int)(c % C::NISSUE) != who) {  // the other issuer's chain
      g += FOLD;
      stage += FOLD;
      while (stage >= STAGES) {
        stage -= STAGES;
        phase ^= 1u;
      }
      continue;
    }
    const int acc = (int)(c & 1);
    if (!mbar_wait(&tempty[acc], ((tph >> acc) & 1u) ^ 1u, abort_flag)) {
      set_err(a.err, 2);
      ok = false;
      break;
    }
    const uint32_t d = tmem_base + C::ACC0 + (uint32_t)acc * C::ACCW;
#pragma unroll
    for (int t = 0; t < FOLD; ++t, ++g) {
      if (!mbar_wait(&full[stage], phase, abort_flag)) {
        set_err(a.err, 3);
        ok = false;
        break;
      }
      fence_after();
      const uint64_t ad = ad_base + (uint64_t)stage * kStageD;
      const uint64_t bd = ad + (C::A_BYTES >> 4);
      const uint32_t first = (t == 0) ? 0u : 1u;
#pragma unroll
      for (int j = 0; j < C::KSL; ++j) {
        const uint64_t off = (uint64_t)(j & 3) * 2u;  // 32-byte K slice within a 128-byte row
        const uint64_t adj = ad + (uint64_t)(j >> 2) * kAtomD + off;
        const uint64_t bdj = bd + (uint64_t)(j >> 2) * kBAtomD + off;
        const uint32_t accum = (j == 0) ? first : 1u;
        if constexpr (C::F32) {
          mma_tf32_ss(d, adj, bdj, idesc, accum);
        } else if constexpr (C::F8) {
          mma_e4m3(d, adj, bdj, idesc, accum);
          if constexpr (C::JOIN) mma_e4m3(d, adj, bdj + kLoD, idesc, 1u);
        } else {
          mma_bf16(d, adj, bdj, idesc, accum);
        }
      }
      if constexpr (C::F32) {
        // S_lo H once the converter warps have stored S_lo in TMEM: as
        // kind::f16 against bf16(H) (kp <= 32), else as tf32 against H_hi
        // into the H_lo part
        const int ab = C::SLO16 ? stage : (int)(g % C::NABUF);
        const uint32_t aparity = C::SLO16 ? phase : (uint32_t)((g / C::NABUF) & 1);
        if (!mbar_wait(&afull[ab], aparity, abort_flag)) {
          set_err(a.err, 3);
          ok = false;
          break;
        }
        fence_after();
        if constexpr (C::SLO16) {
          constexpr uint32_t idesc16 = idesc_bf16(128, C::N2);
          const uint64_t bd2 = bd + (C::B_BYTES >> 4);
#pragma unroll
          for (int j = 0; j < C::APS * 2; ++j) {
            const uint32_t alo = tmem_base + (uint32_t)ab * C::ABUF + (uint32_t)j * 8u;
            mma_bf16_ta(d + N, alo, bd2 + (uint64_t)j * 2u, idesc16, (j == 0) ? first : 1u);
          }
        } else {
          constexpr uint32_t idesc_lo = idesc_tf32(128, KP >= 16 ? KP : N);
#pragma unroll
          for (int j = 0; j < C::KSL; ++j) {
            const uint64_t bdj = bd + (uint64_t)(j >> 2) * kBAtomD + (uint64_t)(j & 3) * 2u;
            const uint32_t alo = tmem_base + (uint32_t)ab * C::ABUF + (uint32_t)j * 8u;
            mma_tf32_ta(d + (KP >= 16 ? KP : 0), alo, bdj, idesc_lo, 1u);
          }
          mma_commit(&aempty[ab]);
        }
      }
      mma_commit(&empty[stage]);
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
    if (!ok) break;
    mma_commit(&tfull[acc]);
    tph ^= 1u << acc;
  }
  if (!ok) *abort_flag = 1;
  consumed[who] = (int)g;
  mma_commit(&drain[who]);
  if (!mbar_wait(&drain[who], 0, abort_flag, 100000000ull) && !*abort_flag) set_err(a.err, 4);
}

// -------------------------------------------------------------------- kernel
template <int DT, int KP>
__global__ void __launch_bounds__(Cfg<DT, KP>::THREADS, 1)
    step_tc_kernel(const __grid_constant__ CUtensorMap mapS,
                   const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapB2, const TcArgs a, const EpiArgs e) {
  using C = Cfg<DT, KP>;
  constexpr int N = C::N;
  constexpr int STAGES = C::STAGES;
  constexpr bool F32 = C::F32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * C::STAGE);
  uint64_t *empty = full + STAGES;
  uint64_t *afull = empty + STAGES;
  uint64_t *aempty = afull + 8;
  uint64_t *tfull = aempty + 4;
  uint64_t *tempty = tfull + 2;
  uint64_t *pfull = tempty + 2;
  uint64_t *pempty = pfull + 2;
  uint64_t *drain = pempty + 2;  // one per MMA issuer
  uint32_t *holder = reinterpret_cast<uint32_t *>(drain + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(holder + 1);
  int *consumed = const_cast<int *>(abort_flag) + 1;  // one per MMA issuer
  volatile int *sflag = consumed + 2;
  float *Hs = reinterpret_cast<float *>(smem + STAGES * C::STAGE + C::BAR_BYTES);
  double *scratch = reinterpret_cast<double *>(
      (reinterpret_cast<uintptr_t>(Hs + C::EPI_FLOATS) + 15) & ~uintptr_t(15));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], F32 ? 5 : 1);  // (4 converter warps +) the MMA commit
    }
    for (int i = 0; i < 8; ++i) mbar_init(&afull[i], 4);
    for (int i = 0; i < 4; ++i) mbar_init(&aempty[i], 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
      mbar_init(&pfull[i], 4);
      mbar_init(&pempty[i], 8);
    }
    mbar_init(&drain[0], 1);
    mbar_init(&drain[1], 1);
    *abort_flag = 0;
    consumed[0] = consumed[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(holder, C::TMEM_COLS);
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *holder;

  const int b = blockIdx.x;
  const Segs sg = cta_segments(a, b);
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapS)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
      if constexpr (C::SLO16)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB2)) : "memory");
      // unit coordinates are stepped, not divided: one thread issues every
      // copy, and a 64-bit division per stage would bound the stream
      int stage = 0;
      uint32_t phase = 0;
      bool stop = false;
      for (int si = 0; si < 2 && !stop; ++si) {
        if (sg.hi[si] <= sg.lo[si]) continue;
        int tp = (int)(sg.lo[si] / a.n_cols);
        int ci = unit_col(a, sg.lo[si]);
        int cpos = (int)(sg.lo[si] - (int64_t)tp * a.n_cols);
        int rt = a.row_list ? a.row_list[tp] : tp;
        for (int64_t L = sg.lo[si]; L < sg.hi[si] && !stop; ++L) {
          const int ct = a.col_list ? a.col_list[ci] : ci;
#pragma unroll 1
          for (int kc = 0; kc < C::SPU; ++kc) {
            if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) {
              set_err(a.err, 1);
              *abort_flag = 1;
              stop = true;
              break;
            }
            uint8_t *sa = smem + stage * C::STAGE;
            uint8_t *sb = sa + C::A_BYTES;
            const int x0 = ct * 128 + kc * (C::APS * C::ATOM_COLS);
            mbar_expect_tx(&full[stage], C::STAGE);
#pragma unroll
            for (int at = 0; at < C::APS; ++at) {
              tma_load_2d(sa + at * kAtomBytes, &mapS, &full[stage], x0 + at * C::ATOM_COLS, rt * 128);
              tma_load_2d(sb + at * C::B_ATOM, &mapB, &full[stage], x0 + at * C::ATOM_COLS, 0);
            }
            if constexpr (C::SLO16)  // bf16 H^T rows for the stage's 64 columns
              tma_load_2d(sb + C::B_BYTES, &mapB2, &full[stage], x0, 0);
            ++issued;
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
          // next unit: the column steps by one (mod n_cols) and the row
          // position advances at the end of each tile row
          if (++ci == a.n_cols) ci = 0;
          if (++cpos == a.n_cols && L + 1 < sg.hi[si]) {
            cpos = 0;
            ++tp;
            rt = a.row_list ? a.row_list[tp] : tp;
          }
        }
      }
    }
  } else if (warp == 1 || (C::NISSUE == 2 && warp == 14)) {
    if (lane == 0)
      mma_role<DT, KP>(a, sg, smem, tmem_base, full, empty, afull, aempty, tfull, tempty, drain,
                       consumed, abort_flag, warp == 1 ? 0 : 1);
  } else if (warp >= 10 && warp < 14) {
    const Hand hd{pfull, pempty, sflag};
    folder_role<DT, KP>(a, tmem_base, smem, full, empty, afull, aempty, tfull, tempty, hd,
                        abort_flag, sg, b, reinterpret_cast<float *>(scratch + 64));
  } else if (warp >= 2 && warp < 10) {
    const Hand hd{pfull, pempty, sflag};
    epilogue_role<DT, KP>(a, e, tmem_base, Hs, scratch, hd, abort_flag, sg);
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && *abort_flag) {
    // drain TMA copies that were issued but never consumed (bounded)
    const int from = C::NISSUE == 2 ? min(consumed[0], consumed[1]) : consumed[0];
    int stage = from % STAGES;
    uint32_t phase = (uint32_t)((from / STAGES) & 1);
    for (int i = from; i < issued; ++i) {
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

// ------------------------------------------------------------------- host
template <int DT, int KP>
cudaError_t launch_cfg(const ProdArgs &p, const EpiArgs &e, cudaStream_t s, const TcArgs &ta) {
  using C = Cfg<DT, KP>;
  const CUtensorMapDataType t = C::F32  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                : C::F8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                        : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint64_t es = C::F32 ? 4 : C::F8 ? 1 : 2;
  CUtensorMap mS, mB;
  if (!make_map_2d(&mS, p.S, t, (uint64_t)p.n, (uint64_t)p.n, (uint64_t)p.lds * es, C::ATOM_COLS,
                   128))
    return cudaErrorInvalidValue;
  if (!make_map_2d(&mB, p.Bt, t, (uint64_t)p.ldb, (uint64_t)(2 * KP), (uint64_t)p.ldb * es,
                   C::ATOM_COLS, 2 * KP))
    return cudaErrorInvalidValue;
  CUtensorMap mB2 = mB;
  if constexpr (C::SLO16) {
    if (!make_map_2d(&mB2, bt_b16(const_cast<void *>(p.Bt), KP, p.ldb),
                     CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (uint64_t)p.ldb, (uint64_t)C::N2,
                     (uint64_t)p.ldb * 2, 64, C::N2))
      return cudaErrorInvalidValue;
  }
  cudaError_t err = cudaFuncSetAttribute(step_tc_kernel<DT, KP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (err != cudaSuccess) return err;
  // fused steps may start while the previous iteration's reduction kernel
  // runs: the stream of S needs only H_t, which the previous step wrote
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ta.G);
  cfg.blockDim = dim3(C::THREADS);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = ta.fused ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, step_tc_kernel<DT, KP>, mS, mB, mB2, ta, e);
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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
                 uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                 int swizzle_bytes) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_supported(int dtype, int kp) {
  return (dtype == 0 || dtype == 1 || dtype == 2) && (kp == 8 || kp == 16 || kp == 32 || kp == 64) &&
         encode_fn() != nullptr;
}

cudaError_t launch_step_tc(const ProdArgs &a, const EpiArgs *epi, int *tile_cnt, cudaStream_t s,
                           int num_sms, int *G_out, int *err) {
  if (a.n_rows_list <= 0 || a.n_cols_list <= 0) return cudaSuccess;
  TcArgs ta{};
  ta.W = (int64_t)a.n_rows_list * a.n_cols_list;
  ta.G = (int)std::max<int64_t>(1, std::min<int64_t>(ta.W, num_sms));
  ta.n_cols = a.n_cols_list;
  ta.row_list = a.row_list;
  ta.col_list = a.col_list;
  ta.out = a.out;
  ta.err = err;
  ta.fused = (epi != nullptr) ? 1 : 0;
  ta.tile_cnt = tile_cnt;
  // every row position shared stream-K style (owning whole tiles makes the
  // leftover tiles' last arrivers add ~G / R partials each while HBM is
  // saturated, which measured slower)
  ta.R = a.n_rows_list;
  ta.sS = a.scales;
  ta.ld_sS = a.ld_scales;
  *G_out = ta.G;
  EpiArgs e{};
  if (epi) e = *epi;
  const int want_fmt = (a.dtype == 0) ? 1 : (a.dtype == 2) ? 2 : 0;
  if (a.bt_fmt != want_fmt) return cudaErrorInvalidValue;
  if (a.dtype == 2) {
    if (!a.scales) return cudaErrorInvalidValue;
    ta.deq = bt_deq(const_cast<void *>(a.Bt), a.kp, a.ldb);
  }
#define SYMNMF_TC_CASE(DTV)                           \
  switch (a.kp) {                                     \
    case 8: return launch_cfg<DTV, 8>(a, e, s, ta);   \
    case 16: return launch_cfg<DTV, 16>(a, e, s, ta); \
    case 32: return launch_cfg<DTV, 32>(a, e, s, ta); \
    case 64: return launch_cfg<DTV, 64>(a, e, s, ta); \
    default: return cudaErrorInvalidValue;            \
  }
  if (a.dtype == 0) {
    SYMNMF_TC_CASE(0)
  } else if (a.dtype == 1) {
    SYMNMF_TC_CASE(1)
  } else if (a.dtype == 2) {
    SYMNMF_TC_CASE(2)
  }
#undef SYMNMF_TC_CASE
  return cudaErrorInvalidValue;
}

}  // namespace symnmf
