// Internal declarations shared by the host runtime (capi.cu) and the kernels.
// Layout conventions (all owned buffers):
//   * row tiles are 128 rows; ntiles = ceil(n / 128)
//   * n x k state arrays (H, G / v, m, mu, g) are stored row-major with kp
//     (8, 16, 32 or 64 >= k) columns and ntiles * 128 rows; columns k..kp-1
//     and rows past n are held at exactly 0, so the padding never moves
//   * product partial slots are 128 x kp row-major blocks
//   * the MMA copy of H is stored transposed, [2*kp][ldb] with rows 0..kp-1
//     = hi(H^T) and kp..2kp-1 = lo(H^T), ldb = ntiles * 128 (columns past n
//     are 0), in one of two formats (bt_fmt):
//       0: bfloat16, hi = bf16(H), lo = bf16(H - hi)      (BF16 / FP8 S)
//       1: float holding tf32 values, hi = H with the 13 low mantissa bits
//          cleared, lo = (H - hi) rounded to tf32, followed by a bf16
//          copy [max(kp,16)][ldb] with rows 0..kp-1 = bf16(H^T) and the
//          rest 0 (the operand of the S_lo H product)      (FP32 S)
//       2: e4m3 bytes, hi = e4m3(H / d), lo = e4m3(16 (H / d - hi)), with d a
//          power of two per 128-row tile of H (the smallest with
//          max|H_tile| / d <= 448); the 2 kp rows are followed by the
//          ntiles FP32 values d                               (FP8 S)
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace symnmf {

constexpr int kTileRows = 128;

// bytes of one MMA copy of H in format fmt, and the tile factors d of format 2
__host__ __device__ inline int bt_n2(int kp) { return kp < 16 ? 16 : kp; }
inline size_t bt_bytes(int fmt, int kp, int64_t ldb) {
  const size_t es = fmt == 1 ? 4 : fmt == 2 ? 1 : 2;
  size_t b = (size_t)2 * kp * ldb * es;
  if (fmt == 1) b += (size_t)bt_n2(kp) * ldb * 2;
  if (fmt == 2) b += (size_t)(ldb / kTileRows) * sizeof(float);
  return b;
}
// format 1: the bf16 copy of H^T after the tf32 hi/lo rows
__host__ __device__ inline uint16_t *bt_b16(void *Bt, int kp, int64_t ldb) {
  return reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(Bt) + (size_t)2 * kp * ldb * 4);
}
__host__ __device__ inline float *bt_deq(void *Bt, int kp, int64_t ldb) {
  return reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(Bt) + (size_t)2 * kp * ldb);
}

constexpr int kRing = 1024;  // device record ring (iterations)

enum Mode : int { MODE_FULL = 0, MODE_ROWS = 1, MODE_BLOCK = 2, MODE_GRAD_ONLY = 3 };

struct DevRecord {
  long long t;
  double f, E, kkt, tr, gram2, sumA;
  int nonfinite;
  int full;
};

// S x H product over a list of 128-row tiles and a list of 128-column tiles.
// Partial slot s holds 128 x kp values at out[(s * 128 + r) * kp + c].
struct ProdArgs {
  const void *S;
  int64_t lds;           // row pitch of S in elements
  int dtype;
  const float *scales;   // FP8 tile scales or nullptr
  int64_t ld_scales;
  int64_t n;
  int k, kp;
  const float *H;        // FP32 master, row-major n x kp (SIMT path)
  const void *Bt;        // hi/lo transposed copy (tensor-core path)
  int bt_fmt;
  int64_t ldb;
  const int *row_list;   // row tile indices (nullptr: all tiles in order)
  int n_rows_list;
  const int *col_list;   // column tile indices (nullptr: all tiles in order)
  int n_cols_list;
  int nsplit;
  float *out;
};

// Partial-sum layout of a product launch: split layout (SIMT: nsplit
// contiguous column shares, slot = split * n_rows + row_pos) or stream-K
// layout (tensor core: CTA b's segment of row position p in slot b + p,
// CTA b covering units [b W / G, (b+1) W / G) of W = n_rows * n_cols).
struct PartLayout {
  int nsplit = 1;
  int skG = 0;      // > 0: stream-K with skG CTAs
  int ncols = 0;
};

struct EpiArgs {
  int64_t n;
  int k, kp, ntiles;
  int mode;              // Mode
  int method;            // symnmf_method
  int update;            // 0: gradient only, no state change
  int store_mu;          // write mu = g (full pass of an SVRG method)
  float eta, eps, alpha, mom;
  const float *H;        // H_t (n x kp)
  float *Hn;             // H_{t+1}
  void *Btn;             // MMA copy of H_{t+1}
  int bt_fmt;
  int64_t ldb;
  float *A, *M, *mu;     // state (n x kp)
  float *gout;           // g (n x kp) or nullptr
  float *gcaller;        // g in caller layout n x k (symnmf_grad) or nullptr
  const float *gram;     // Gram of H_t, kp x kp FP32 (full / rows)
  const float *gramI;    // block mode: H_I^T H_I
  const float *gramJ;    // block mode: H_J^T H_J
  const float *P;        // product partials for rows in list 1
  int nsplit;
  int skG1, ncols1;      // stream-K layout of P (skG1 > 0); block mode: ncols1 = 0, no P
  const int *pos1;       // tile -> position in list 1 (or -1); nullptr in full mode
  int n1;                // length of list 1
  // block mode: list 1 = I, P = S_{I, J\I} H_{J\I}; list 2 = J,
  // Q = S_{J, I\J} H_{I\J}; list 3 = I u J, R = S_{IuJ, K} H_K with K = I n J.
  // S_IJ H_J = P + R on the rows of I, S_JI H_I = Q + R on the rows of J.
  const float *Q;
  int nsplit2;
  int skG2, ncols2;
  const int *pos2;
  int n2;
  const float *R;
  int nsplit3;
  int skG3, ncols3;
  const int *pos3;
  int n3;
  float coef;            // 4 (full/rows) or 2 (block)
  double *slots;         // per tile: [tr, kkt2, sumA, nonfinite]
  float *gram_part;      // per tile kp x kp partial of H_{t+1}^T H_{t+1} (nullptr: skip)
  float rho;             // ADMM penalty
  const float *minv;     // ADMM: (2 Gram_t + rho I)^-1, kp x kp row-major
};

// Cross-tile reduction of one iteration (launch_reduce_iter)
struct ReduceArgs {
  const double *slots;       // per tile [tr, kkt2, sumA, nonfinite] or nullptr
  const float *gram_part;    // per tile Gram partials or nullptr
  int ntiles;
  int k;
  int64_t n;
  double normS2;
  long long t;
  int full;
  const double *gram64_cur;  // Gram of H_t (for ||H_t^T H_t||^2) or nullptr
  double *gram64_next;
  float *gram32_next;
  DevRecord *rec;            // record destination or nullptr
  double *lvl1;              // ceil(ntiles/32) x (4 + kp^2) scratch
  int *counters;             // >= ceil((4 + kp^2)/128) counters, zero between launches
  int kb;                    // restarts along N: Gram entries whose columns lie in
                             // different blocks of kb columns are set to 0 (0: none)
};

constexpr int kSlotStride = 4;

// launchers (return cudaError_t of the launch)
cudaError_t launch_prod_simt(const ProdArgs &a, cudaStream_t s);
// tensor-core product; with epi != nullptr (full row and column lists only)
// the kernel also runs the per-tile epilogue and the cross-tile reduction
cudaError_t launch_step_tc(const ProdArgs &a, const EpiArgs *epi, int *tile_cnt, cudaStream_t s,
                           int num_sms, int *G_out, int *err);
bool tc_supported(int dtype, int kp);
// TMA descriptor of a 2-D row-major array: inner extent, outer extent, row
// pitch in bytes, box; 128-byte (or 64-byte) swizzle, zero fill out of
// bounds
bool make_map_2d(CUtensorMap *m, const void *base, CUtensorMapDataType dt, uint64_t inner,
                 uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                 int swizzle_bytes = 128);
// ADMM (appendix, Family 6): minv = (2 G + rho I)^-1 for the FP64 Gram G
// (kp x kp, entries past k ignored; minv is the identity there).  Launched
// as a programmatic dependent of the preceding kernel.
cudaError_t launch_admm_minv(const double *gram64, int k, int kp, double rho, float *minv,
                             cudaStream_t s);
cudaError_t launch_epilogue(const EpiArgs &a, cudaStream_t s);
// per-tile Bt copy and Gram partial of H (init / teacher forcing)
cudaError_t launch_prepare_tiles(const float *H, int64_t n, int k, int kp, void *Bt, int bt_fmt,
                                 int64_t ldb, float *gram_part, cudaStream_t s);
// fixed-order FP64 reduction of the per-tile slots and Gram partials of an
// iteration: Gram of the next iterate (FP64 and FP32) and the record
cudaError_t launch_reduce_iter(const ReduceArgs &a, int kp, cudaStream_t s);
// Gram of a subset of tiles (lists of tile indices) -> FP32 kp x kp, two lists
cudaError_t launch_gram_subset(const float *gram_part, int kp, const int *list1, int n1,
                               const int *list2, int n2, float *out1, float *out2, int kb,
                               cudaStream_t s);
cudaError_t launch_norm_s2(const void *S, int64_t n, int64_t lds, int dtype, const float *scales,
                           int64_t ld_scales, double *partials, int nparts, double *out,
                           cudaStream_t s);
// n x k (pitch k) <-> n x kp (pitch kp, pads zeroed)
cudaError_t launch_pack(const float *src, float *dst, int64_t n, int k, int kp, cudaStream_t s);
cudaError_t launch_unpack(const float *src, float *dst, int64_t n, int k, int kp, cudaStream_t s);
// lower median of g^2 over the n x kw entries in columns c0 .. c0 + kw - 1
// (radix select on the FP32 bit patterns); result in *out (device)
cudaError_t launch_median_g2(const float *g, int64_t n, int c0, int kw, int kp, unsigned *hist,
                             unsigned *sel, float *out, cudaStream_t s);
// Piecewise reset of columns c0 .. c0 + kw - 1: A = c * max(g^2, med);
// per-tile sum of those entries of A into slots[.][2]
cudaError_t launch_reset(float *A, const float *g, const float *med, float c, int64_t n, int c0,
                         int kw, int kp, double *slots, cudaStream_t s);
// per-tile power-of-two scaled E4M3 codes of a rows x cols FP32 / BF16 matrix
cudaError_t launch_quantize_fp8(const void *src, int src_dtype, int64_t rows, int64_t cols,
                                int64_t ld_src, uint8_t *q, int64_t ldq, float *scales,
                                int64_t ld_scales, double *tile_sumsq, cudaStream_t s);
cudaError_t launch_sum_slot(const double *slots, int ntiles, int which, double *out,
                            cudaStream_t s);

// Dependence matrix S = |D^-1/2 Y^T Y D^-1/2| (Sec. 3), k_dep.cu; err is a
// device int the kernels set on a bounded-wait timeout
cudaError_t launch_dependence(const float *Y, int64_t T, int64_t n, int64_t ldy, int center,
                              int out, void *S, int64_t lds, float *scales, int64_t ld_scales,
                              double *normS2, int *err, cudaStream_t s,
                              bool exact_norm = false);

// Spherical K-means (Sec. 6): the kernels around the two product passes of
// one Lloyd iteration (k_kmeans.cu)
struct KmArgs {
  int64_t n;
  int K, ntiles;
  const float *P;        // product partials (layout: nsplit / skG / ncols)
  int nsplit, skG, ncols;
  float *C;              // centroid sums, n x kp (the next operand)
  double *colsq;         // per tile kp FP64 column sums of squares of C
  float *inv_norm;       // kp: 1 / ||c_k|| (0 for an empty cluster)
  const double *rn;      // ||s_i||
  const int *labels_in;
  int *labels_out;
  double *slots;         // per tile [sum (1 - cos), changed]
  double *out;           // [J, changed]
};
cudaError_t launch_row_norms(const void *S, int64_t n, int64_t lds, int dtype, const float *scales,
                             int64_t ld_scales, double *rn, cudaStream_t s);
// operand D^-1 B (rows_alloc x kp): 1 / ||s_i|| in column labels[i]
cudaError_t launch_km_operand(const int *labels, const double *rn, int64_t n, int kp, float *H,
                              int64_t rows_alloc, cudaStream_t s);
// C from the partials of S (D^-1 B), its column norms
cudaError_t launch_km_centroids(const KmArgs &a, int kp, cudaStream_t s);
// labels from the partials of S C, J and the changed count into out
cudaError_t launch_km_assign(const KmArgs &a, int kp, cudaStream_t s);

}  // namespace symnmf
