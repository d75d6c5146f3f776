// Host runtime of libsymnmf: handle lifecycle, the per-iteration launch
// sequence, the scalar controller (Sec. 4.1 AND rule; Piecewise reset and
// AdaptGrow growth control of Sec. 5.1 and the appendix), counter-based
// sampling of row blocks, and checkpoints.  Every arithmetic step of the
// solver runs in the kernels; this file only orders launches and makes the
// scalar decisions at check iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "../../include/symnmf.h"
#include "restart_stats.h"
#include "symnmf_internal.h"

using namespace symnmf;

namespace {

constexpr int kStages = 8;          // pinned/device staging slots for sampled lists
constexpr int kListArrays = 9;      // ntiles-long int arrays per staging slot
constexpr size_t kTraceCap = 1u << 20;
constexpr uint64_t kMagic = 0x31764D4E4D59534EULL;  // "NSYMNMv1"

int pad_k(int k) { return k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : 64; }
size_t esize(int dtype) { return dtype == SYMNMF_F32 ? 4 : dtype == SYMNMF_BF16 ? 2 : 1; }

}  // namespace

struct symnmf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  const void *S = nullptr;
  int64_t n = 0, lds = 0;
  int k = 0, kp = 0, dtype = 0;
  const float *scales = nullptr;
  int64_t ld_scales = 0;
  double normS2 = NAN;
  int ntiles = 0;
  int64_t ldb = 0;
  int num_sms = 0;
  int impl_req = 0;   // 0 auto, 1 simt, 2 tc
  bool tc_layout_ok = false;
  // owned device memory
  float *H[2] = {nullptr, nullptr};
  void *Bt[2] = {nullptr, nullptr};
  int bt_fmt = 0;          // 0: bf16 hi/lo, 1: tf32 hi/lo in float, 2: e4m3 pieces
  float *gram_part[2] = {nullptr, nullptr};
  double *gram64[2] = {nullptr, nullptr};
  float *gram32[2] = {nullptr, nullptr};
  int cur = 0;
  float *A = nullptr, *M = nullptr, *mu = nullptr, *g = nullptr, *tmp = nullptr;
  float *P = nullptr, *Q = nullptr, *R = nullptr;  // product partials
  int64_t pq_cap_tiles = 0;
  double *slots = nullptr, *chunk = nullptr;
  int nchunks = 1;
  float *gramI = nullptr, *gramJ = nullptr;
  float *minv = nullptr;    // ADMM: (2 Gram_t + rho I)^-1
  int *dlists = nullptr;    // kStages x kListArrays x ntiles
  int *hlists = nullptr;    // pinned mirror
  cudaEvent_t stage_ev[kStages] = {};
  bool stage_used[kStages] = {};
  DevRecord *ring = nullptr;  // kRing + 1 (last = scratch)
  DevRecord *hring = nullptr; // pinned
  unsigned *hist = nullptr, *sel = nullptr;
  float *dmed = nullptr;
  double *dsum = nullptr, *hsum = nullptr;  // dsum[0..3], pinned hsum
  float *hmed = nullptr;
  double *norm_parts = nullptr;
  int n_norm_parts = 0;
  int *dev_err = nullptr;     // device error word (bounded-wait timeouts)
  int *counters = nullptr;    // reduction last-arriver counters
  int *tile_cnt = nullptr;    // per-tile stream-K arrival counters
  double *lvl1 = nullptr;     // reduction level-1 sums
  int ntc = 0;                // tile chunks of 32
  int *host_err = nullptr;    // pinned mirror
  // host state
  symnmf_ctrl ctrl{};
  std::deque<symnmf_record> trace;
  int64_t copied_upto = 0;
  std::string err;
  bool bad = false;
  int64_t last_check = -1;
  symnmf_record last_check_rec{};
  // product-kernel timing
  bool profiling = false;
  std::vector<cudaEvent_t> prof_ev;   // pairs
  size_t prof_used = 0;                // events used (2 per launch)
  double prof_bytes = 0.0;
  int64_t prof_kernels = 0;  // kernels launched by the solver loop while profiling
  int ctas = 0;              // CTA cap of the tensor-core launches (0: all SMs)
  int restarts = 1;          // independent restarts concatenated along N
  // per-restart checks (restarts > 1): AND rule state and the last check
  struct RestartCtl {
    double E0 = NAN, E_prev = NAN;
    bool have_prev = false;
    // Piecewise AdaGrad's reset state, per restart
    bool cooldown = false, resets_enabled = true;
    int resets = 0;
    double E_at_reset = NAN, sumA_post = 0.0;
  };
  std::vector<RestartCtl> rctl;
  std::vector<double> rE, rkkt;
  std::vector<int32_t> rconv;
  double *rs_part = nullptr, *rs_out = nullptr, *rs_host = nullptr;  // host: pinned
  // spherical K-means scratch, allocated by the first symnmf_spkmeans
  double *km_rn = nullptr;      // ||s_i||
  int *km_lab = nullptr;        // two label buffers of n
  double *km_colsq = nullptr;   // ntiles x kp
  float *km_inv = nullptr;      // kp
  double *km_slots = nullptr;   // ntiles x 2
  double *km_out = nullptr;     // [J, changed]
  double *km_hout = nullptr;    // pinned mirror
};

namespace {

int fail(symnmf_t h, int status, const std::string &msg) {
  if (h) {
    h->err = msg;
    if (status == SYMNMF_ERR_CUDA || status == SYMNMF_ERR_TIMEOUT ||
        status == SYMNMF_ERR_NONFINITE)
      h->bad = true;
  }
  return status;
}

int cuda_fail(symnmf_t h, cudaError_t e, const char *where) {
  return fail(h, SYMNMF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                     \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);           \
  } while (0)

void reset_ctrl(symnmf_ctrl *c) {
  std::memset(c, 0, sizeof(*c));
  c->t = 0;
  c->E0 = NAN;
  c->E_prev = NAN;
  c->phi = 1.0;
  c->E_at_reset = NAN;
  c->resets_enabled = 1;
}

template <class T>
cudaError_t dalloc(T **p, size_t count) {
  cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(1, count) * sizeof(T));
  if (e == cudaSuccess) e = cudaMemset(*p, 0, std::max<size_t>(1, count) * sizeof(T));
  return e;
}

void free_all(symnmf_t h) {
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->H[i]);
    cudaFree(h->Bt[i]);
    cudaFree(h->gram_part[i]);
    cudaFree(h->gram64[i]);
    cudaFree(h->gram32[i]);
  }
  for (void *p : {(void *)h->A, (void *)h->M, (void *)h->mu, (void *)h->g, (void *)h->tmp,
                  (void *)h->P, (void *)h->Q, (void *)h->R, (void *)h->slots, (void *)h->chunk,
                  (void *)h->gramI, (void *)h->gramJ, (void *)h->minv, (void *)h->dlists, (void *)h->ring,
                  (void *)h->hist, (void *)h->sel, (void *)h->dmed, (void *)h->dsum,
                  (void *)h->norm_parts, (void *)h->dev_err, (void *)h->counters, (void *)h->tile_cnt,
                  (void *)h->lvl1, (void *)h->km_rn, (void *)h->km_lab, (void *)h->km_colsq,
                  (void *)h->km_inv, (void *)h->km_slots, (void *)h->km_out, (void *)h->rs_part,
                  (void *)h->rs_out})
    cudaFree(p);
  for (void *p : {(void *)h->hlists, (void *)h->hring, (void *)h->hsum, (void *)h->hmed,
                  (void *)h->host_err, (void *)h->km_hout, (void *)h->rs_host})
    if (p) cudaFreeHost(p);
  for (int i = 0; i < kStages; ++i)
    if (h->stage_ev[i]) cudaEventDestroy(h->stage_ev[i]);
  for (cudaEvent_t ev : h->prof_ev) cudaEventDestroy(ev);
}

cudaError_t prof_event(symnmf_t h, cudaEvent_t *ev) {
  if (h->prof_used >= h->prof_ev.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    h->prof_ev.push_back(e);
  }
  *ev = h->prof_ev[h->prof_used++];
  return cudaSuccess;
}

bool use_tc(symnmf_t h) {
  if (h->impl_req == 1) return false;
  return h->tc_layout_ok && tc_supported(h->dtype, h->kp);
}

int compute_norm(symnmf_t h) {
  CK(launch_norm_s2(h->S, h->n, h->lds, h->dtype, h->scales, h->ld_scales, h->norm_parts,
                    h->n_norm_parts, h->dsum, h->stream));
  CK(cudaMemcpyAsync(h->hsum, h->dsum, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->normS2 = h->hsum[0];
  return SYMNMF_OK;
}

ReduceArgs reduce_args(symnmf_t h, const double *slots, const float *gram_part, long long t,
                       int full) {
  ReduceArgs r{};
  r.slots = slots;
  r.gram_part = gram_part;
  r.ntiles = h->ntiles;
  r.k = h->k;
  r.n = h->n;
  // R restarts: f and E of the concatenated problem, sum_r f_r and its
  // mean E (the Gram is block diagonal, so the cross terms vanish)
  r.normS2 = h->normS2 * h->restarts;
  r.kb = h->restarts > 1 ? h->k / h->restarts : 0;
  r.t = t;
  r.full = full;
  r.gram64_cur = h->gram64[h->cur];
  r.gram64_next = h->gram64[1 - h->cur];
  r.gram32_next = h->gram32[1 - h->cur];
  r.rec = h->ring + (t >= 0 ? (t % kRing) : kRing);
  r.lvl1 = h->lvl1;
  r.counters = h->counters;
  return r;
}

// Bt copy, per-tile Gram partials and the reduced Gram of H[cur]
int refresh_derived(symnmf_t h) {
  const int c = h->cur;
  CK(launch_prepare_tiles(h->H[c], h->n, h->k, h->kp, h->Bt[c], h->bt_fmt, h->ldb,
                          h->gram_part[c], h->stream));
  ReduceArgs r = reduce_args(h, nullptr, h->gram_part[c], -1, 0);
  r.gram64_cur = nullptr;
  r.gram64_next = h->gram64[c];
  r.gram32_next = h->gram32[c];
  r.rec = nullptr;
  CK(launch_reduce_iter(r, h->kp, h->stream));
  return SYMNMF_OK;
}

// --------------------------------------------------------------- sampling
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

void sample(uint64_t seed, int64_t t, int stream, int64_t nb, int64_t m, std::vector<int64_t> &out) {
  m = std::min(m, nb);
  std::vector<int64_t> perm(nb);
  for (int64_t i = 0; i < nb; ++i) perm[i] = i;
  const uint64_t st = seed * kGamma + (uint64_t)t * 0xBF58476D1CE4E5B9ULL +
                      (uint64_t)stream * 0x94D049BB133111EBULL;
  for (int64_t d = 0; d < m; ++d) {
    const uint64_t u = mix64(st + (uint64_t)(d + 1) * kGamma);
    const int64_t j = d + (int64_t)(u % (uint64_t)(nb - d));
    std::swap(perm[d], perm[j]);
  }
  out.assign(perm.begin(), perm.begin() + m);
  std::sort(out.begin(), out.end());
}

int64_t sample_count(double frac, int64_t n, int64_t block_rows) {
  const int64_t nb = (n + block_rows - 1) / block_rows;
  const int64_t rows = (int64_t)std::ceil(frac * (double)n);
  return std::min(nb, (rows + block_rows - 1) / block_rows);
}

// ------------------------------------------------------------- controller
struct CheckOut {
  bool converged = false, reset = false, grow = false;
  double ratio = NAN;
  double median = NAN;  // median(g_t^2) when the check evaluated it
};

template <class MedianFn>
void ctrl_check(symnmf_ctrl *c, const symnmf_hparams *hp, int64_t n, int64_t t, double E,
                double kkt, double sumA, MedianFn median, CheckOut *o) {
  if (t == 0 || !(c->E0 == c->E0)) c->E0 = E;
  const double tau_g = hp->tau_g > 0 ? hp->tau_g : 1e-4 * std::max(1.0, 1e4 / (double)n);
  const double ratio = c->have_prev ? (c->E_prev - E) / c->E0 : NAN;
  const bool stag = c->have_prev && t >= hp->warmup && ratio < hp->tau_stag;
  o->ratio = ratio;
  if (E < hp->tau_E && kkt < tau_g && stag) {
    c->converged = 1;
    o->converged = true;
    return;
  }
  if (hp->method == SYMNMF_PIECEWISE_ADAGRAD) {
    if (c->cooldown && sumA >= 2.0 * c->sumA_post) c->cooldown = 0;
    if (!c->cooldown && c->resets_enabled && stag && kkt > hp->c_r * tau_g) {
      const double med = median();
      o->median = med;
      if (med > hp->eps) {
        if (c->resets > 0 && !(E < c->E_at_reset - hp->tau_stag * c->E0)) {
          c->resets_enabled = 0;
        } else {
          o->reset = true;
          c->cooldown = 1;
          c->E_at_reset = E;
          c->resets += 1;
        }
      }
    }
  }
  if (hp->method == SYMNMF_BLOCK_SVRG_ADAPTGROW) {
    c->stag_count = stag ? c->stag_count + 1 : 0;
    if (c->stag_count >= 3 && kkt > hp->growth_kkt_mult * tau_g && c->phi < 1.0) {
      c->phi = std::min(2.0 * c->phi, 1.0);
      c->stag_count = 0;
      o->grow = true;
    }
  }
  c->E_prev = E;
  c->have_prev = 1;
}

int validate_hp(const symnmf_hparams *hp) {
  if (!hp) return SYMNMF_ERR_INVALID;
  if (hp->method < 0 || hp->method > SYMNMF_ADMM) return SYMNMF_ERR_INVALID;
  if (hp->method == SYMNMF_ADMM && !(hp->rho > 0)) return SYMNMF_ERR_INVALID;
  if (hp->check_interval < 1 || hp->snapshot_period < 1 || hp->warmup < 0)
    return SYMNMF_ERR_INVALID;
  if (hp->block_rows < kTileRows || hp->block_rows % kTileRows) return SYMNMF_ERR_INVALID;
  if (!(hp->eta > 0) || !(hp->eps >= 0)) return SYMNMF_ERR_INVALID;
  if (hp->method == SYMNMF_ROW_SVRG && !(hp->row_frac > 0 && hp->row_frac <= 1))
    return SYMNMF_ERR_INVALID;
  if (hp->method == SYMNMF_BLOCK_SVRG_ADAPTGROW && !(hp->phi0 > 0 && hp->phi0 <= 1))
    return SYMNMF_ERR_INVALID;
  return SYMNMF_OK;
}

// ------------------------------------------------------------ iteration
int stage_slot(symnmf_t h, int64_t t, int **hl, int **dl) {
  const int s = (int)(t % kStages);
  if (h->stage_used[s]) CK(cudaEventSynchronize(h->stage_ev[s]));
  *hl = h->hlists + (size_t)s * kListArrays * h->ntiles;
  *dl = h->dlists + (size_t)s * kListArrays * h->ntiles;
  return SYMNMF_OK;
}

int upload_slot(symnmf_t h, int64_t t, int *hl, int *dl) {
  const int s = (int)(t % kStages);
  CK(cudaMemcpyAsync(dl, hl, sizeof(int) * kListArrays * h->ntiles, cudaMemcpyHostToDevice,
                      h->stream));
  CK(cudaEventRecord(h->stage_ev[s], h->stream));
  h->stage_used[s] = true;
  return SYMNMF_OK;
}

// tile list of the sampled blocks
void blocks_to_tiles(symnmf_t h, const std::vector<int64_t> &blocks, int64_t block_rows,
                     std::vector<int> &tiles) {
  const int bt = (int)(block_rows / kTileRows);
  tiles.clear();
  for (int64_t b : blocks)
    for (int i = 0; i < bt; ++i) {
      const int64_t tt = b * bt + i;
      if (tt < h->ntiles) tiles.push_back((int)tt);
    }
}

void count_kernels(symnmf_t h, int64_t n) {
  if (h->profiling) h->prof_kernels += n;
}

int prod(symnmf_t h, const int *row_list, int n_rows, const int *col_list, int n_cols, float *out,
         PartLayout *lay, const EpiArgs *fuse = nullptr) {
  ProdArgs a{};
  a.S = h->S;
  a.lds = h->lds;
  a.dtype = h->dtype;
  a.scales = h->scales;
  a.ld_scales = h->ld_scales;
  a.n = h->n;
  a.k = h->k;
  a.kp = h->kp;
  a.H = h->H[h->cur];
  a.Bt = h->Bt[h->cur];
  a.bt_fmt = h->bt_fmt;
  a.ldb = h->ldb;
  a.row_list = row_list;
  a.n_rows_list = n_rows;
  a.col_list = col_list;
  a.n_cols_list = n_cols;
  a.out = out;
  const int target = 3 * h->num_sms;
  int ns = (target + n_rows - 1) / std::max(1, n_rows);
  ns = std::max(1, std::min(ns, std::min(64, n_cols)));
  if ((int64_t)ns * n_rows > h->pq_cap_tiles) ns = (int)std::max<int64_t>(1, h->pq_cap_tiles / n_rows);
  a.nsplit = ns;
  lay->nsplit = ns;
  lay->skG = 0;
  lay->ncols = n_cols;
  const bool tc = use_tc(h);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->profiling) {
    CK(prof_event(h, &e0));
    CK(prof_event(h, &e1));
    CK(cudaEventRecord(e0, h->stream));
  }
  cudaError_t e;
  if (tc) {
    a.nsplit = 1;
    lay->nsplit = 1;
    const int sms = (h->ctas > 0 && h->ctas < h->num_sms) ? h->ctas : h->num_sms;
    e = launch_step_tc(a, fuse, h->tile_cnt, h->stream, sms, &lay->skG, h->dev_err);
  } else {
    e = launch_prod_simt(a, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "product kernel");
  count_kernels(h, 1);
  if (h->profiling) {
    CK(cudaEventRecord(e1, h->stream));
    const double rows = std::min<double>((double)n_rows * kTileRows, (double)h->n);
    const double cols = std::min<double>((double)n_cols * kTileRows, (double)h->n);
    h->prof_bytes += rows * cols * (double)esize(h->dtype);
  }
  return SYMNMF_OK;
}

EpiArgs base_epi(symnmf_t h, const symnmf_hparams *hp) {
  EpiArgs e{};
  e.n = h->n;
  e.k = h->k;
  e.kp = h->kp;
  e.ntiles = h->ntiles;
  e.method = hp ? hp->method : 0;
  e.eta = hp ? (float)hp->eta : 0.f;
  e.eps = hp ? (float)hp->eps : 0.f;
  e.alpha = hp ? (float)hp->alpha : 0.f;
  e.mom = hp ? (float)hp->mu : 0.f;
  e.H = h->H[h->cur];
  e.ldb = h->ldb;
  e.A = h->A;
  e.M = h->M;
  e.mu = h->mu;
  e.coef = 4.f;
  e.rho = hp ? (float)hp->rho : 0.f;
  e.minv = h->minv;
  return e;
}

bool is_full(symnmf_t h, const symnmf_hparams *hp, int64_t t) {
  if (hp->method == SYMNMF_ROW_SVRG)
    return hp->row_frac >= 1.0 || t % hp->snapshot_period == 0 || t % hp->check_interval == 0;
  if (hp->method == SYMNMF_BLOCK_SVRG_ADAPTGROW)
    return h->ctrl.phi >= 1.0 || t % hp->snapshot_period == 0 || t % hp->check_interval == 0;
  return true;
}

// need_g: also write the gradient buffer g (read by the Piecewise reset at
// checks and by symnmf_get_buffer after a call)
int run_iteration(symnmf_t h, const symnmf_hparams *hp, int64_t t, bool need_g) {
  const int cur = h->cur, nxt = 1 - cur;
  const bool full = is_full(h, hp, t);
  EpiArgs e = base_epi(h, hp);
  e.Hn = h->H[nxt];
  e.Btn = h->Bt[nxt];
  e.bt_fmt = h->bt_fmt;
  e.gram_part = h->gram_part[nxt];
  e.slots = h->slots;
  e.gout = need_g ? h->g : nullptr;
  e.update = 1;
  int rc;
  bool fused_done = false;
  if (hp->method == SYMNMF_ADMM) {
    // (2 W^T W + rho I)^-1 from the FP64 Gram of W = H_t (appendix, Family 6)
    CK(launch_admm_minv(h->gram64[cur], h->k, h->kp, hp->rho, h->minv, h->stream));
    count_kernels(h, 1);
  }
  if (full) {
    e.mode = MODE_FULL;
    e.gram = h->gram32[cur];
    e.P = h->P;
    e.n1 = h->ntiles;
    e.store_mu = (hp->method == SYMNMF_ROW_SVRG || hp->method == SYMNMF_BLOCK_SVRG_ADAPTGROW);
    PartLayout ly;
    if (use_tc(h)) {
      // one fused launch: product and per-tile epilogue
      if ((rc = prod(h, nullptr, h->ntiles, nullptr, h->ntiles, h->P, &ly, &e))) return rc;
      fused_done = true;
    } else {
      if ((rc = prod(h, nullptr, h->ntiles, nullptr, h->ntiles, h->P, &ly))) return rc;
      e.nsplit = ly.nsplit;
      e.skG1 = ly.skG;
      e.ncols1 = ly.ncols;
    }
  } else {
    int *hl = nullptr, *dl = nullptr;
    if ((rc = stage_slot(h, t, &hl, &dl))) return rc;
    const int nt = h->ntiles;
    int *hI = hl, *hJ = hl + nt, *hposI = hl + 2 * nt, *hposJ = hl + 3 * nt;
    const int64_t br = hp->block_rows;
    const int64_t nb = (h->n + br - 1) / br;
    std::vector<int64_t> bI, bJ;
    std::vector<int> tI, tJ;
    for (int i = 0; i < nt; ++i) hposI[i] = hposJ[i] = -1;
    if (hp->method == SYMNMF_ROW_SVRG) {
      sample(hp->seed, t, 0, nb, sample_count(hp->row_frac, h->n, br), bI);
    } else {
      const int64_t m = sample_count(std::sqrt(h->ctrl.phi), h->n, br);
      sample(hp->seed, t, 1, nb, m, bI);
      sample(hp->seed, t, 2, nb, m, bJ);
    }
    blocks_to_tiles(h, bI, br, tI);
    blocks_to_tiles(h, bJ, br, tJ);
    for (size_t i = 0; i < tI.size(); ++i) {
      hI[i] = tI[i];
      hposI[tI[i]] = (int)i;
    }
    for (size_t i = 0; i < tJ.size(); ++i) {
      hJ[i] = tJ[i];
      hposJ[tJ[i]] = (int)i;
    }
    // Block-SVRG: the rows of I need S_IJ, the rows of J need S_JI, and S
    // is symmetric, so every tile position is read once.  With K = I n J
    // the positions split into (I u J) x K, I x (J \ I) and J x (I \ J):
    // alpha, beta and gamma.  S_IJ H_J = alpha + beta on the rows of I and
    // S_JI H_I = alpha + gamma on the rows of J.
    int *hU = hl + 4 * nt, *hposU = hl + 5 * nt, *hK = hl + 6 * nt, *hJmI = hl + 7 * nt,
        *hImJ = hl + 8 * nt;
    int nU = 0, nK = 0, nJmI = 0, nImJ = 0;
    if (hp->method == SYMNMF_BLOCK_SVRG_ADAPTGROW) {
      for (int i = 0; i < nt; ++i) hposU[i] = -1;
      for (int x : tI) {
        hposU[x] = nU;
        hU[nU++] = x;
        if (hposJ[x] >= 0) hK[nK++] = x;
        else hImJ[nImJ++] = x;
      }
      for (int x : tJ)
        if (hposI[x] < 0) {
          hposU[x] = nU;
          hU[nU++] = x;
          hJmI[nJmI++] = x;
        }
    }
    if ((rc = upload_slot(h, t, hl, dl))) return rc;
    int *dI = dl, *dJ = dl + nt, *dposI = dl + 2 * nt, *dposJ = dl + 3 * nt;
    int *dU = dl + 4 * nt, *dposU = dl + 5 * nt, *dK = dl + 6 * nt, *dJmI = dl + 7 * nt,
        *dImJ = dl + 8 * nt;
    if (hp->method == SYMNMF_ROW_SVRG) {
      PartLayout ly;
      if ((rc = prod(h, dI, (int)tI.size(), nullptr, h->ntiles, h->P, &ly))) return rc;
      e.mode = MODE_ROWS;
      e.gram = h->gram32[cur];
      e.P = h->P;
      e.nsplit = ly.nsplit;
      e.skG1 = ly.skG;
      e.ncols1 = ly.ncols;
      e.pos1 = dposI;
      e.n1 = (int)tI.size();
    } else {
      CK(launch_gram_subset(h->gram_part[cur], h->kp, dI, (int)tI.size(), dJ, (int)tJ.size(),
                            h->gramI, h->gramJ, h->restarts > 1 ? h->k / h->restarts : 0,
                            h->stream));
      count_kernels(h, 1);
      // an empty list contributes zero (ncols = 0 in the layout)
      PartLayout l1{}, l2{}, l3{};
      if (nJmI > 0 && (rc = prod(h, dI, (int)tI.size(), dJmI, nJmI, h->P, &l1))) return rc;
      if (nImJ > 0 && (rc = prod(h, dJ, (int)tJ.size(), dImJ, nImJ, h->Q, &l2))) return rc;
      if (nK > 0 && (rc = prod(h, dU, nU, dK, nK, h->R, &l3))) return rc;
      e.mode = MODE_BLOCK;
      e.coef = 2.f;
      e.gramI = h->gramI;
      e.gramJ = h->gramJ;
      e.P = h->P;
      e.nsplit = l1.nsplit;
      e.skG1 = l1.skG;
      e.ncols1 = l1.ncols;
      e.pos1 = dposI;
      e.n1 = (int)tI.size();
      e.Q = h->Q;
      e.nsplit2 = l2.nsplit;
      e.skG2 = l2.skG;
      e.ncols2 = l2.ncols;
      e.pos2 = dposJ;
      e.n2 = (int)tJ.size();
      e.R = h->R;
      e.nsplit3 = l3.nsplit;
      e.skG3 = l3.skG;
      e.ncols3 = l3.ncols;
      e.pos3 = dposU;
      e.n3 = nU;
    }
  }
  if (!fused_done) CK(launch_epilogue(e, h->stream));
  CK(launch_reduce_iter(reduce_args(h, h->slots, h->gram_part[nxt], t, full ? 1 : 0), h->kp,
                        h->stream));
  count_kernels(h, fused_done ? 1 : 2);
  h->cur = nxt;
  return SYMNMF_OK;
}

symnmf_record to_record(const DevRecord &d, double phi) {
  symnmf_record r{};
  r.t = d.t;
  r.full = d.full;
  r.f = d.full ? d.f : NAN;
  r.E = d.full ? d.E : NAN;
  r.kkt = d.full ? d.kkt : NAN;
  r.sumA = d.sumA;
  r.nonfinite = d.nonfinite;
  r.stag_ratio = NAN;
  r.phi = phi;
  r.median_g2 = NAN;
  return r;
}

// enqueue the copy of device records [h->copied_upto, upto) and of the
// device error word to the host (no wait)
int enqueue_records(symnmf_t h, int64_t upto) {
  const int64_t from = h->copied_upto;
  if (upto <= from) return SYMNMF_OK;
  int64_t a = from;
  while (a < upto) {
    const int64_t s = a % kRing;
    const int64_t len = std::min<int64_t>(upto - a, kRing - s);
    CK(cudaMemcpyAsync(h->hring + s, h->ring + s, sizeof(DevRecord) * len,
                       cudaMemcpyDeviceToHost, h->stream));
    a += len;
  }
  CK(cudaMemcpyAsync(h->host_err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  return SYMNMF_OK;
}

// wait for enqueue_records and append the records to the host trace
int finish_records(symnmf_t h, int64_t upto, const std::vector<double> &phis) {
  const int64_t from = h->copied_upto;
  if (upto <= from) return SYMNMF_OK;
  CK(cudaStreamSynchronize(h->stream));
  if (h->host_err[0] != 0)
    return fail(h, SYMNMF_ERR_TIMEOUT,
                "a bounded device wait gave up (code " + std::to_string(h->host_err[0]) + ")");
  for (int64_t t = from; t < upto; ++t) {
    const double phi = (t - from) < (int64_t)phis.size() ? phis[t - from] : h->ctrl.phi;
    h->trace.push_back(to_record(h->hring[t % kRing], phi));
    if (h->trace.size() > kTraceCap) h->trace.pop_front();
  }
  h->copied_upto = upto;
  return SYMNMF_OK;
}

// copy device records [h->copied_upto, upto) into the host trace
int sync_records(symnmf_t h, int64_t upto, const std::vector<double> &phis) {
  int rc = enqueue_records(h, upto);
  if (rc) return rc;
  return finish_records(h, upto, phis);
}

// lower median of g^2 over columns c0 .. c0 + kw - 1 (left on the device
// in dmed for reset_columns)
int median_g2(symnmf_t h, int c0, int kw, double *out) {
  CK(launch_median_g2(h->g, h->n, c0, kw, h->kp, h->hist, h->sel, h->dmed, h->stream));
  count_kernels(h, 7);  // selection init + 3 x (histogram, select)
  CK(cudaMemcpyAsync(h->hmed, h->dmed, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = (double)h->hmed[0];
  return SYMNMF_OK;
}

// Piecewise reset of columns c0 .. c0 + kw - 1 with the median in dmed;
// *sumA_post = the sum of the reset entries
int reset_columns(symnmf_t h, const symnmf_hparams *hp, int c0, int kw, double *sumA_post) {
  CK(launch_reset(h->A, h->g, h->dmed, (float)hp->c, h->n, c0, kw, h->kp, h->slots, h->stream));
  CK(launch_sum_slot(h->slots, h->ntiles, 2, h->dsum, h->stream));
  count_kernels(h, 2);
  CK(cudaMemcpyAsync(h->hsum, h->dsum, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *sumA_post = h->hsum[0];
  return SYMNMF_OK;
}

int check_handle(symnmf_t h) {
  if (!h) return SYMNMF_ERR_INVALID;
  if (h->bad) return fail(h, SYMNMF_ERR_STATE, "handle is in an error state: " + h->err);
  if (h->dtype == SYMNMF_FP8E4M3 && !h->scales)
    return fail(h, SYMNMF_ERR_INVALID, "FP8 storage needs symnmf_set_tile_scales first");
  return SYMNMF_OK;
}

void fill_stats(symnmf_t h, symnmf_stats *st) {
  if (!st) return;
  std::memset(st, 0, sizeof(*st));
  st->iter = h->ctrl.t;
  st->last_check = h->last_check;
  st->f = h->last_check_rec.f;
  st->E = h->last_check_rec.E;
  st->kkt = h->last_check_rec.kkt;
  st->stag_ratio = h->last_check_rec.stag_ratio;
  st->phi = h->ctrl.phi;
  st->converged = h->ctrl.converged;
  st->resets = h->ctrl.resets;
}

// first half of an iteration: launch it and, when its records are due on
// the host (a check, or a ring about to wrap), enqueue their copy
int iterate_launch(symnmf_t h, const symnmf_hparams *hp, std::vector<double> &phis, bool last) {
  const int64_t t = h->ctrl.t;
  if (t == 0 && h->copied_upto == 0 && h->trace.empty())
    h->ctrl.phi = hp->method == SYMNMF_BLOCK_SVRG_ADAPTGROW ? hp->phi0 : 1.0;
  phis.push_back(h->ctrl.phi);
  int rc = run_iteration(h, hp, t, last || t % hp->check_interval == 0);
  if (rc) return rc;
  if (t % hp->check_interval == 0 || t + 1 - h->copied_upto >= kRing / 2)
    return enqueue_records(h, t + 1);
  return SYMNMF_OK;
}

// second half: the check (Eq. 11 and the method's control); returns OK,
// CONVERGED or an error
void reset_restart_checks(symnmf_t h) {
  h->rctl.assign(h->restarts, symnmf_ctx::RestartCtl{});
  h->rE.assign(h->restarts, NAN);
  h->rkkt.assign(h->restarts, NAN);
  h->rconv.assign(h->restarts, 0);
}

// Per-restart checks at check t (restarts > 1): H_t is in the other H
// buffer (the step has flipped cur) and g holds its gradient; the Gram of
// H_t is block diagonal.  f_r = ||S||^2 - ||Gram_rr||^2 + sum(H_r .* g_r) / 2,
// E_r = f_r / ||S||^2, kkt_r = ||grad_proj,r|| / (n kb).  Sets *any when a
// restart meets Eq. 11 (E0 and the stagnation test per restart, as for a
// handle of its own).  Piecewise AdaGrad (appendix, Family 3) decides and
// applies its reset per restart as ctrl_check does for a handle, on the
// restart's E_r, kkt_r, sum(A_r) and the median of g_r^2 over its own n kb
// entries; no restart resets at a check where the handle stops.
int restart_checks(symnmf_t h, const symnmf_hparams *hp, int64_t t, bool stopping, bool *any,
                   bool *any_reset) {
  *any = false;
  *any_reset = false;
  const int R = h->restarts, kp = h->kp, kb = h->k / R;
  const int prev = 1 - h->cur;
  constexpr int Q = kRestartSums;
  CK(launch_restart_stats(h->H[prev], h->g, h->A, h->n, h->k, kp, R, h->rs_part, h->rs_out,
                          h->stream));
  CK(cudaMemcpyAsync(h->rs_host, h->rs_out, sizeof(double) * Q * R, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(h->rs_host + Q * R, h->gram64[prev], sizeof(double) * kp * kp,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  count_kernels(h, 2);
  const double *G = h->rs_host + Q * R;
  const double tau_g = hp->tau_g > 0 ? hp->tau_g : 1e-4 * std::max(1.0, 1e4 / (double)h->n);
  bool stag[8];
  for (int r = 0; r < R; ++r) {
    double g2 = 0.0;
    for (int c = r * kb; c < (r + 1) * kb; ++c)
      for (int d = r * kb; d < (r + 1) * kb; ++d) g2 += G[c * kp + d] * G[c * kp + d];
    const double f = h->normS2 - g2 + 0.5 * h->rs_host[Q * r];
    const double E = f / h->normS2;
    const double kkt = std::sqrt(h->rs_host[Q * r + 1]) / ((double)h->n * (double)kb);
    symnmf_ctx::RestartCtl &c = h->rctl[r];
    if (t == 0 || !(c.E0 == c.E0)) c.E0 = E;
    const double ratio = c.have_prev ? (c.E_prev - E) / c.E0 : NAN;
    stag[r] = c.have_prev && t >= hp->warmup && ratio < hp->tau_stag;
    c.E_prev = E;
    c.have_prev = true;
    h->rE[r] = E;
    h->rkkt[r] = kkt;
    if (E < hp->tau_E && kkt < tau_g && stag[r]) {
      h->rconv[r] = 1;
      *any = true;
    }
  }
  if (hp->method != SYMNMF_PIECEWISE_ADAGRAD || *any || stopping) return SYMNMF_OK;
  for (int r = 0; r < R; ++r) {
    symnmf_ctx::RestartCtl &c = h->rctl[r];
    const double E = h->rE[r], sumA = h->rs_host[Q * r + 2];
    if (c.cooldown && sumA >= 2.0 * c.sumA_post) c.cooldown = false;
    if (c.cooldown || !c.resets_enabled || !stag[r] || !(h->rkkt[r] > hp->c_r * tau_g)) continue;
    double med = NAN;
    int rc = median_g2(h, r * kb, kb, &med);
    if (rc) return rc;
    if (!(med > hp->eps)) continue;
    if (c.resets > 0 && !(E < c.E_at_reset - hp->tau_stag * c.E0)) {
      c.resets_enabled = false;
      continue;
    }
    if ((rc = reset_columns(h, hp, r * kb, kb, &c.sumA_post))) return rc;
    c.cooldown = true;
    c.E_at_reset = E;
    c.resets += 1;
    *any_reset = true;
  }
  return SYMNMF_OK;
}

int iterate_finish(symnmf_t h, const symnmf_hparams *hp, std::vector<double> &phis) {
  const int64_t t = h->ctrl.t;
  int rc;
  if (t % hp->check_interval == 0) {
    if ((rc = finish_records(h, t + 1, phis))) return rc;
    phis.clear();
    symnmf_record &rec = h->trace.back();
    if (rec.nonfinite > 0) {
      h->ctrl.t = t + 1;
      return fail(h, SYMNMF_ERR_NONFINITE, "non-finite gradient entries at iteration " + std::to_string(t));
    }
    CheckOut o;
    int mrc = SYMNMF_OK;
    auto med = [&]() {
      double m = NAN;
      mrc = median_g2(h, 0, h->k, &m);
      return m;
    };
    // with restarts concatenated the Piecewise reset is each restart's own
    // (restart_checks); the handle's check keeps the AND rule
    symnmf_hparams hpc = *hp;
    if (h->restarts > 1 && hpc.method == SYMNMF_PIECEWISE_ADAGRAD) hpc.method = SYMNMF_ADAGRAD;
    ctrl_check(&h->ctrl, &hpc, h->n, t, rec.E, rec.kkt, rec.sumA, med, &o);
    if (mrc) return mrc;
    bool restart_reset = false;
    if (h->restarts > 1) {
      // a concatenated handle stops when any of its restarts converges
      bool any = false;
      if ((rc = restart_checks(h, hp, t, o.converged, &any, &restart_reset))) return rc;
      if (any && !o.converged) {
        o.converged = true;
        o.reset = false;
        h->ctrl.converged = 1;
      }
    }
    rec.check = 1;
    rec.median_g2 = o.median;
    rec.stag_ratio = o.ratio;
    rec.converged = o.converged ? 1 : 0;
    rec.reset = (o.reset || restart_reset) ? 1 : 0;
    h->last_check = t;
    h->last_check_rec = rec;
    if (o.converged) {
      h->cur = 1 - h->cur;  // the certified iterate is H_t (its buffers are intact)
      return SYMNMF_CONVERGED;
    }
    if (o.reset && (rc = reset_columns(h, hp, 0, h->k, &h->ctrl.sumA_post))) return rc;
  } else if (t + 1 - h->copied_upto >= kRing / 2) {
    if ((rc = finish_records(h, t + 1, phis))) return rc;
    phis.clear();
  }
  h->ctrl.t = t + 1;
  return SYMNMF_OK;
}

// one iteration plus its check; returns OK, CONVERGED or an error
int iterate_once(symnmf_t h, const symnmf_hparams *hp, std::vector<double> &phis, bool last) {
  int rc = iterate_launch(h, hp, phis, last);
  if (rc) return rc;
  return iterate_finish(h, hp, phis);
}

}  // namespace

// ====================================================================== API
extern "C" {

const char *symnmf_status_string(int32_t s) {
  switch (s) {
    case SYMNMF_OK: return "ok";
    case SYMNMF_CONVERGED: return "converged";
    case SYMNMF_ERR_INVALID: return "invalid argument";
    case SYMNMF_ERR_UNSUPPORTED: return "unsupported";
    case SYMNMF_ERR_OOM: return "out of memory";
    case SYMNMF_ERR_CUDA: return "CUDA error";
    case SYMNMF_ERR_TIMEOUT: return "device wait timed out";
    case SYMNMF_ERR_NONFINITE: return "non-finite values";
    case SYMNMF_ERR_STATE: return "handle in error state";
    default: return "unknown status";
  }
}

const char *symnmf_last_error(symnmf_t h) { return h ? h->err.c_str() : "null handle"; }

int symnmf_hparams_default(int32_t method, symnmf_hparams *hp) {
  if (!hp || method < 0 || method > SYMNMF_ADMM) return SYMNMF_ERR_INVALID;
  std::memset(hp, 0, sizeof(*hp));
  hp->method = method;
  hp->check_interval = 10;
  hp->warmup = 50;
  hp->snapshot_period = 10;
  hp->block_rows = kTileRows;
  hp->eta = 2.0;
  hp->eps = 1e-10;
  hp->alpha = 0.99;
  hp->mu = 0.5;
  hp->c = 10.0;
  hp->c_r = 10.0;
  hp->row_frac = 0.5;
  hp->phi0 = 0.5;
  hp->tau_E = 0.1;
  hp->tau_g = 0.0;
  hp->tau_stag = 1e-5;
  hp->growth_kkt_mult = 3.0;
  hp->seed = 0;
  hp->rho = 500.0;
  if (method == SYMNMF_RMSPROP) {
    hp->eta = 0.05;
    hp->eps = 1e-8;
  } else if (method == SYMNMF_PIECEWISE_ADAGRAD) {
    hp->eta = 1.0;
  } else if (method == SYMNMF_BLOCK_SVRG_ADAPTGROW) {
    hp->snapshot_period = 2;  // ~1/phi0
  }
  return SYMNMF_OK;
}

int symnmf_create_ld(const void *S, int64_t n, int64_t lds, int32_t k, int32_t dtype,
                     symnmf_t *out) {
  if (!out) return SYMNMF_ERR_INVALID;
  *out = nullptr;
  if (!S || n < 1 || lds < n || dtype < 0 || dtype > 2) return SYMNMF_ERR_INVALID;
  if (k < 1 || k > 64) return SYMNMF_ERR_UNSUPPORTED;
  if (n > (int64_t)INT32_MAX * kTileRows / 4) return SYMNMF_ERR_UNSUPPORTED;
  symnmf_ctx *h = new (std::nothrow) symnmf_ctx();
  if (!h) return SYMNMF_ERR_OOM;
  h->S = S;
  h->n = n;
  h->lds = lds;
  h->k = k;
  h->kp = pad_k(k);
  h->dtype = dtype;
  h->ntiles = (int)((n + kTileRows - 1) / kTileRows);
  h->ldb = (int64_t)h->ntiles * kTileRows;
  h->tc_layout_ok = ((uintptr_t)S % 16 == 0) && ((lds * (int64_t)esize(dtype)) % 16 == 0);
  h->bt_fmt = (dtype == SYMNMF_F32) ? 1 : (dtype == SYMNMF_FP8E4M3) ? 2 : 0;
  reset_ctrl(&h->ctrl);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  const int64_t nkp = (int64_t)h->ntiles * kTileRows * h->kp;  // tile column-major
  h->pq_cap_tiles = h->ntiles + 3 * (int64_t)std::max(1, h->num_sms);
  h->nchunks = std::max(1, std::min(h->ntiles, 64));
  h->n_norm_parts = 4 * std::max(1, h->num_sms);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = dalloc(&h->H[i], nkp);
    if (e == cudaSuccess)
      e = dalloc((uint8_t **)&h->Bt[i], bt_bytes(h->bt_fmt, h->kp, h->ldb));
    if (e == cudaSuccess) e = dalloc(&h->gram_part[i], (size_t)h->ntiles * h->kp * h->kp);
    if (e == cudaSuccess) e = dalloc(&h->gram64[i], (size_t)h->kp * h->kp);
    if (e == cudaSuccess) e = dalloc(&h->gram32[i], (size_t)h->kp * h->kp);
  }
  if (e == cudaSuccess) e = dalloc(&h->A, nkp);
  if (e == cudaSuccess) e = dalloc(&h->M, nkp);
  if (e == cudaSuccess) e = dalloc(&h->mu, nkp);
  if (e == cudaSuccess) e = dalloc(&h->g, nkp);
  if (e == cudaSuccess) e = dalloc(&h->tmp, nkp);
  if (e == cudaSuccess) e = dalloc(&h->P, (size_t)h->pq_cap_tiles * kTileRows * h->kp);
  if (e == cudaSuccess) e = dalloc(&h->Q, (size_t)h->pq_cap_tiles * kTileRows * h->kp);
  if (e == cudaSuccess) e = dalloc(&h->R, (size_t)h->pq_cap_tiles * kTileRows * h->kp);
  if (e == cudaSuccess) e = dalloc(&h->slots, (size_t)h->ntiles * kSlotStride);
  if (e == cudaSuccess) e = dalloc(&h->chunk, (size_t)h->nchunks * (4 + h->kp * h->kp));
  if (e == cudaSuccess) e = dalloc(&h->gramI, (size_t)h->kp * h->kp);
  if (e == cudaSuccess) e = dalloc(&h->gramJ, (size_t)h->kp * h->kp);
  if (e == cudaSuccess) e = dalloc(&h->minv, (size_t)h->kp * h->kp);
  if (e == cudaSuccess) e = dalloc(&h->dlists, (size_t)kStages * kListArrays * h->ntiles);
  if (e == cudaSuccess) e = dalloc(&h->ring, (size_t)kRing + 1);
  if (e == cudaSuccess) e = dalloc(&h->hist, 2048);
  if (e == cudaSuccess) e = dalloc(&h->sel, 4);
  if (e == cudaSuccess) e = dalloc(&h->dmed, 1);
  if (e == cudaSuccess) e = dalloc(&h->dsum, 4);
  if (e == cudaSuccess) e = dalloc(&h->norm_parts, (size_t)h->n_norm_parts);
  if (e == cudaSuccess) e = dalloc(&h->dev_err, 4);
  h->ntc = (h->ntiles + 31) / 32;
  if (e == cudaSuccess) e = dalloc(&h->counters, 64);
  if (e == cudaSuccess) e = dalloc(&h->tile_cnt, (size_t)h->ntiles);
  if (e == cudaSuccess) e = dalloc(&h->lvl1, (size_t)h->ntc * (4 + h->kp * h->kp));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->host_err, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hlists, sizeof(int) * kStages * kListArrays * h->ntiles);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hring, sizeof(DevRecord) * (kRing + 1));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hsum, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hmed, sizeof(float) * 4);
  for (int i = 0; i < kStages && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&h->stage_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    const int st = (e == cudaErrorMemoryAllocation) ? SYMNMF_ERR_OOM : SYMNMF_ERR_CUDA;
    cudaGetLastError();
    free_all(h);
    delete h;
    return st;
  }
  if (dtype != SYMNMF_FP8E4M3) {
    const int rc = compute_norm(h);
    if (rc) {
      free_all(h);
      delete h;
      return rc;
    }
  }
  *out = h;
  return SYMNMF_OK;
}

int symnmf_create(const void *S, int64_t n, int32_t k, int32_t dtype, symnmf_t *out) {
  return symnmf_create_ld(S, n, n, k, dtype, out);
}

void symnmf_destroy(symnmf_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

int symnmf_set_stream(symnmf_t h, void *stream) {
  if (!h) return SYMNMF_ERR_INVALID;
  h->stream = (cudaStream_t)stream;
  return SYMNMF_OK;
}

int symnmf_set_tile_scales(symnmf_t h, const float *scales, int64_t ld_scales) {
  if (!h || !scales || ld_scales < h->ntiles) return SYMNMF_ERR_INVALID;
  if (h->dtype != SYMNMF_FP8E4M3) return fail(h, SYMNMF_ERR_INVALID, "tile scales apply to FP8 storage only");
  h->scales = scales;
  h->ld_scales = ld_scales;
  return compute_norm(h);
}

int symnmf_quantize_fp8(const void *src, int32_t src_dtype, int64_t rows, int64_t cols,
                        int64_t ld_src, uint8_t *q, int64_t ldq, float *scales, int64_t ld_scales,
                        double *tile_sumsq, void *stream) {
  if (!src || !q || !scales || rows < 1 || cols < 1 || ld_src < cols || ldq < cols ||
      ld_scales < (cols + kTileRows - 1) / kTileRows)
    return SYMNMF_ERR_INVALID;
  if (src_dtype != SYMNMF_F32 && src_dtype != SYMNMF_BF16) return SYMNMF_ERR_INVALID;
  if ((rows + kTileRows - 1) / kTileRows > 65535) return SYMNMF_ERR_UNSUPPORTED;
  const cudaError_t e = launch_quantize_fp8(src, src_dtype, rows, cols, ld_src, q, ldq, scales,
                                            ld_scales, tile_sumsq, (cudaStream_t)stream);
  return e == cudaSuccess ? SYMNMF_OK : SYMNMF_ERR_CUDA;
}

int symnmf_get_restart_ctrl(symnmf_t h, int32_t count, int32_t *resets, int32_t *resets_enabled,
                            int32_t *cooldown, double *sumA_post) {
  if (!h || count < h->restarts) return SYMNMF_ERR_INVALID;
  for (int r = 0; r < h->restarts; ++r) {
    const bool have = h->restarts > 1 && r < (int)h->rctl.size();
    const symnmf_ctx::RestartCtl c = have ? h->rctl[r] : symnmf_ctx::RestartCtl{};
    if (resets) resets[r] = have ? c.resets : h->ctrl.resets;
    if (resets_enabled) resets_enabled[r] = have ? (c.resets_enabled ? 1 : 0) : h->ctrl.resets_enabled;
    if (cooldown) cooldown[r] = have ? (c.cooldown ? 1 : 0) : h->ctrl.cooldown;
    if (sumA_post) sumA_post[r] = have ? c.sumA_post : h->ctrl.sumA_post;
  }
  return SYMNMF_OK;
}

int symnmf_get_restart_stats(symnmf_t h, int32_t count, double *E, double *kkt,
                             int32_t *converged) {
  if (!h || count < h->restarts) return SYMNMF_ERR_INVALID;
  for (int r = 0; r < h->restarts; ++r) {
    const bool have = h->restarts > 1 && r < (int)h->rE.size();
    if (E) E[r] = have ? h->rE[r] : h->last_check_rec.E;
    if (kkt) kkt[r] = have ? h->rkkt[r] : h->last_check_rec.kkt;
    if (converged) converged[r] = have ? h->rconv[r] : h->ctrl.converged;
  }
  return SYMNMF_OK;
}

// Rebind h to S (stream-ordered; the caller has validated the arguments):
// H stays as the warm start, the rest of the solver state starts afresh.
// ||S||^2 is left to the caller.
static int rebind_matrix(symnmf_t h, const void *S, int64_t lds, const float *scales,
                         int64_t ld_scales) {
  h->S = S;
  h->lds = lds;
  h->tc_layout_ok = ((uintptr_t)S % 16 == 0) && ((lds * (int64_t)esize(h->dtype)) % 16 == 0);
  if (h->dtype == SYMNMF_FP8E4M3) {
    h->scales = scales;
    h->ld_scales = ld_scales;
  }
  // H (and its MMA copy and Gram) is kept as the warm start; the optimizer
  // state, the snapshot, the gradient, the controller and the trace start
  // afresh for the new problem
  const size_t bytes = sizeof(float) * (size_t)h->ntiles * kTileRows * h->kp;
  CK(cudaMemsetAsync(h->A, 0, bytes, h->stream));
  CK(cudaMemsetAsync(h->M, 0, bytes, h->stream));
  CK(cudaMemsetAsync(h->mu, 0, bytes, h->stream));
  CK(cudaMemsetAsync(h->g, 0, bytes, h->stream));
  reset_ctrl(&h->ctrl);
  reset_restart_checks(h);
  h->trace.clear();
  h->copied_upto = 0;
  h->last_check = -1;
  std::memset(&h->last_check_rec, 0, sizeof(h->last_check_rec));
  if (h->km_rn) {
    CK(launch_row_norms(h->S, h->n, h->lds, h->dtype, h->scales, h->ld_scales, h->km_rn,
                        h->stream));
  }
  return SYMNMF_OK;
}

int symnmf_set_matrix(symnmf_t h, const void *S, int64_t lds, const float *scales,
                      int64_t ld_scales) {
  if (!h || !S || lds < h->n) return SYMNMF_ERR_INVALID;
  if (h->dtype == SYMNMF_FP8E4M3 && (!scales || ld_scales < h->ntiles)) return SYMNMF_ERR_INVALID;
  // every launch that reads the old matrix has finished
  CK(cudaStreamSynchronize(h->stream));
  int rc = rebind_matrix(h, S, lds, scales, ld_scales);
  if (rc) return rc;
  return compute_norm(h);
}

int symnmf_window_update(symnmf_t h, const float *Y, int64_t T, int64_t ldy, int32_t center,
                         void *S, int64_t lds, float *scales, int64_t ld_scales) {
  if (!h || !Y || !S || T < 1 || ldy < h->n || lds < h->n) return SYMNMF_ERR_INVALID;
  if (center && T < 2) return SYMNMF_ERR_INVALID;
  const int64_t es = esize(h->dtype);
  if ((lds * es) % 16 != 0 || reinterpret_cast<uintptr_t>(S) % 16 != 0) return SYMNMF_ERR_INVALID;
  const bool f8 = (h->dtype == SYMNMF_FP8E4M3);
  if (f8 && (!scales || ld_scales < h->ntiles)) return SYMNMF_ERR_INVALID;
  if (h->n > 2097120 || T > (int64_t)1 << 30) return SYMNMF_ERR_UNSUPPORTED;
  CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
  // the build, ordered after every launch that reads the old matrix; it
  // leaves ||S||^2 of the stored values in dsum (F32 / BF16)
  const int dt = h->dtype == SYMNMF_F32 ? 0 : h->dtype == SYMNMF_BF16 ? 1 : 2;
  cudaError_t e = launch_dependence(Y, T, h->n, ldy, center ? 1 : 0, dt, S, lds, scales,
                                    ld_scales, f8 ? nullptr : h->dsum, h->dev_err, h->stream,
                                    true);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(h, SYMNMF_ERR_OOM, "dependence build scratch");
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "dependence build");
  CK(cudaMemcpyAsync(h->host_err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  int rc = rebind_matrix(h, S, lds, scales, ld_scales);
  if (rc) return rc;
  if (f8) {
    rc = compute_norm(h);  // synchronises the stream
    if (rc) return rc;
  } else {
    CK(cudaMemcpyAsync(h->hsum, h->dsum, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->normS2 = h->hsum[0];
  }
  if (h->host_err[0] != 0)
    return fail(h, SYMNMF_ERR_TIMEOUT,
                "a bounded device wait gave up (code " + std::to_string(h->host_err[0]) + ")");
  return SYMNMF_OK;
}

int symnmf_set_restarts(symnmf_t h, int32_t restarts) {
  if (!h || restarts < 1 || restarts > 8 || h->k % restarts != 0) return SYMNMF_ERR_INVALID;
  if (restarts > 1 && !h->rs_part) {
    cudaError_t e = dalloc(&h->rs_part, (size_t)h->ntiles * kRestartSums * 8);
    if (e == cudaSuccess) e = dalloc(&h->rs_out, kRestartSums * 8);
    if (e == cudaSuccess)
      e = cudaMallocHost((void **)&h->rs_host, sizeof(double) * (kRestartSums * 8 + 64 * 64));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, SYMNMF_ERR_OOM, "restart check scratch");
    }
  }
  h->restarts = restarts;
  reset_restart_checks(h);
  // the Gram of the current H under the new block structure
  return refresh_derived(h);
}

int symnmf_set_norm(symnmf_t h, double normS2) {
  if (!h || !(normS2 > 0) || !std::isfinite(normS2)) return SYMNMF_ERR_INVALID;
  h->normS2 = normS2;
  return SYMNMF_OK;
}

int symnmf_get_norm(symnmf_t h, double *normS2) {
  if (!h || !normS2) return SYMNMF_ERR_INVALID;
  *normS2 = h->normS2;
  return SYMNMF_OK;
}

int symnmf_set_impl(symnmf_t h, int32_t impl) {
  if (!h || impl < 0 || impl > 2) return SYMNMF_ERR_INVALID;
  if (impl == 2 && !(h->tc_layout_ok && tc_supported(h->dtype, h->kp)))
    return fail(h, SYMNMF_ERR_UNSUPPORTED, "tensor-core product unavailable for this layout");
  h->impl_req = impl;
  return SYMNMF_OK;
}

int symnmf_get_impl(symnmf_t h, int32_t *impl) {
  if (!h || !impl) return SYMNMF_ERR_INVALID;
  *impl = use_tc(h) ? 2 : 1;
  return SYMNMF_OK;
}

int symnmf_set_H(symnmf_t h, const float *H) {
  if (!h || !H) return SYMNMF_ERR_INVALID;
  h->bad = false;
  h->err.clear();
  h->cur = 0;
  CK(launch_pack(H, h->H[0], h->n, h->k, h->kp, h->stream));
  const size_t bytes = sizeof(float) * (size_t)h->ntiles * kTileRows * h->kp;
  CK(cudaMemsetAsync(h->H[1], 0, bytes, h->stream));
  CK(cudaMemsetAsync(h->A, 0, bytes, h->stream));
  CK(cudaMemsetAsync(h->M, 0, bytes, h->stream));
  CK(cudaMemsetAsync(h->mu, 0, bytes, h->stream));
  CK(cudaMemsetAsync(h->g, 0, bytes, h->stream));
  CK(cudaMemsetAsync(h->counters, 0, sizeof(int) * 64, h->stream));
  CK(cudaMemsetAsync(h->tile_cnt, 0, sizeof(int) * h->ntiles, h->stream));
  reset_ctrl(&h->ctrl);
  reset_restart_checks(h);
  h->trace.clear();
  h->copied_upto = 0;
  h->last_check = -1;
  std::memset(&h->last_check_rec, 0, sizeof(h->last_check_rec));
  int rc = refresh_derived(h);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return SYMNMF_OK;
}

int symnmf_get_H(symnmf_t h, float *H) {
  if (!h || !H) return SYMNMF_ERR_INVALID;
  CK(launch_unpack(h->H[h->cur], H, h->n, h->k, h->kp, h->stream));
  return SYMNMF_OK;
}

// symnmf_solve_host after its argument checks: the uploads, the solve and
// the copy of H back (see the header)
static int solve_host_run(symnmf_t h, const void *S_host, int64_t lds_host,
                          const float *scales_host, int64_t ld_scales_host, double normS2,
                          const float *H0_host, const symnmf_hparams *hp, int32_t iters,
                          float *H_out, symnmf_stats *stats) {
  const bool f8 = (h->dtype == SYMNMF_FP8E4M3);
  const int64_t nt = (h->n + kTileRows - 1) / kTileRows;
  const size_t es = esize(h->dtype);
  // the device buffer the handle was created on (and its FP8 scales) take
  // the caller's matrix; H_0 goes through the staging buffer
  if (lds_host == h->lds) {
    // one contiguous copy: a pitched copy of 2D rows moves far fewer bytes
    // per second from pinned memory
    const size_t bytes = ((size_t)(h->n - 1) * (size_t)h->lds + (size_t)h->n) * es;
    CK(cudaMemcpyAsync(const_cast<void *>(h->S), S_host, bytes, cudaMemcpyHostToDevice,
                       h->stream));
  } else {
    CK(cudaMemcpy2DAsync(const_cast<void *>(h->S), (size_t)h->lds * es, S_host,
                         (size_t)lds_host * es, (size_t)h->n * es, (size_t)h->n,
                         cudaMemcpyHostToDevice, h->stream));
  }
  if (f8)
    CK(cudaMemcpy2DAsync(const_cast<float *>(h->scales), (size_t)h->ld_scales * 4, scales_host,
                         (size_t)ld_scales_host * 4, (size_t)nt * 4, (size_t)nt,
                         cudaMemcpyHostToDevice, h->stream));
  const size_t nk = sizeof(float) * (size_t)h->n * (size_t)h->k;
  CK(cudaMemcpyAsync(h->tmp, H0_host, nk, cudaMemcpyHostToDevice, h->stream));
  int rc;
  if (normS2 > 0 && std::isfinite(normS2)) h->normS2 = normS2;
  else if ((rc = compute_norm(h))) return rc;
  if ((rc = symnmf_set_H(h, h->tmp))) return rc;
  symnmf_stats st{};
  const int src = symnmf_step(h, hp, iters, stats ? stats : &st);
  if (src < 0) return src;
  CK(launch_unpack(h->H[h->cur], h->tmp, h->n, h->k, h->kp, h->stream));
  CK(cudaMemcpyAsync(H_out, h->tmp, nk, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return src;
}

int symnmf_solve_host(symnmf_t h, const void *S_host, int64_t lds_host, const float *scales_host,
                      int64_t ld_scales_host, double normS2, const float *H0_host,
                      const symnmf_hparams *hp, int32_t iters, float *H_out, symnmf_stats *stats) {
  if (!h || !S_host || !H0_host || !H_out || !hp || iters < 0 || lds_host < h->n)
    return SYMNMF_ERR_INVALID;
  const int64_t nt = (h->n + kTileRows - 1) / kTileRows;
  if (h->dtype == SYMNMF_FP8E4M3 && (!scales_host || !h->scales || ld_scales_host < nt))
    return SYMNMF_ERR_INVALID;
  const int rc = solve_host_run(h, S_host, lds_host, scales_host, ld_scales_host, normS2, H0_host,
                                hp, iters, H_out, stats);
  // on an error no copy may still be reading the caller's host buffers
  if (rc < 0) cudaStreamSynchronize(h->stream);
  return rc;
}

int symnmf_get_buffer(symnmf_t h, int32_t which, float *dst) {
  if (!h || !dst) return SYMNMF_ERR_INVALID;
  const float *src = which == SYMNMF_BUF_H ? h->H[h->cur]
                     : which == SYMNMF_BUF_ACC ? h->A
                     : which == SYMNMF_BUF_MOM ? h->M
                     : which == SYMNMF_BUF_SNAPSHOT ? h->mu
                     : which == SYMNMF_BUF_GRAD ? h->g : nullptr;
  if (!src) return SYMNMF_ERR_INVALID;
  CK(launch_unpack(src, dst, h->n, h->k, h->kp, h->stream));
  return SYMNMF_OK;
}

int symnmf_set_buffer(symnmf_t h, int32_t which, const float *src) {
  if (!h || !src) return SYMNMF_ERR_INVALID;
  float *dst = which == SYMNMF_BUF_H ? h->H[h->cur]
               : which == SYMNMF_BUF_ACC ? h->A
               : which == SYMNMF_BUF_MOM ? h->M
               : which == SYMNMF_BUF_SNAPSHOT ? h->mu : nullptr;
  if (!dst) return SYMNMF_ERR_INVALID;
  CK(launch_pack(src, dst, h->n, h->k, h->kp, h->stream));
  if (which == SYMNMF_BUF_H) {
    int rc = refresh_derived(h);
    if (rc) return rc;
  }
  return SYMNMF_OK;
}

int symnmf_get_ctrl(symnmf_t h, symnmf_ctrl *out) {
  if (!h || !out) return SYMNMF_ERR_INVALID;
  *out = h->ctrl;
  return SYMNMF_OK;
}

int symnmf_set_ctrl(symnmf_t h, const symnmf_ctrl *in) {
  if (!h || !in || in->t < 0) return SYMNMF_ERR_INVALID;
  h->ctrl = *in;
  h->copied_upto = in->t;
  return SYMNMF_OK;
}

int symnmf_grad(symnmf_t h, float *G) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!G) return SYMNMF_ERR_INVALID;
  EpiArgs e = base_epi(h, nullptr);
  e.mode = MODE_GRAD_ONLY;
  e.gram = h->gram32[h->cur];
  e.P = h->P;
  e.n1 = h->ntiles;
  e.gcaller = G;
  PartLayout ly;
  if (use_tc(h)) return prod(h, nullptr, h->ntiles, nullptr, h->ntiles, h->P, &ly, &e);
  if ((rc = prod(h, nullptr, h->ntiles, nullptr, h->ntiles, h->P, &ly))) return rc;
  e.nsplit = ly.nsplit;
  e.skG1 = ly.skG;
  e.ncols1 = ly.ncols;
  CK(launch_epilogue(e, h->stream));
  return SYMNMF_OK;
}

int symnmf_objective(symnmf_t h, double *f, double *E) {
  int rc = check_handle(h);
  if (rc) return rc;
  EpiArgs e = base_epi(h, nullptr);
  e.mode = MODE_GRAD_ONLY;
  e.gram = h->gram32[h->cur];
  e.P = h->P;
  e.n1 = h->ntiles;
  e.slots = h->slots;
  PartLayout ly;
  if (use_tc(h)) {
    if ((rc = prod(h, nullptr, h->ntiles, nullptr, h->ntiles, h->P, &ly, &e))) return rc;
  } else {
    if ((rc = prod(h, nullptr, h->ntiles, nullptr, h->ntiles, h->P, &ly))) return rc;
    e.nsplit = ly.nsplit;
    e.skG1 = ly.skG;
    e.ncols1 = ly.ncols;
    CK(launch_epilogue(e, h->stream));
  }
  CK(launch_reduce_iter(reduce_args(h, h->slots, nullptr, -1, 1), h->kp, h->stream));
  CK(cudaMemcpyAsync(h->hring + kRing, h->ring + kRing, sizeof(DevRecord),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (f) *f = h->hring[kRing].f;
  if (E) *E = h->hring[kRing].E;
  return SYMNMF_OK;
}

int symnmf_build_dependence(const float *Y, int64_t T, int64_t n, int64_t ldy, int32_t center,
                            int32_t out_dtype, void *S, int64_t lds, float *scales,
                            int64_t ld_scales, double *normS2, void *stream) {
  if (!Y || !S || T < 1 || n < 1 || ldy < n || lds < n) return SYMNMF_ERR_INVALID;
  if (center && T < 2) return SYMNMF_ERR_INVALID;
  if (out_dtype != SYMNMF_F32 && out_dtype != SYMNMF_BF16 && out_dtype != SYMNMF_FP8E4M3)
    return SYMNMF_ERR_INVALID;
  const int64_t es = out_dtype == SYMNMF_F32 ? 4 : out_dtype == SYMNMF_BF16 ? 2 : 1;
  if ((lds * es) % 16 != 0 || reinterpret_cast<uintptr_t>(S) % 16 != 0) return SYMNMF_ERR_INVALID;
  const int64_t nt = (n + 127) / 128;
  if (out_dtype == SYMNMF_FP8E4M3 && (!scales || ld_scales < nt)) return SYMNMF_ERR_INVALID;
  if (n > 2097120 || T > (int64_t)1 << 30) return SYMNMF_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  int *derr = nullptr;
  int herr = 0;
  cudaError_t e = cudaMallocAsync((void **)&derr, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    const int dt = out_dtype == SYMNMF_F32 ? 0 : out_dtype == SYMNMF_BF16 ? 1 : 2;
    e = launch_dependence(Y, T, n, ldy, center ? 1 : 0, dt, S, lds, scales, ld_scales, normS2,
                          derr, s);
  }
  if (derr) {
    cudaError_t e2 = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(derr, s);
    if (e == cudaSuccess) e = e2;
  }
  cudaError_t es2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = es2;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return SYMNMF_ERR_OOM;
  }
  if (e != cudaSuccess) return SYMNMF_ERR_CUDA;
  if (herr != 0) return SYMNMF_ERR_TIMEOUT;
  return SYMNMF_OK;
}

int symnmf_spkmeans(symnmf_t h, const int32_t *labels0, int32_t *labels, int32_t max_iter,
                    double tol, double *J_trace, symnmf_kmeans_stats *stats) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!labels0 || !labels || max_iter < 1 || !(tol >= 0))
    return fail(h, SYMNMF_ERR_INVALID, "spkmeans: null labels, max_iter < 1 or tol < 0");
  if (!h->km_rn) {
    cudaError_t e = dalloc(&h->km_rn, (size_t)h->n);
    if (e == cudaSuccess) e = dalloc(&h->km_lab, (size_t)2 * h->n);
    if (e == cudaSuccess) e = dalloc(&h->km_colsq, (size_t)h->ntiles * h->kp);
    if (e == cudaSuccess) e = dalloc(&h->km_inv, (size_t)h->kp);
    if (e == cudaSuccess) e = dalloc(&h->km_slots, (size_t)h->ntiles * 2);
    if (e == cudaSuccess) e = dalloc(&h->km_out, 2);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->km_hout, 2 * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      for (void *p : {(void *)h->km_rn, (void *)h->km_lab, (void *)h->km_colsq, (void *)h->km_inv,
                      (void *)h->km_slots, (void *)h->km_out})
        cudaFree(p);
      if (h->km_hout) cudaFreeHost(h->km_hout);
      h->km_rn = nullptr;
      h->km_lab = nullptr;
      h->km_colsq = nullptr;
      h->km_inv = nullptr;
      h->km_slots = nullptr;
      h->km_out = nullptr;
      h->km_hout = nullptr;
      return fail(h, SYMNMF_ERR_OOM, "spkmeans scratch");
    }
    CK(launch_row_norms(h->S, h->n, h->lds, h->dtype, h->scales, h->ld_scales, h->km_rn,
                        h->stream));
    count_kernels(h, 1);
  }
  // the two product operands go through the solver's other H buffer and MMA
  // copy, so H_t, its copy and its Gram stay as they are
  struct KeepCur {
    symnmf_t h;
    int c;
    ~KeepCur() { h->cur = c; }
  } keep{h, h->cur};
  h->cur = 1 - keep.c;
  float *Hop = h->H[h->cur];
  const int64_t rows_alloc = (int64_t)h->ntiles * kTileRows;
  CK(cudaMemcpyAsync(h->km_lab, labels0, sizeof(int32_t) * h->n, cudaMemcpyDeviceToDevice,
                     h->stream));
  KmArgs a{};
  a.n = h->n;
  a.K = h->k;
  a.ntiles = h->ntiles;
  a.P = h->P;
  a.C = Hop;
  a.colsq = h->km_colsq;
  a.inv_norm = h->km_inv;
  a.rn = h->km_rn;
  a.slots = h->km_slots;
  a.out = h->km_out;
  symnmf_kmeans_stats st{};
  st.J = st.J_prev = NAN;
  int li = 0;
  for (int32_t t = 0; t < max_iter; ++t) {
    int *lin = h->km_lab + (size_t)li * h->n;
    int *lout = h->km_lab + (size_t)(1 - li) * h->n;
    // pass 1: C = S (D^-1 B)
    CK(launch_km_operand(lin, h->km_rn, h->n, h->kp, Hop, rows_alloc, h->stream));
    CK(launch_prepare_tiles(Hop, h->n, h->k, h->kp, h->Bt[h->cur], h->bt_fmt, h->ldb, nullptr,
                            h->stream));
    PartLayout ly;
    if ((rc = prod(h, nullptr, h->ntiles, nullptr, h->ntiles, h->P, &ly))) return rc;
    a.nsplit = ly.nsplit;
    a.skG = ly.skG;
    a.ncols = ly.ncols;
    CK(launch_km_centroids(a, h->kp, h->stream));
    // pass 2: P = S C, then the assignment
    CK(launch_prepare_tiles(Hop, h->n, h->k, h->kp, h->Bt[h->cur], h->bt_fmt, h->ldb, nullptr,
                            h->stream));
    if ((rc = prod(h, nullptr, h->ntiles, nullptr, h->ntiles, h->P, &ly))) return rc;
    a.nsplit = ly.nsplit;
    a.skG = ly.skG;
    a.ncols = ly.ncols;
    a.labels_in = lin;
    a.labels_out = lout;
    CK(launch_km_assign(a, h->kp, h->stream));
    count_kernels(h, 6);
    CK(cudaMemcpyAsync(h->km_hout, h->km_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaMemcpyAsync(h->host_err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->host_err[0] != 0)
      return fail(h, SYMNMF_ERR_TIMEOUT,
                  "a bounded device wait gave up (code " + std::to_string(h->host_err[0]) + ")");
    const double J = h->km_hout[0];
    const int64_t changed = (int64_t)h->km_hout[1];
    if (!std::isfinite(J)) return fail(h, SYMNMF_ERR_NONFINITE, "spkmeans: non-finite objective");
    if (J_trace) J_trace[t] = J;
    li = 1 - li;
    st.iters = t + 1;
    st.J_prev = st.J;
    st.J = J;
    st.changed = changed;
    if (changed == 0 || (t >= 1 && st.J_prev - J <= tol * st.J_prev)) {
      st.converged = 1;
      break;
    }
  }
  CK(cudaMemcpyAsync(labels, h->km_lab + (size_t)li * h->n, sizeof(int32_t) * h->n,
                     cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (stats) *stats = st;
  return SYMNMF_OK;
}

int symnmf_step(symnmf_t h, const symnmf_hparams *hp, int32_t iters, symnmf_stats *stats) {
  int rc = check_handle(h);
  if (rc) return rc;
  if ((rc = validate_hp(hp))) return fail(h, rc, "invalid hyper-parameters");
  if (iters < 0) return fail(h, SYMNMF_ERR_INVALID, "iters < 0");
  std::vector<double> phis;
  rc = SYMNMF_OK;
  for (int32_t i = 0; i < iters; ++i) {
    rc = iterate_once(h, hp, phis, i + 1 == iters);
    if (rc) break;
  }
  if (rc == SYMNMF_OK || rc == SYMNMF_CONVERGED) {
    const int64_t upto = h->ctrl.converged && rc == SYMNMF_CONVERGED ? h->ctrl.t + 1 : h->ctrl.t;
    int rc2 = sync_records(h, std::max(upto, h->copied_upto), phis);
    if (rc2) rc = rc2;
  }
  fill_stats(h, stats);
  return rc;
}

int symnmf_batch_step(symnmf_t *hs, int32_t count, const symnmf_hparams *hps, int32_t iters,
                      symnmf_stats *outs) {
  if (!hs || !hps || count < 0 || iters < 0) return SYMNMF_ERR_INVALID;
  std::vector<int> live(count, 1);
  std::vector<std::vector<double>> phis(count);
  int first_err = SYMNMF_OK;
  for (int32_t i = 0; i < count; ++i) {
    int rc = check_handle(hs[i]);
    if (!rc) rc = validate_hp(&hps[i]);
    if (rc) {
      live[i] = 0;
      if (!first_err) first_err = rc;
    }
  }
  for (int32_t it = 0; it < iters; ++it) {
    // every live handle's iteration is launched before any check waits, so
    // one handle's check does not hold back the others' launches
    for (int32_t i = 0; i < count; ++i) {
      if (!live[i]) continue;
      const int rc = iterate_launch(hs[i], &hps[i], phis[i], it + 1 == iters);
      if (rc) {
        live[i] = 0;
        if (!first_err) first_err = rc;
      }
    }
    bool any = false;
    for (int32_t i = 0; i < count; ++i) {
      if (!live[i]) continue;
      const int rc = iterate_finish(hs[i], &hps[i], phis[i]);
      if (rc == SYMNMF_CONVERGED) {
        live[i] = 0;
      } else if (rc) {
        live[i] = 0;
        if (!first_err) first_err = rc;
      } else {
        any = true;
      }
    }
    if (!any) break;
  }
  for (int32_t i = 0; i < count; ++i) {
    if (!hs[i]) continue;
    if (!hs[i]->bad) {
      symnmf_t h = hs[i];
      const int64_t upto = h->ctrl.converged ? h->ctrl.t + 1 : h->ctrl.t;
      int rc = sync_records(h, std::max(upto, h->copied_upto), phis[i]);
      if (rc && !first_err) first_err = rc;
    }
    if (outs) fill_stats(hs[i], &outs[i]);
  }
  return first_err;
}

int symnmf_set_ctas(symnmf_t h, int32_t ctas) {
  if (!h || ctas < 0) return SYMNMF_ERR_INVALID;
  h->ctas = ctas;
  return SYMNMF_OK;
}

int symnmf_get_ctas(symnmf_t h, int32_t *ctas) {
  if (!h || !ctas) return SYMNMF_ERR_INVALID;
  *ctas = (h->ctas > 0 && h->ctas < h->num_sms) ? h->ctas : h->num_sms;
  return SYMNMF_OK;
}

int symnmf_batch_autotune(symnmf_t *hs, int32_t count, const symnmf_hparams *hps, int32_t iters,
                          int32_t *ctas_out) {
  if (!hs || !hps || count < 1 || iters < 1) return SYMNMF_ERR_INVALID;
  for (int32_t i = 0; i < count; ++i)
    if (!hs[i]) return SYMNMF_ERR_INVALID;
  const int sms = std::max(1, hs[0]->num_sms);
  std::vector<double> w(count);
  double W = 0.0;
  for (int32_t i = 0; i < count; ++i) {
    w[i] = (double)hs[i]->n * (double)hs[i]->n * (double)esize(hs[i]->dtype);
    W += w[i];
  }
  // schedule m = 0: every handle on all SMs; m > 0: handle i gets a share
  // m * sms * w_i / W of the SMs (at least one CTA), so that m = 1 fills
  // the GPU once if all handles stream at the same time
  const double ms[] = {0.0, 1.0, 2.0, 4.0};
  double best_rate = -1.0;
  std::vector<int32_t> best(count, 0), cur(count, 0);
  std::vector<symnmf_stats> st(count);
  for (double m : ms) {
    for (int32_t i = 0; i < count; ++i) {
      cur[i] = (m == 0.0)
                   ? 0
                   : (int32_t)std::min<double>(sms, std::max(1.0, std::ceil(m * sms * w[i] / W)));
      hs[i]->ctas = cur[i];
    }
    int64_t before = 0, after = 0;
    for (int32_t i = 0; i < count; ++i) before += hs[i]->ctrl.t;
    if (cudaDeviceSynchronize() != cudaSuccess) return SYMNMF_ERR_CUDA;
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = symnmf_batch_step(hs, count, hps, iters, st.data());
    if (cudaDeviceSynchronize() != cudaSuccess) return SYMNMF_ERR_CUDA;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rc < 0) return rc;
    for (int32_t i = 0; i < count; ++i) after += hs[i]->ctrl.t;
    const double rate = (double)(after - before) / std::max(el, 1e-9);
    if (rate > best_rate) {
      best_rate = rate;
      best = cur;
    }
  }
  for (int32_t i = 0; i < count; ++i) {
    hs[i]->ctas = best[i];
    if (ctas_out) ctas_out[i] = best[i] > 0 ? best[i] : sms;
  }
  return SYMNMF_OK;
}

int symnmf_set_profiling(symnmf_t h, int32_t enable) {
  if (!h) return SYMNMF_ERR_INVALID;
  if (enable) {
    h->prof_used = 0;
    h->prof_bytes = 0.0;
    h->prof_kernels = 0;
  }
  h->profiling = enable != 0;
  return SYMNMF_OK;
}

int symnmf_get_profile(symnmf_t h, double *product_ms, int64_t *launches, double *s_bytes,
                       int64_t *kernel_launches) {
  if (!h) return SYMNMF_ERR_INVALID;
  CK(cudaStreamSynchronize(h->stream));
  double ms = 0.0;
  for (size_t i = 0; i + 1 < h->prof_used; i += 2) {
    float x = 0.f;
    CK(cudaEventElapsedTime(&x, h->prof_ev[i], h->prof_ev[i + 1]));
    ms += x;
  }
  if (product_ms) *product_ms = ms;
  if (launches) *launches = (int64_t)(h->prof_used / 2);
  if (s_bytes) *s_bytes = h->prof_bytes;
  if (kernel_launches) *kernel_launches = h->prof_kernels;
  return SYMNMF_OK;
}

int symnmf_get_trace(symnmf_t h, symnmf_record *out, int64_t max, int64_t *count) {
  if (!h || !count || max < 0 || (max > 0 && !out)) return SYMNMF_ERR_INVALID;
  *count = (int64_t)h->trace.size();
  const int64_t m = std::min<int64_t>(max, *count);
  for (int64_t i = 0; i < m; ++i) out[i] = h->trace[i];
  return SYMNMF_OK;
}

int symnmf_state_bytes(symnmf_t h, size_t *bytes) {
  if (!h || !bytes) return SYMNMF_ERR_INVALID;
  *bytes = 4 * sizeof(int64_t) + sizeof(symnmf_ctrl) + 4 * sizeof(float) * (size_t)h->n * h->k;
  return SYMNMF_OK;
}

int symnmf_get_state(symnmf_t h, void *buf, size_t bytes) {
  size_t need = 0;
  if (!h || !buf || symnmf_state_bytes(h, &need) || bytes < need) return SYMNMF_ERR_INVALID;
  char *p = (char *)buf;
  const int64_t hdr[4] = {(int64_t)kMagic, h->n, h->k, (int64_t)sizeof(symnmf_ctrl)};
  std::memcpy(p, hdr, sizeof(hdr));
  p += sizeof(hdr);
  std::memcpy(p, &h->ctrl, sizeof(symnmf_ctrl));
  p += sizeof(symnmf_ctrl);
  const size_t nk = sizeof(float) * (size_t)h->n * h->k;
  const float *srcs[4] = {h->H[h->cur], h->A, h->M, h->mu};
  for (int i = 0; i < 4; ++i) {
    CK(launch_unpack(srcs[i], h->tmp, h->n, h->k, h->kp, h->stream));
    CK(cudaMemcpyAsync(p, h->tmp, nk, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    p += nk;
  }
  return SYMNMF_OK;
}

int symnmf_set_state(symnmf_t h, const void *buf, size_t bytes) {
  size_t need = 0;
  if (!h || !buf || symnmf_state_bytes(h, &need) || bytes < need) return SYMNMF_ERR_INVALID;
  const char *p = (const char *)buf;
  int64_t hdr[4];
  std::memcpy(hdr, p, sizeof(hdr));
  if (hdr[0] != (int64_t)kMagic || hdr[1] != h->n || hdr[2] != h->k ||
      hdr[3] != (int64_t)sizeof(symnmf_ctrl))
    return fail(h, SYMNMF_ERR_INVALID, "checkpoint does not match this handle");
  p += sizeof(hdr);
  symnmf_ctrl c;
  std::memcpy(&c, p, sizeof(c));
  p += sizeof(symnmf_ctrl);
  const size_t nk = sizeof(float) * (size_t)h->n * h->k;
  float *dsts[4] = {h->H[h->cur], h->A, h->M, h->mu};
  for (int i = 0; i < 4; ++i) {
    CK(cudaMemcpyAsync(h->tmp, p, nk, cudaMemcpyHostToDevice, h->stream));
    CK(launch_pack(h->tmp, dsts[i], h->n, h->k, h->kp, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    p += nk;
  }
  h->ctrl = c;
  h->trace.clear();
  h->copied_upto = c.t;
  h->bad = false;
  h->err.clear();
  int rc = refresh_derived(h);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return SYMNMF_OK;
}

uint64_t symnmf_splitmix64(uint64_t state, uint64_t index) {
  return mix64(state + (index + 1) * kGamma);
}

int symnmf_sample_blocks(uint64_t seed, int64_t t, int32_t stream, int64_t nb, int64_t m,
                         int64_t *out) {
  if (!out || nb < 1 || m < 0 || t < 0) return SYMNMF_ERR_INVALID;
  std::vector<int64_t> v;
  sample(seed, t, stream, nb, m, v);
  std::copy(v.begin(), v.end(), out);
  return SYMNMF_OK;
}

int symnmf_controller_check(symnmf_ctrl *c, const symnmf_hparams *hp, int64_t n, int64_t t,
                            double E, double kkt, double sumA, double median_g2,
                            int32_t *decisions, double *stag_ratio) {
  if (!c || !hp || !decisions || n < 1 || t < 0) return SYMNMF_ERR_INVALID;
  CheckOut o;
  ctrl_check(c, hp, n, t, E, kkt, sumA, [&]() { return median_g2; }, &o);
  decisions[0] = o.converged;
  decisions[1] = o.reset;
  decisions[2] = o.grow;
  if (stag_ratio) *stag_ratio = o.ratio;
  return SYMNMF_OK;
}

}  // extern "C"
