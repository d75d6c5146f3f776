/*
 * symnmf.h -- C ABI of the GB300 SymNMF solver hot path.
 *
 * Problem (Sec. 2, Eq. 1): given a symmetric, entrywise non-negative
 * S in R^{n x n}, minimise f(H) = ||S - H H^T||_F^2 over H in R_+^{n x k}.
 * The library evaluates f through the trace identity of Eq. 2,
 *     f(H) = ||S||_F^2 - 2 tr(H^T S H) + ||H^T H||_F^2,
 * and the gradient of Sec. 2.1, grad f = 4 (H (H^T H) - S H), without ever
 * forming an n x n intermediate, and runs the projected adaptive solvers of
 * the appendix (Family 3) with the stopping rule of Sec. 4.1.
 *
 * Conventions shared by every call:
 *  - Device pointers are CUDA device addresses on the current device; host
 *    pointers are ordinary process memory.  Each argument says which.
 *  - S is BORROWED: the caller keeps it alive and unmodified until
 *    symnmf_destroy.  It is never copied.  Every other buffer (H ping-pong,
 *    optimizer state, snapshot, partial sums, diagnostics) is owned by the
 *    handle and freed by symnmf_destroy.
 *  - Work is ordered on the handle's stream (symnmf_set_stream; default the
 *    legacy default stream).  Calls that return host scalars synchronise
 *    that stream before returning; the others only enqueue.
 *  - Every call returns a symnmf_status; nothing throws across the ABI.
 *    SYMNMF_ERR_INVALID / SYMNMF_ERR_UNSUPPORTED leave the handle unchanged
 *    and usable.  SYMNMF_ERR_CUDA, _TIMEOUT and _NONFINITE put the handle in
 *    an error state in which solver calls return SYMNMF_ERR_STATE until
 *    symnmf_set_H or symnmf_set_state.  symnmf_last_error gives the text.
 *  - Handles are not thread-safe; distinct handles may be used from
 *    distinct threads.
 */
#ifndef SYMNMF_H
#define SYMNMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct symnmf_ctx *symnmf_t;

/* Storage type of S.  FP32: 4-byte IEEE.  BF16: bfloat16.  FP8E4M3: OCP
 * E4M3 (bias 7, max 448) with one FP32 scale per 128 x 128 tile, so that
 * S_ij = scale[i/128][j/128] * q_ij (symnmf_set_tile_scales). */
enum symnmf_dtype { SYMNMF_F32 = 0, SYMNMF_BF16 = 1, SYMNMF_FP8E4M3 = 2 };

/* Solvers (appendix, Family 3; Sec. 5.1). */
enum symnmf_method {
  SYMNMF_ADAGRAD = 0,             /* G += g*g; H = [H - eta g/(sqrt(G)+eps)]_+      */
  SYMNMF_RMSPROP = 1,             /* v = a v + (1-a) g*g; m = mu m + eta g/(sqrt(v)+eps); H = [H - m]_+ */
  SYMNMF_PIECEWISE_ADAGRAD = 2,   /* AdaGrad + stagnation-triggered accumulator reset */
  SYMNMF_ROW_SVRG = 3,            /* fresh rows on sampled I, snapshot mu elsewhere   */
  SYMNMF_BLOCK_SVRG_ADAPTGROW = 4, /* I x J block estimate, snapshot elsewhere, phi growth */
  SYMNMF_ADMM = 5                  /* appendix, Family 6: H = (2 S W + rho (W - U)) (2 W^T W + rho I)^-1,
                                      W = [H + U]_+, U += H - W; the handle's H is W, its
                                      accumulator buffer holds U; f, E and the check use W */
};

enum symnmf_status {
  SYMNMF_OK = 0,
  SYMNMF_CONVERGED = 1,        /* informative: the AND rule (Eq. 11) held at a check */
  SYMNMF_ERR_INVALID = -1,     /* null pointer, n < 1, bad enum, bad size            */
  SYMNMF_ERR_UNSUPPORTED = -2, /* k outside 1..64, S row stride not 16-byte aligned for the tensor-core path, ... */
  SYMNMF_ERR_OOM = -3,         /* a device or pinned allocation failed              */
  SYMNMF_ERR_CUDA = -4,        /* a CUDA runtime call failed                         */
  SYMNMF_ERR_TIMEOUT = -5,     /* a bounded device wait gave up                      */
  SYMNMF_ERR_NONFINITE = -6,   /* a NaN/Inf appeared in the gradient                 */
  SYMNMF_ERR_STATE = -7        /* the handle is in an error state                    */
};

/* Handle-owned n x k buffers that tests and checkpoints can read/write.
 * All are FP32, row-major n x k (row pitch k) in caller memory. */
enum symnmf_buffer {
  SYMNMF_BUF_H = 0,        /* current factor H_t                                    */
  SYMNMF_BUF_ACC = 1,      /* AdaGrad accumulator G (RMSprop: second moment v)      */
  SYMNMF_BUF_MOM = 2,      /* RMSprop momentum m                                    */
  SYMNMF_BUF_SNAPSHOT = 3, /* SVRG snapshot mu                                      */
  SYMNMF_BUF_GRAD = 4      /* gradient g used by the last update (read-only)        */
};

/* Solver hyper-parameters (appendix, Family 3; Sec. 4.1; Tab. phase2_config).
 * symnmf_hparams_default fills the paper's Phase-1 anchors. */
typedef struct symnmf_hparams {
  int32_t method;          /* enum symnmf_method */
  int32_t check_interval;  /* delta of Eq. 10 (default 10)                       */
  int32_t warmup;          /* stagnation suppressed while t < warmup (default 50) */
  int32_t snapshot_period; /* s: full pass every s iterations (SVRG methods)    */
  int32_t block_rows;      /* sampling granularity in rows, multiple of 128     */
  int32_t reserved0;
  double eta;              /* learning rate                                     */
  double eps;              /* epsilon of sqrt(G)+eps (AdaGrad 1e-10, RMSprop 1e-8) */
  double alpha;            /* RMSprop EMA factor                                */
  double mu;               /* RMSprop momentum                                  */
  double c;                /* Piecewise reset scale                             */
  double c_r;              /* Piecewise gradient-margin multiplier              */
  double row_frac;         /* Row-SVRG |I|/n                                    */
  double phi0;             /* Block-SVRG initial entry fraction                 */
  double tau_E;            /* loss gate (Eq. 7), default 0.1                    */
  double tau_g;            /* KKT gate (Eq. 8); <= 0 selects tau_g(n) of Eq. 9   */
  double tau_stag;         /* stagnation threshold tau of Eq. 10, default 1e-5  */
  double growth_kkt_mult;  /* AdaptGrow grows only while KKT > mult * tau_g (3) */
  uint64_t seed;           /* sampling seed (SplitMix64 counter streams)        */
  double rho;              /* ADMM penalty (default 500)                        */
} symnmf_hparams;

/* Scalar controller state carried between iterations (part of a checkpoint). */
typedef struct symnmf_ctrl {
  int64_t t;               /* next iteration index                              */
  double E0;               /* E at H_0 (NaN until the first check)              */
  double E_prev;           /* E at the previous check                           */
  double phi;              /* Block-SVRG entry fraction                         */
  double sumA_post;        /* Piecewise: sum(G) right after the last reset       */
  double E_at_reset;       /* Piecewise: E at the last reset                     */
  int32_t have_prev;
  int32_t stag_count;      /* consecutive stagnating checks (AdaptGrow)          */
  int32_t resets;          /* Piecewise resets fired                             */
  int32_t resets_enabled;
  int32_t cooldown;
  int32_t converged;
} symnmf_ctrl;

/* One iteration's diagnostics (Sec. 4.1, "At each check interval ..."). f,
 * E and kkt are those of H_t, the iterate the step started from; they are
 * NaN for sampled (non-full) iterations. */
typedef struct symnmf_record {
  int64_t t;
  double f, E, kkt;        /* objective, E_t = f/||S||^2, ||grad_proj||_F/(nk)  */
  double stag_ratio;       /* (E_{t-delta} - E_t)/E_0 at checks, else NaN        */
  double phi;              /* entry fraction used by iteration t                */
  double sumA;             /* sum of the accumulator after the update           */
  int32_t full, check, reset, converged;
  int32_t nonfinite;       /* NaN/Inf gradient entries seen                     */
  int32_t reserved;
  double median_g2;        /* Piecewise: lower median of the n*k values g_t^2 (FP32,
                              radix-selected) when this check evaluated it, else NaN */
} symnmf_record;

typedef struct symnmf_stats {
  int64_t iter;            /* ctrl.t after the call                             */
  int64_t last_check;      /* iteration of the last check (-1 if none)          */
  double f, E, kkt, stag_ratio, phi;  /* at the last check                      */
  int32_t converged, resets;
} symnmf_stats;

/* ---------------------------------------------------------------- handles */

/* Create a handle for S (device, n x n, row pitch n elements, dtype) and
 * rank k.  Computes ||S||_F^2 in FP64 (a single streaming pass; for FP8 at
 * symnmf_set_tile_scales).  Returns INVALID for n < 1 or null S/out,
 * UNSUPPORTED for k outside 1..64. */
int symnmf_create(const void *S, int64_t n, int32_t k, int32_t dtype, symnmf_t *out);
/* As symnmf_create with an explicit row pitch lds >= n (elements).  The
 * tensor-core path needs lds * sizeof(element) to be a multiple of 16 bytes
 * and S 16-byte aligned; otherwise the handle uses the SIMT product. */
int symnmf_create_ld(const void *S, int64_t n, int64_t lds, int32_t k, int32_t dtype,
                     symnmf_t *out);
void symnmf_destroy(symnmf_t h);
/* stream: a cudaStream_t passed as void* (NULL = legacy default stream). */
int symnmf_set_stream(symnmf_t h, void *stream);
/* FP8 only: scales (device, FP32, ceil(n/128) x ceil(n/128), row pitch
 * ld_scales) with S_ij = scales[i/128][j/128] * q_ij.  Borrowed like S.
 * Recomputes ||S||^2 from the dequantised values. */
int symnmf_set_tile_scales(symnmf_t h, const float *scales, int64_t ld_scales);
/* FP8 E4M3 storage of a matrix (all of S, or a band of its rows) with one
 * power-of-two scale per 128 x 128 tile.  Storage format of this library
 * (the paper runs FP32; Sec. 2.1 only needs S H and ||S||_F^2 from S).
 * For each tile: scale = the smallest power of two with
 * max|tile| / scale <= 448 (1 for an all-zero tile) and
 * q_ij = e4m3(S_ij / scale), rounded to nearest even (|S_ij| / scale <= 448,
 * so nothing saturates; S_ij / scale is exact).  Inputs (device): src,
 * rows x cols values of src_dtype (SYMNMF_F32 or SYMNMF_BF16) with row
 * pitch ld_src elements.  Outputs (device, caller-owned): q, rows x cols
 * bytes with row pitch ldq; scales, ceil(rows/128) x ceil(cols/128) FP32
 * with row pitch ld_scales; tile_sumsq (may be NULL), the FP64 sum of
 * squares of each unquantised tile in the layout of scales (for
 * symnmf_set_norm).  Tiles start at the band's first row and column, so a
 * band of a larger S must start at a multiple of 128 rows.  Asynchronous on
 * stream (cudaStream_t as void*, NULL = legacy default stream).  INVALID for
 * null q/src/scales, rows or cols < 1, a pitch below its width or another
 * src_dtype; UNSUPPORTED for more than 65535 row tiles in one call; CUDA
 * for a launch failure. */
int symnmf_quantize_fp8(const void *src, int32_t src_dtype, int64_t rows, int64_t cols,
                        int64_t ld_src, uint8_t *q, int64_t ldq, float *scales, int64_t ld_scales,
                        double *tile_sumsq, void *stream);
/* Override / read ||S||_F^2 used by the objective (e.g. the norm of the
 * unquantised matrix when S is stored in BF16 or FP8). */
int symnmf_set_norm(symnmf_t h, double normS2);
int symnmf_get_norm(symnmf_t h, double *normS2);
/* Force the product implementation: 0 = automatic, 1 = SIMT, 2 = tensor
 * core (UNSUPPORTED if the layout does not allow it). */
int symnmf_set_impl(symnmf_t h, int32_t impl);
int symnmf_get_impl(symnmf_t h, int32_t *impl);

/* ------------------------------------------------------------ the factor */

/* H (device, FP32, n x k row-major) becomes H_0; optimizer state, snapshot
 * and controller are reset (G = v = m = mu = 0, t = 0). */
int symnmf_set_H(symnmf_t h, const float *H);
/* Copy the current factor to H (device, FP32, n x k). */
int symnmf_get_H(symnmf_t h, float *H);
/* One solve from host memory, the call for data that lives on the host:
 * copies S (host, n rows of row pitch lds_host elements of the handle's
 * storage type; FP8: also its tile scales, host, ceil(n/128) rows of pitch
 * ld_scales_host) into the device buffers the handle was created on, which
 * it overwrites; takes normS2 > 0 as ||S||^2, else computes it from the
 * copied S as symnmf_create does; copies H_0 (host, n x k row-major FP32)
 * and starts from it as symnmf_set_H; runs up to iters iterations as
 * symnmf_step (stats: host, may be NULL); copies the final H (the certified
 * iterate on convergence) to H_out (host, n x k).  Pinned host buffers make
 * the copies asynchronous DMA on the handle's stream; pageable ones are
 * staged by the driver.  Synchronises before returning.  Returns OK or
 * CONVERGED.  Errors: INVALID for a null pointer, iters < 0, lds_host < n,
 * or FP8 without scales (host, or set on the handle) or with ld_scales_host
 * < ceil(n/128); otherwise those of symnmf_step. */
int symnmf_solve_host(symnmf_t h, const void *S_host, int64_t lds_host, const float *scales_host,
                      int64_t ld_scales_host, double normS2, const float *H0_host,
                      const symnmf_hparams *hp, int32_t iters, float *H_out, symnmf_stats *stats);
/* Read / write one handle buffer (enum symnmf_buffer) from / to device
 * memory (FP32 n x k).  Writing SYMNMF_BUF_H replaces H_t without touching
 * the optimizer state (teacher forcing); SYMNMF_BUF_GRAD is read-only. */
int symnmf_get_buffer(symnmf_t h, int32_t which, float *dst);
int symnmf_set_buffer(symnmf_t h, int32_t which, const float *src);
int symnmf_get_ctrl(symnmf_t h, symnmf_ctrl *out);
int symnmf_set_ctrl(symnmf_t h, const symnmf_ctrl *in);

/* ------------------------------------------------------------ the hot path */

/* G (device, FP32, n x k) = 4 (H (H^T H) - S H) at the current H (Sec. 2.1).
 * No state changes. */
int symnmf_grad(symnmf_t h, float *G);
/* f (host) = ||S||^2 - 2 tr(H^T S H) + ||H^T H||^2 at the current H (Eq. 2),
 * tr and the Gram reduced in FP64 across tiles; E (host) = f / ||S||^2.
 * Either pointer may be NULL. */
int symnmf_objective(symnmf_t h, double *f, double *E);
/* Fill hp with the paper's anchors for method (appendix; Sec. 5.1). */
int symnmf_hparams_default(int32_t method, symnmf_hparams *hp);
/* Run up to iters iterations of hp->method from the handle's state.  Checks
 * (every check_interval iterations) evaluate the AND rule of Eq. 11 and the
 * method's control (Piecewise reset, AdaptGrow growth).  Returns
 * SYMNMF_CONVERGED when the rule holds; the handle's H is then the certified
 * iterate H_t.  stats (host) may be NULL. */
int symnmf_step(symnmf_t h, const symnmf_hparams *hp, int32_t iters, symnmf_stats *stats);
/* Step count handles together: each iteration of every live handle is
 * launched on the handle's own stream before any of them is checked, so
 * the handles' kernels overlap on the GPU; one host loop.  hps and
 * outs are arrays of count (outs may be NULL).  Returns the first error, or
 * SYMNMF_OK; per-handle convergence is in outs[i].converged. */
int symnmf_batch_step(symnmf_t *hs, int32_t count, const symnmf_hparams *hps, int32_t iters,
                      symnmf_stats *outs);
/* Cap the CTAs of the handle's tensor-core launches (0 = one per SM, the
 * default).  Several handles with small caps on different streams run
 * their iterations side by side (batching: symnmf_batch_step).  This
 * library's scheduling knob; the paper runs one solve at a time. */
int symnmf_set_ctas(symnmf_t h, int32_t ctas);
/* The CTA count the handle's launches use (host). */
int symnmf_get_ctas(symnmf_t h, int32_t *ctas);
/* Autotune the CTA caps of a batch of handles (each on its own stream):
 * tries every handle on all SMs, then shares m * SMs * w_i / sum(w) for
 * m = 1, 2, 4 (w_i = bytes of S the handle streams per iteration), each
 * for iters real iterations of symnmf_batch_step (they advance the solves),
 * and keeps the schedule with the most iterations per second.  ctas_out
 * (host, count entries, may be NULL) receives the chosen caps. */
int symnmf_batch_autotune(symnmf_t *hs, int32_t count, const symnmf_hparams *hps, int32_t iters,
                          int32_t *ctas_out);
/* Time every product-kernel launch (the S H stream, the dominant kernel)
 * with a CUDA event pair on the handle's stream.  enable != 0 starts a new
 * accumulation; enable == 0 stops recording. */
int symnmf_set_profiling(symnmf_t h, int32_t enable);
/* Synchronise the stream and return the accumulated product-kernel time in
 * milliseconds (host), the number of timed launches, the algorithmic bytes
 * of S those launches streamed (rows x columns x element size), and the
 * number of kernels of this library that symnmf_step / symnmf_batch_step
 * launched while profiling was on (product, epilogue, reductions, median,
 * reset).  Any output pointer may be NULL. */
int symnmf_get_profile(symnmf_t h, double *product_ms, int64_t *launches, double *s_bytes,
                       int64_t *kernel_launches);
/* Copy up to max per-iteration records (oldest first) to out (host) and the
 * number available to *count.  The handle keeps the last 1<<20 records. */
int symnmf_get_trace(symnmf_t h, symnmf_record *out, int64_t max, int64_t *count);

/* ------------------------------------------------------------ checkpoints */

/* Size in bytes of a checkpoint blob (controller + H, G/v, m, mu). */
int symnmf_state_bytes(symnmf_t h, size_t *bytes);
/* Serialise into / restore from a host buffer of symnmf_state_bytes bytes.
 * Restoring clears an error state. */
int symnmf_get_state(symnmf_t h, void *buf, size_t bytes);
int symnmf_set_state(symnmf_t h, const void *buf, size_t bytes);

/* ------------------------------------------- objective without allocation */

/* Size of the fixed device scratch of symnmf_objective_noalloc (8 MiB). */
#define SYMNMF_NOALLOC_SCRATCH_BYTES (8u << 20)

/* f (device, one double) = normS2 - 2 tr(H^T S H) + ||H^T H||_F^2, the
 * objective ||S - H H^T||_F^2 without the n x n residual, for a caller's S
 * and H, with no handle and no device allocation.  The paper has no
 * counterpart; this library adds it for callers that cannot
 * allocate at the moment they need an objective: a monitor thread that
 * must not stall a running solve (cudaMalloc and cudaFree can synchronise
 * the device), a process whose device memory is fully reserved by another
 * allocator, or an application that promised its host a fixed device
 * footprint.  Its scratch is one array of SYMNMF_NOALLOC_SCRATCH_BYTES in
 * device memory, created with the library's module on each device, so a
 * call only launches kernels (three).
 * Arguments: S (device, n x n, row pitch lds >= n elements, storage dtype;
 * FP8 also takes the tile scales of symnmf_set_tile_scales, else scales
 * may be NULL), H (device, FP32, n x k with row pitch k, 1 <= k <= 64),
 * normS2 = ||S||_F^2 (for example from symnmf_get_norm), f (device, one
 * double, written).  Nothing is kept after the call's kernels finish.
 * Arithmetic: S H by FP32 FMA; tr and the Gram summed across 128-row tiles
 * in FP64 in a fixed order, so the same inputs give the same bits.
 * Limit: the call needs ceil(n/128) * (64 + 4 kp^2) bytes of scratch (kp =
 * k rounded up to 8, 16, 32 or 64; plus under 256 bytes of alignment), at
 * most SYMNMF_NOALLOC_SCRATCH_BYTES: n <= 3,355,392 for kp = 8, 986,880 for
 * kp = 16, 258,048 for kp = 32, 65,280 for kp = 64.  A larger call returns
 * SYMNMF_ERR_UNSUPPORTED and launches nothing.
 * Zero state: no part of the scratch has to start at zero; every slot the
 * last kernel reads is written earlier in the same call.
 * Set-up: the first call on each device does that device's set-up, with
 * that device current: looking up the scratch address (cudaGetSymbolAddress)
 * loads this library's module on the device, which creates the scratch
 * array and may synchronise the device, and the call then loads every
 * kernel it can launch (with lazy module loading each would otherwise load
 * at its first launch, inside a later call).  So make the first call at
 * set-up time, before any stream capture begins and before the code that
 * must not allocate runs; from then on a call only launches kernels.
 * Concurrency: all calls on one device share the one scratch, so calls
 * whose kernels can overlap in time (different streams, or host threads
 * without an order between them) race and give wrong values; order them,
 * for example on one stream.  Asynchronous on stream (cudaStream_t as
 * void*, NULL = legacy default stream).
 * Errors: INVALID for null S/H/f, n < 1, lds < n, k outside 1..64, an
 * unknown dtype, or FP8 without scales or with ld_scales < ceil(n/128);
 * UNSUPPORTED for the scratch limit above; CUDA for a failed launch or
 * look-up. */
int symnmf_objective_noalloc(const void *S, int64_t n, int64_t lds, int32_t dtype,
                             const float *scales, int64_t ld_scales, const float *H, int32_t k,
                             double normS2, double *f, void *stream);
/* Host-only check of symnmf_objective_noalloc's arguments, with no CUDA
 * call: returns the status that entry point returns for these sizes before
 * it launches anything (OK, INVALID or UNSUPPORTED; have_scales says
 * whether a scales pointer would be passed) and, when need is not NULL,
 * the scratch bytes such a call uses (also set when the size is beyond the
 * limit).  Lets a caller size its problems ahead of time. */
int symnmf_objective_noalloc_check(int64_t n, int64_t lds, int32_t dtype, int32_t have_scales,
                                   int64_t ld_scales, int32_t k, size_t *need);

/* Independent restarts concatenated along N: a handle of rank k with
 * restarts = R (k divisible by R) runs R solves of rank k / R on the same S
 * from one stream of S per iteration.  Column block r of H (columns
 * r k/R .. (r+1) k/R - 1) is restart r.  The Gram H^T H is kept block
 * diagonal (the entries between different blocks are set to 0 when it is
 * reduced), so H Gram gives each block its own H_r (H_r^T H_r) and every
 * update (AdaGrad, RMSprop, ADMM's k x k inverse) acts on each restart
 * alone; the gradient, objective, KKT measure and stopping rule are those
 * of the concatenated problem: f = sum_r f_r, E = f / (R ||S||^2) (the
 * restarts' mean E), ||grad_proj|| over all blocks, divided by n k.  At
 * every check each restart also gets its own E_r and KKT measure (from the
 * gradient the step wrote: f_r = ||S||^2 - ||Gram_rr||^2 + sum(H_r .* g_r) / 2)
 * and its own AND rule (Eq. 11); the handle stops (SYMNMF_CONVERGED) when
 * the concatenated problem or any restart meets it, with H_t kept.
 * Piecewise AdaGrad resets each restart on its own (appendix, Family 3): at
 * a check the restart's stagnation, KKT gate, loss-reduction test and
 * cooldown use its E_r, KKT measure and sum(A_r), the median is that of
 * g_r^2 over its n k/R entries, and only its columns of A are reset (the
 * handle's own controller makes no reset; the record's reset flag says
 * whether any restart reset).  No restart resets at a check where the handle
 * stops.  Call before stepping; the current H's Gram is recomputed.
 * Default 1.  The per-restart check state (each restart's E0, previous E
 * and reset state) is not part of the checkpoint blob: after
 * symnmf_set_state it starts again at the next check.
 * Errors: INVALID for restarts < 1 or > 8 or k not divisible by restarts;
 * OOM when the check scratch cannot be allocated. */
int symnmf_set_restarts(symnmf_t h, int32_t restarts);
/* E, KKT measure and converged flag of each restart at the last check (host
 * arrays of count >= restarts entries, any may be NULL); with one restart
 * the handle's own. */
int symnmf_get_restart_stats(symnmf_t h, int32_t count, double *E, double *kkt,
                             int32_t *converged);
/* Piecewise AdaGrad reset state of each restart (host arrays of count >=
 * restarts entries, any may be NULL): resets fired, resets still enabled,
 * cooldown running, sum(A_r) right after its last reset; with one restart
 * the handle's own controller.  Errors: INVALID for a null handle or
 * count < restarts. */
int symnmf_get_restart_ctrl(symnmf_t h, int32_t count, int32_t *resets, int32_t *resets_enabled,
                            int32_t *cooldown, double *sumA_post);

/* Rolling windows: rebind the handle to another matrix S of the same n and
 * storage type (device, row pitch lds >= n; FP8 also takes its tile scales,
 * else scales may be NULL) without reallocating.  The handle first waits
 * for its stream, so the previous matrix may be overwritten after the call
 * returns.  H, its MMA copy and its Gram are kept as the warm start of the
 * new problem; the optimizer state, the snapshot, the gradient buffer, the
 * controller and the trace start afresh, and ||S||^2 (and the K-means row
 * norms, if computed) are recomputed for the new matrix.  The paper names
 * rolling-window solves as future work (Sec. 8); this is the library's
 * warm-start primitive for them.
 * Errors: INVALID for a null S, lds < n, or FP8 without scales or with
 * ld_scales < ceil(n/128); CUDA as for the other calls. */
int symnmf_set_matrix(symnmf_t h, const void *S, int64_t lds, const float *scales,
                      int64_t ld_scales);

/* ------------------------------------------------- dependence matrix */

/* The solver's input from data (Sec. 3, "Correlation matrices" and the
 * empirical TPDM): S = |D^-1/2 G D^-1/2| with G = Y^T Y and D = diag(G),
 * i.e. S_ij = |G_ij| / sqrt(G_ii G_jj), S_ii = 1, clamped to [0, 1].
 * center = 1 subtracts each column's mean first, giving the absolute
 * Pearson correlation of the n variables over the T observations (rows of
 * Y); center = 0 with Y = Omega, the n_exc x n matrix of exceedance angles,
 * gives the unit-diagonal empirical TPDM (its n / n_exc factor cancels).
 * Arguments: Y (device FP32, T x n, row pitch ldy >= n elements), S
 * (device, n x n, row pitch lds >= n elements, 16-byte aligned with
 * lds * element size a multiple of 16) written in out_dtype (SYMNMF_F32,
 * SYMNMF_BF16 round to nearest, or SYMNMF_FP8E4M3 with one power-of-two
 * scale per 128 x 128 tile written to scales[ceil(n/128)][ld_scales], the
 * layout of symnmf_set_tile_scales), normS2 (device, one double, or NULL):
 * ||S||_F^2 (of the stored values for F32 / BF16, of the values before
 * quantisation for FP8), summed in FP32 over runs of 32 entries of a row
 * and in FP64 across runs (relative error below 32 * 2^-24).  stream: cudaStream_t as void* (NULL =
 * legacy default); the call synchronises it once at the end.
 * Arithmetic: the centred values are FP32; G is formed on the tensor cores
 * from tf32 hi / lo pieces of each value (hi hi + hi lo + lo hi, FP32
 * accumulation), about FP32 accuracy; column norms are FP64.  A column with
 * zero variance gives a zero row and column in S except S_ii = 1.
 * Scratch: n (8 T' + 12) + ceil(n/128) ceil(n/256) 8 bytes of stream-ordered
 * device memory (T' = T rounded up to 32), freed before return.
 * Errors: INVALID for null pointers, T < 1 (T < 2 with center), n < 1,
 * pitches below n, a misaligned S or pitch, an unknown out_dtype, or FP8
 * without scales or with ld_scales < ceil(n/128); UNSUPPORTED for n above
 * 2,097,120; OOM when the scratch cannot be allocated; TIMEOUT when a
 * bounded device wait gave up; CUDA for other failures. */
int symnmf_build_dependence(const float *Y, int64_t T, int64_t n, int64_t ldy, int32_t center,
                            int32_t out_dtype, void *S, int64_t lds, float *scales,
                            int64_t ld_scales, double *normS2, void *stream);

/* The next window of a rolling solve (Sec. 8, streaming SymNMF over rolling
 * windows; Sec. 3 for S) in one call on the handle's stream: the dependence
 * matrix of the window Y (as symnmf_build_dependence, in the handle's
 * storage type) is written into S, the handle is rebound to it (as
 * symnmf_set_matrix: H kept as the warm start, the optimizer state,
 * controller and trace fresh), and ||S||^2 is taken from the build's own
 * epilogue rather than from a second pass over S (FP32 / BF16: the stored
 * values' squares summed as float-float pairs over runs of 32 entries,
 * about 2^-44 relative, and in FP64 across runs; with FP8 storage, whose
 * build sums the values before quantisation, it is recomputed from the
 * stored codes).  S may be the buffer the handle reads
 * now: the build is ordered after the handle's earlier launches.  The
 * next symnmf_step is the window's first solver step.
 * Arguments: Y (device FP32, T x n, pitch ldy >= n, n the handle's), center
 * (1: absolute correlation, 0: TPDM from exceedance angles), S (device, n x
 * n, pitch lds >= n, the alignment symnmf_build_dependence asks for), FP8:
 * scales / ld_scales as there, else NULL / 0.  Synchronises the handle's
 * stream once.
 * Errors: those of symnmf_build_dependence and symnmf_set_matrix. */
int symnmf_window_update(symnmf_t h, const float *Y, int64_t T, int64_t ldy, int32_t center,
                         void *S, int64_t lds, float *scales, int64_t ld_scales);

/* ------------------------------------------------ spherical K-means */

typedef struct {
  int32_t iters;      /* Lloyd iterations this call ran */
  int32_t converged;  /* 1: the stop rule held at the last iteration */
  int64_t changed;    /* labels the last iteration changed */
  double J;           /* objective of the last iteration, sum_i (1 - max_k cos_ik) */
  double J_prev;      /* the iteration before it (NaN after a single iteration) */
} symnmf_kmeans_stats;

/* Spherical K-means (Lloyd) on the rows of S (Sec. 6, "Clustering
 * alternatives", the spherical K-means theorem), K = the handle's k
 * clusters.  The observations are the normalised rows x_i = s_i / ||s_i||;
 * cluster k's centroid is the normalised sum of its members,
 * c_k = sum_{i in C_k} x_i; an iteration assigns every row the cluster of
 * largest cosine <x_i, c_k / ||c_k||> (lowest index on ties; an empty
 * cluster has cosine 0 with every row) and J = sum_i (1 - that cosine).
 * The run stops after the first iteration that changes no label, or whose
 * relative drop (J_prev - J) <= tol * J_prev (the paper's criterion uses
 * tol = 1e-4), or after max_iter iterations.
 * One iteration is two passes of the streamed product (S symmetric):
 * C = S (D^-1 B) with D = diag ||s_i|| and B the one-hot labels, then
 * P = S C, with cos_ik = P_ik / (||s_i|| ||c_k||); FP32 products, FP64
 * norms and FP64 fixed-order cross-tile sums, so runs are bit-reproducible.
 * Arguments: labels0 (device, n int32, entries in 0..K-1; an entry outside
 * that range puts its row in no cluster for the first iteration), labels
 * (device, n int32, written: the final labels), max_iter >= 1, tol >= 0,
 * J_trace (host, max_iter doubles, J per iteration, or NULL), stats (host,
 * or NULL).  ||s_i|| is computed on the first call and kept (S is borrowed
 * and must not change); rows with ||s_i|| = 0 are not valid input.  The
 * solver state (H, its MMA copy, the Gram, the optimizer buffers) is not
 * touched; the call synchronises the handle's stream once per iteration.
 * Errors: INVALID for null labels, max_iter < 1 or tol < 0 or NaN; OOM when
 * the scratch (n (8 + 8) + ceil(n/128) (16 + 8 kp) bytes) cannot be
 * allocated; CUDA / STATE as for symnmf_step. */
int symnmf_spkmeans(symnmf_t h, const int32_t *labels0, int32_t *labels, int32_t max_iter,
                    double tol, double *J_trace, symnmf_kmeans_stats *stats);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * thread waits, with the bounded mbarrier wait the tensor-core kernels use,
 * on a barrier that nothing completes, for limit_s seconds (0 < limit_s <=
 * 10), on the legacy default stream, then the call synchronises the device.
 * Returns SYMNMF_ERR_TIMEOUT when the wait gave up and recorded its error
 * code (the expected outcome; the context stays usable), SYMNMF_OK if it
 * did not, INVALID for a limit out of range, CUDA for a failed launch. */
int symnmf_selftest_wait_timeout(double limit_s);

const char *symnmf_last_error(symnmf_t h);
const char *symnmf_status_string(int32_t status);

/* ---------------------------------------------- host-only pure functions */

/* SplitMix64 (Steele, Lea & Flood 2014): the (index+1)-th output of the
 * generator started at state. */
uint64_t symnmf_splitmix64(uint64_t state, uint64_t index);
/* m distinct sorted block indices of 0..nb-1 drawn for iteration t on a
 * stream (0: Row-SVRG I; 1, 2: Block-SVRG I, J) by a partial Fisher-Yates
 * shuffle whose d-th swap partner is d + u_d mod (nb - d), u_d the d-th
 * output started at seed*0x9E3779B97F4A7C15 + t*0xBF58476D1CE4E5B9 +
 * stream*0x94D049BB133111EB.  out (host) holds m entries. */
int symnmf_sample_blocks(uint64_t seed, int64_t t, int32_t stream, int64_t nb, int64_t m,
                         int64_t *out);
/* The controller's decision at a check (Sec. 4.1 AND rule; Piecewise reset
 * and AdaptGrow growth control), as a pure function for replay: updates
 * *c in place given iteration t, E_t, the KKT norm, sum(G) and the lower
 * median of g_t^2.  decisions[0..2] (host) receive converged, reset, grow;
 * *stag_ratio the stagnation ratio (may be NULL). */
int symnmf_controller_check(symnmf_ctrl *c, const symnmf_hparams *hp, int64_t n, int64_t t,
                            double E, double kkt, double sumA, double median_g2,
                            int32_t *decisions, double *stag_ratio);

#ifdef __cplusplus
}
#endif
#endif /* SYMNMF_H */
