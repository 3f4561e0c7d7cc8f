/*
 * slse.h - C ABI of the GB300 (sm_103a) implementation of SLSE-FRS, the
 * "Sequential Least-Squares Estimators with Fast Randomized Sketching" method
 * (arXiv 2509.06856).
 *
 * Problem (paper Sec. 1): given tall data X (N x d, N >> d, full column rank) and
 * Y (N), return the OLS estimator beta-hat = argmin 1/2 ||Y - X beta||^2.
 * SLSE-FRS (Algorithm 2, Sec. 3) forms one randomized Hadamard transform of
 * [X | Y], takes nested row samples of growing size m_1 < ... < m_K from it, runs
 * a_i momentum-IHS (M-IHS) steps on each sketched subproblem (1st stage, Eq. (7))
 * and finishes with full-data M-IHS steps (2nd stage, Eq. (8)).  Every M-IHS step
 * is preconditioned by the fixed sketched Hessian H-hat = (S-hat X)^T (S-hat X),
 * applied through the R factor of a QR of S-hat X (Appendix, implementation
 * details).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are row-major.  X has leading dimension ldx >= d (elements).
 * - Pointers named "device" must be CUDA device (or managed) memory of the
 *   current device; the call enqueues its kernels on `stream` (0 = legacy
 *   default stream).  Pointers named "host" are ordinary host memory.
 * - Workspace: `workspace` is caller-owned device memory of `ws_bytes` bytes,
 *   aligned to 256 bytes.  If `workspace` is NULL the library allocates the
 *   workspace itself with cudaMallocAsync on `stream` and frees it before
 *   returning (stream-ordered).  If `workspace` is not NULL and `ws_bytes` is
 *   smaller than slse_workspace_size(...), the call returns SLSE_ENOMEM and
 *   launches nothing.
 * - Errors are returned as slse_status codes; no C++ exception crosses the ABI.
 *   SLSE_EINVAL means an argument failed validation and nothing was launched.
 * - Same inputs + same seed => bit-identical random draws and sketch, and a
 *   deterministic estimate (all reductions have a fixed order).
 * - Gradient sign: g = X^T (Y - X beta), i.e. minus the paper's
 *   nabla f = X^T (X beta - Y) (Sec. 1); the M-IHS step adds mu H-hat^{-1} g.
 * - Limits of the library: 1 <= d <= 512, d <= N, N' = 2^ceil(log2 N) <= 2^24.
 */
#ifndef SLSE_H
#define SLSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *slse_stream_t; /* the same type as cudaStream_t */

typedef enum {
  SLSE_OK = 0,
  SLSE_EINVAL = 1,   /* invalid argument; nothing launched */
  SLSE_ENOMEM = 2,   /* workspace too small, or the internal allocation failed */
  SLSE_ECUDA = 3,    /* a CUDA runtime call failed */
  SLSE_ENOTCONV = 4, /* tol > 0 and the 2nd stage reached T first; beta_out holds the last iterate */
  SLSE_ENUMERIC = 5, /* NaN/Inf in an iterate, or a zero pivot in the QR */
  SLSE_ETIMEOUT = 6  /* a bounded device-side wait gave up (grid barrier in the QR kernel) */
} slse_status;

typedef enum { SLSE_F64 = 0, SLSE_F32 = 1, SLSE_BF16 = 2 } slse_dtype;

/* Sketch families.
 * SLSE_SRHT: subsampled randomized Hadamard transform (Sec. 3), the paper's method.
 * SLSE_COUNTSKETCH: the sparse projection of Sec. 2 (one random sign per column, in a
 *   uniformly random row), used in place of the SRHT in the SLSE-FRS-CS experiment of
 *   Sec. 5.  Row k of [X|Y] goes with sign s(k) to bucket h(k) mod m; h(k) and s(k) are
 *   word 0 and bit 0 of word 1 of Philox4x32-10 at counter (k, 3).  Sizes are powers of
 *   two, so a smaller sketch of the family is a fold of a larger one.  No scale factor
 *   (E[S^T S] = I).
 * SLSE_COUNTSKETCH_HAT: the independent CountSketch used for the Hessian sketch with the
 *   CountSketch family: m buckets (any m >= 1), bucket floor(w0 m / 2^32) and sign bit 0
 *   of w1 at counter (k, 4).
 * SLSE_GAUSSIAN: the Gaussian sketch of Sec. 2, S = G / sqrt(m) with i.i.d. standard normal
 *   G[i, k]: Philox4x32-10 at counter (q mod 2^32, q div 2^32, 5, i), q = k div 8, gives the
 *   entries G[i, 8q .. 8q+7]; output word j yields G[i, 8q+2j] = sqrt(-2 ln u1) cos(2 pi u2) and
 *   G[i, 8q+2j+1] = sqrt(-2 ln u1) sin(2 pi u2) (Box-Muller) with u1 = (w mod 2^16 + 1/2) 2^-16,
 *   u2 = (w div 2^16 + 1/2) 2^-16.  Used for the Hessian sketch only (a schedule of this kind
 *   keeps the SRHT subproblems).  MIXED_BF16: entries drawn in FP32 with the hardware log2,
 *   sine, cosine and reciprocal square root (absolute error below 1e-4, then BF16 rounding),
 *   products on the tensor cores with FP32 accumulation; FP64: entries and products in FP64. */
typedef enum { SLSE_SRHT = 0, SLSE_COUNTSKETCH = 1, SLSE_GAUSSIAN = 2, SLSE_COUNTSKETCH_HAT = 3 } slse_sketch_kind;

/* Arithmetic of the path.
 * SLSE_PREC_FP64: every step in FP64 (X stored F64 or F32; F32 values are widened exactly).
 * SLSE_PREC_MIXED_BF16: sketch applied in FP32 and stored in BF16; 1st-stage gradients on
 *   the BF16 sketch with FP32 accumulation; 2nd-stage residual-gradient in FP32 with
 *   error-free (TwoProd/TwoSum) residuals against an FP64 base point and two-sum
 *   compensated accumulation; QR, preconditioner and update in FP64.  Requires X F32. */
/* SLSE_PREC_MIXED_FP8: as MIXED_BF16, but the sampled sketch rows U are stored as E4M3 values
 *   with one power-of-two scale 2^k per 32-column block of a row (k + 127 in a byte; k is
 *   the smallest integer with max|block| <= 448 2^k), so the 1st-stage subproblems read one
 *   byte per element; the pass-1 intermediate and the sketch of Y stay BF16.  No paper
 *   counterpart (the paper's sketches are double precision).  Requires X F32, kind SRHT. */
typedef enum { SLSE_PREC_FP64 = 0, SLSE_PREC_MIXED_BF16 = 1, SLSE_PREC_MIXED_FP8 = 2 } slse_precision;

/* Form of the 2nd-stage passes (Eq. (8)) on the mixed precisions; ignored by SLSE_PREC_FP64.
 * SLSE_STAGE2_FULL: every 2nd-stage step streams X in FP32 (the compensated residual-gradient
 *   pass of SLSE_PREC_MIXED_BF16).
 * SLSE_STAGE2_CORRECTION: defect correction of the same iteration.  An exact pass (the FP32
 *   pass above) gives g(b_e) = X^T (Y - X b_e); the steps after it (correction steps) use
 *   g(b) = g(b_e) - G_b (b - b_e) with G_b = Xb^T Xb the Gram matrix of a BF16 copy Xb of X,
 *   formed once on the tensor cores before the 2nd stage: a d x d product per step instead of a
 *   pass over X.  The next exact pass comes when a step falls
 *   below 1/10^4 of the first step after the last exact pass, rises above it, is the 20th
 *   correction step of the cycle, or meets the
 *   stopping test; the iteration stops only on the step of an exact pass, so the stopping test
 *   and the fixed point (g(b) = 0, the least-squares estimate) are those of the full form.  When
 *   a cycle (an exact pass and k correction steps) shrinks the exact step by less than
 *   rho^(1 + k/50), rho = sqrt(d/r) (a correction step counted as 1/50 of a pass), i.e. less than
 *   full-form steps gain in that time, or by less than 10x (the BF16 Hessian term too coarse for
 *   an ill-conditioned X), the remaining steps take the full form.  No paper counterpart (the
 *   paper streams X in double precision); the workspace grows by the Gram stage's scratch
 *   (slse_workspace_size with SLSE_OP_GRAM gives it). */
typedef enum { SLSE_STAGE2_FULL = 0, SLSE_STAGE2_CORRECTION = 1 } slse_stage2_form;

typedef struct {
  int64_t N;       /* rows, N >= d */
  int32_t d;       /* columns, 1 <= d <= 512 */
  int32_t dtype;   /* slse_dtype of X and Y: SLSE_F64 or SLSE_F32 */
  const void *X;   /* N x d row-major, leading dimension ldx: device memory, or (slse_fit only)
                      host memory, pinned or pageable, which slse_fit copies into its workspace */
  int64_t ldx;     /* >= d */
  const void *Y;   /* N, same dtype and the same kind of memory as X */
} slse_problem;

typedef struct {
  int32_t K;            /* number of sketched subproblems (0 = no 1st stage) */
  const int64_t *m;     /* host, K ascending sketch sizes, 1 <= m_i <= N' */
  const int32_t *a;     /* host, K inner iteration counts a_i >= 0 */
  int64_t r;            /* Hessian sketch size, d <= r <= N' */
  double mu, eta;       /* M-IHS step and momentum */
  int32_t T;            /* cap on the total number of iterations (both stages) */
  double tol;           /* 2nd stage stops when ||b+ - b|| <= tol (1-rho)/rho ||b+||, rho = sqrt(d/r); <= 0: run to T */
  int32_t kind;         /* SLSE_SRHT, or SLSE_COUNTSKETCH: S_i X is the 2^l-bucket CountSketch
                           (all m_i powers of two, unscaled) and S-hat X the independent
                           r-bucket SLSE_COUNTSKETCH_HAT sketch, or SLSE_GAUSSIAN: SRHT
                           subproblems and S-hat X = G X / sqrt(r) from the r x N Gaussian
                           sketch (prec FP64 or MIXED_BF16) */
  int32_t prec;         /* slse_precision */
  int32_t momentum_reset; /* 0: momentum carries across subproblems (Algorithm 2's global t);
                             1: beta_{-1} = beta_0 at each subproblem and at the 2nd stage (proof of Thm 4.1) */
  int32_t stage2;       /* slse_stage2_form (mixed precisions; ignored by FP64) */
} slse_schedule;

typedef struct {
  double ms_copy_in;      /* host inputs only: CUDA-event time of the host-to-device copies on the side
                             stream (overlaps ms_draws): Y, and X unless the first SRHT pass reads it */
  double ms_draws, ms_sketch, ms_qr, ms_stage1, ms_stage2, ms_total; /* CUDA-event phase times */
  double ms_srht_pass1, ms_srht_pass2; /* the two sketch passes (pass 2 is 0 for single-pass sizes) */
  double ms_grad2;        /* summed CUDA-event time of the 2nd-stage gradient launches */
  int32_t n_grad2;        /* number of those launches that did a full pass */
  int32_t kernels;        /* kernel launches made by the call */
  int32_t iters_stage1, iters_stage2;
  double final_rel_step;  /* ||b_T - b_{T-1}|| / ||b_T|| of the last iteration */
  double bytes_moved;     /* algorithmic HBM bytes of the sketch passes and gradient passes */
  double bytes_grad2;     /* algorithmic HBM bytes of one 2nd-stage gradient pass */
  int32_t rebases;        /* mixed path: number of 2nd-stage residual re-bases (exact passes) */
  int32_t status;
  double ms_corr;         /* SLSE_STAGE2_CORRECTION: summed CUDA-event time of the correction steps (not
                             included in ms_grad2, which then covers the exact passes over X) */
  int32_t n_corr;         /* number of correction steps */
  int32_t stage2_full;    /* 1 if a correction run fell back to the full form */
  double ms_gram;         /* CUDA-event time of forming the Gram matrix of the BF16 rounding of X */
  double flops_gram;      /* its tensor-core FLOPs: the upper block triangle, 2 N' 128 sum_b (ncp - 128 b),
                             ncp = d rounded up to 128, N' = N rounded up to 32 (64 when packed) */
  double bytes_gram;      /* its algorithmic HBM bytes: X read, the per-range FP32 partials written and
                             read (and, for X not read directly, the packed BF16 copy written and read) */
} slse_report;

typedef struct {
  double *beta_hist;  /* device, cap x d: row t = iterate after iteration t+1 (NULL: none) */
  float *ms_hist;     /* host, cap: CUDA-event ms from the call's start to the end of iteration t+1 */
  int32_t cap;
  int32_t count;      /* out: iterations recorded */
  double *hinv_out;   /* device d x d (ld d), nullable: receives the H-hat^{-1} = R^{-1} R^{-T} the fit
                         used, the preconditioner slse_solve_normal takes */
} slse_trace;

/* Workspace query.  op: SLSE_OP_FIT (sched required), SLSE_OP_SKETCH (arg = m; prec and kind
 * from sched->prec and sched->kind if sched != NULL, else FP64 SRHT), SLSE_OP_GRAD, SLSE_OP_DRAWS (arg = N), SLSE_OP_QR
 * (arg = r), SLSE_OP_GRAM.  Returns 0 for invalid arguments. */
enum { SLSE_OP_FIT = 0, SLSE_OP_SKETCH = 1, SLSE_OP_GRAD = 2, SLSE_OP_DRAWS = 3, SLSE_OP_QR = 4, SLSE_OP_GRAM = 5 };
size_t slse_workspace_size(const slse_problem *prob, const slse_schedule *sched, int32_t op, int64_t arg);

/* Algorithm 2 end to end (paper Sec. 3).  seed selects the random draws D, P and the
 * sampling order (Philox4x32-10).  beta_out: host, d doubles.  report, trace: nullable.
 * Synchronous: returns after beta_out is written.  sched == NULL selects the paper's
 * experimental defaults (slse_default_schedule) in FP64.  With host X and Y the copy to the
 * device runs on a side stream while the random draws run on `stream`; the workspace then
 * also holds the device copy (slse_workspace_size accounts for it).  Pinned X with ldx == d
 * and a two-pass transform (N' > 512, SRHT or Gaussian kind) is not copied ahead: the first
 * SRHT pass reads its rows from host memory through the mapped address and stores the device
 * copy as it goes (each row is read once; the estimate is the same bits as from device
 * inputs).  Tracing: each phase's
 * enqueue is wrapped in an NVTX range ("slse_fit: draws", "...: sketch", "...: Hessian factor",
 * "...: stage 1", "...: stage 2"); with SLSE_LOG set in the environment every call prints a
 * one-line summary of its phase times (CUDA events) to stderr. */
slse_status slse_fit(const slse_problem *prob, const slse_schedule *sched, uint64_t seed,
                     double *beta_out, slse_report *report, slse_trace *trace,
                     void *workspace, size_t ws_bytes, slse_stream_t stream);

/* One sketch of size m.  kind SLSE_SRHT (Sec. 3): SX = sqrt(N'/m) * rows sigma[0..m) of
 * H D P X_pad / sqrt(N'), SY likewise.  kind SLSE_COUNTSKETCH (Sec. 2; m a power of two,
 * else SLSE_EINVAL): row b of SX is the signed sum of the rows of X in bucket b.  kind
 * SLSE_COUNTSKETCH_HAT: the same with the Hessian-sketch hash into m buckets.  kind SLSE_GAUSSIAN
 * (prec FP64, or MIXED_BF16 with X F32): SX = G X / sqrt(m), SY = G Y / sqrt(m), G m x N as
 * described at slse_sketch_kind (any 1 <= m < 2^31); SY may be NULL (not formed); a bounded
 * device wait that gave up leaves NaN in SX and SY.  prec FP64 ->
 * SX, SY are double; MIXED_BF16 -> bf16 (CountSketch sums accumulated in FP32, in row
 * order within a bucket, so the result is deterministic).  SX: device m x ldsx (ldsx >= d),
 * SY: device m.  prec MIXED_FP8 (kind SRHT): SX holds m x ldsx E4M3 bytes (ldsx a multiple of
 * 4, SX 4-byte aligned) followed by m x ceil(d/32) block-exponent bytes; SY is bf16.
 * Asynchronous on `stream`; the workspace size comes from
 * slse_workspace_size(SLSE_OP_SKETCH) with sched->kind and sched->prec set. */
slse_status slse_sketch(const slse_problem *prob, int32_t kind, int32_t prec, uint64_t seed, int64_t m,
                        void *SX, int64_t ldsx, void *SY, void *workspace, size_t ws_bytes,
                        slse_stream_t stream);

/* Residual-gradient pass g = X^T (Y - X beta) (Sec. 3, Eq. (8) and its FLOP count).
 * beta: device d doubles; g_out: device d doubles.  prec FP64: FP64 arithmetic.
 * prec MIXED_BF16 (X F32): error-free FP32 residuals and compensated accumulation.
 * Asynchronous on `stream`. */
slse_status slse_grad(const slse_problem *prob, const double *beta, double *g_out, int32_t prec,
                      void *workspace, size_t ws_bytes, slse_stream_t stream);

/* Residual-gradient pass that allocates nothing, for callers that cannot allocate device
 * memory when they need a gradient (host applications that own every device allocation
 * and hand out only fixed buffers, loops that forbid allocation after start-up).  The paper has no counterpart: this is a deployment variant of slse_grad.
 * Same arguments, result and tolerances as slse_grad, but its scratch (a status word and
 * per-CTA partial gradients, 1 MiB + 4 KiB) is a fixed array inside the library that
 * every GPU loading the library keeps until the process exits.  No cudaMalloc, cudaFree
 * or allocating library call is made.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current and loads the code of every
 * kernel this entry point can launch; make that first call before any stream capture.  A
 * cudaDeviceReset destroys the array, and the looked-up address goes stale with it: after a
 * reset, this entry point must not be called again in the same process.  All calls on a device share the one array: calls whose
 * work may overlap on the GPU (different streams without ordering) race and must not be
 * issued.  Each call clears the state it needs and overwrites every partial it reads.
 * Limit: the per-CTA partials must fit in 1 MiB (d <= 512 always fits; fewer CTAs are
 * used for large d); otherwise SLSE_ENOMEM.  Asynchronous on `stream`. */
slse_status slse_grad_noalloc(const slse_problem *prob, const double *beta, double *g_out, int32_t prec,
                              slse_stream_t stream);

/* Gram matrix G = Xb^T Xb (d x d, FP64, row-major, device) of the BF16 rounding Xb of X
 * (prob->dtype F32, device; or prob->dtype SLSE_BF16 with ldx a multiple of 8 and X 16-byte
 * aligned: G = X^T X of those values, Y unused but non-null): the Hessian term of the mixed 2nd
 * stage's correction form
 * (SLSE_STAGE2_CORRECTION; the Hessian X^T X of Sec. 1 with X rounded to BF16).  Products of BF16
 * values are exact in FP32; they are accumulated on the tensor cores in FP32 over ranges of rows
 * and the ranges are added in FP64 in a fixed order; the upper triangle is formed and mirrored, so
 * G is exactly symmetric.  Asynchronous on `stream`; workspace from
 * slse_workspace_size(SLSE_OP_GRAM).  No paper counterpart as an entry point. */
slse_status slse_gram(const slse_problem *prob, double *G, void *workspace, size_t ws_bytes, slse_stream_t stream);

/* The random draws of the sketch (Sec. 3, matrices D, P and B) for N' = 2^ceil(log2 N):
 * P (device int32, N'): the permutation, row j of P X is X[P[j]];
 * sigma (device int32, N'): the sampling order, sketch i keeps rows sigma[0..m_i);
 * D (device int8, N', nullable): the Rademacher signs +-1.  Asynchronous. */
slse_status slse_draws(int64_t N, uint64_t seed, int32_t *P, int32_t *sigma, int8_t *D,
                       void *workspace, size_t ws_bytes, slse_stream_t stream);

/* FP64 Householder QR of the r x d matrix A (device, row-major, lda >= d, r >= d), as used
 * for H-hat^{-1} v = R^{-1} R^{-T} v (Appendix, implementation details).  A is not modified.
 * R: device d x d (ld d), upper triangular with non-negative diagonal.  Hinv: device d x d
 * (ld d) = (R^T R)^{-1}, nullable.  Asynchronous. */
slse_status slse_qr(const double *A, int64_t r, int32_t d, int64_t lda, double *R, double *Hinv,
                    void *workspace, size_t ws_bytes, slse_stream_t stream);

/* The paper's experimental schedule (Sec. 5 preamble): r = 6d, eta = d/r, mu = (1-eta)^2,
 * m_1 = 8d doubling while m_i <= N'/2, a_i = 2, T = 100, tol = 0, FP64, momentum carried
 * across subproblems as in Algorithm 2; stage2 = SLSE_STAGE2_CORRECTION (used only if prec is
 * set to a mixed precision).
 * Writes at most cap entries into m_buf/a_buf (host) and points out->m/out->a at them.
 * Returns K (the number of sizes the schedule wants; > cap means truncated). */
int32_t slse_default_schedule(int64_t N, int32_t d, slse_schedule *out, int64_t *m_buf, int32_t *a_buf,
                              int32_t cap);

/* The same defaults for a given sketch family: kind SLSE_SRHT as above; kind
 * SLSE_COUNTSKETCH with m_1 = 8d rounded up to a power of two (the family's sizes are
 * powers of two).  Returns -1 for other kinds. */
int32_t slse_default_schedule_for(int64_t N, int32_t d, int32_t kind, slse_schedule *out, int64_t *m_buf,
                                  int32_t *a_buf, int32_t cap);

/* Differentiation through the estimate.  SLSE-FRS converges to the least-squares
 * estimate beta-hat = (X^T X)^{-1} X^T Y (its 2nd-stage fixed point solves the normal
 * equations, Sec. 3), so for a loss with v = dL/d(beta-hat) the input gradients are
 * dL/dY = X w and dL/dX = r w^T - (X w) beta-hat^T with w = (X^T X)^{-1} v and
 * r = Y - X beta-hat.  No paper counterpart; an extension for callers that train through
 * the estimator.
 *
 * slse_solve_normal: w = (X^T X)^{-1} v by the 2nd-stage M-IHS iteration (Eqs. (7), (8))
 * with the gradient v - X^T X w and the preconditioner Hinv (device d x d, e.g. from
 * slse_fit's trace->hinv_out): w_0 = 0, w+ = w + mu Hinv (v - X^T X w) + eta (w - w_prev).
 * sched supplies mu, eta, T (iteration cap), tol (the fit's relative-step test with
 * rho = sqrt(d/r)), r and prec (FP64, or MIXED_BF16 for F32 X: compensated FP32 passes);
 * its sizes m, a and kind are ignored.  X device; Y unused.  v, w_out: device d doubles.
 * report (nullable): ms_total, iters_stage2, final_rel_step, rebases, status.  Returns after w_out
 * is written (SLSE_ENOTCONV if tol > 0 was not met within T, w_out holds the last iterate).
 * Workspace: slse_solve_normal_workspace bytes, or NULL for a stream-ordered allocation. */
slse_status slse_solve_normal(const slse_problem *prob, const double *Hinv, const double *v, double *w_out,
                              const slse_schedule *sched, slse_report *report, void *workspace, size_t ws_bytes,
                              slse_stream_t stream);
size_t slse_solve_normal_workspace(const slse_problem *prob, int32_t prec);

/* The input gradients from w (above) in one pass over [X | Y]: dY[i] = x_i . w and
 * dX[i, :] = (y_i - x_i . beta) w - (x_i . w) beta.  dX (ld lddx >= d) and dY have the
 * dtype of X (F32 inputs: both dot products as compensated FP32 sums, so a row whose x_i . w
 * cancels still gets it to about 2^-24 of its size).  All pointers device.  Asynchronous on
 * `stream`. */
slse_status slse_ols_vjp(const slse_problem *prob, const double *beta, const double *w, void *dX, int64_t lddx,
                         void *dY, slse_stream_t stream);

/* The SLSE-FRS-tuning schedule (Sec. 5, sketch size tuning): a few small sketched problems
 * and one large one with a_i = 3; the paper's sizes at d = 2^6 (2^10 .. 2^16 and 2^19) are
 * 16d 2^j (j = 0..6) and 8192d, here dropped above N'/2 (rounded up to powers of two for
 * SLSE_COUNTSKETCH).  Other fields as slse_default_schedule_for.  Returns K, or -1. */
int32_t slse_tuning_schedule(int64_t N, int32_t d, int32_t kind, slse_schedule *out, int64_t *m_buf, int32_t *a_buf,
                             int32_t cap);

/* Theorem 4.3 lower bound on the inner iterations: log_3[((1+omega) r + 1)/omega] with
 * r = sqrt((m_i - d)/(m_prev - d)).  Host-only.  Returns NaN for m_prev <= d or omega <= 0. */
double slse_ai_bound(double omega, int64_t m_prev, int64_t m_i, int32_t d);

const char *slse_status_string(int32_t status);

/* Fault injection for tests (no paper counterpart).  Sets how many polls a grid-wide wait of
 * the library (the grid barrier of the FP64 Householder QR, slse_qr and the FP64 fit) makes
 * before it gives up; the call then reports SLSE_ETIMEOUT and every CTA of the grid stops at
 * that barrier or the next.  polls <= 0 restores the built-in limit (2^25 polls, about a
 * second).  Process-wide; takes effect for calls started afterwards.  Returns the previous
 * setting (0 = built-in).  The mbarrier waits of the tensor-core kernel keep their own fixed
 * time limit. */
int64_t slse_debug_spin_limit(int64_t polls);

/* Library version: major*10000 + minor*100 + patch. */
int32_t slse_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SLSE_H */
