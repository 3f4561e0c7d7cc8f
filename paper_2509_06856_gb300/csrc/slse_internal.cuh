// Internal declarations shared by the CUDA translation units of the SLSE-FRS library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/slse.h"

namespace slse {

// ----------------------------------------------------------------------------------
// Device status word (bit flags), written by kernels, read by the host at the end.
enum : unsigned {
  ST_TIMEOUT = 1u,   // a bounded spin gave up
  ST_NUMERIC = 2u,   // NaN/Inf seen, or zero pivot
  ST_NOTCONV = 4u,   // hit T with tol > 0
};

// Iteration state living in device memory (one per fit).
struct DevState {
  int iter;            // number of M-IHS iterations done
  int done;            // stage-2 stop flag (tol met or T reached)
  int rebase;          // mixed path: next 2nd-stage pass recomputes the base residual
  int rebases;         // count of rebase passes
  unsigned status;     // ST_* bits
  unsigned upd_count;  // last-block counter of the update kernel
  unsigned bar_count;  // grid barrier (QR)
  unsigned bar_gen;
  double rel_step;     // last ||b+ - b|| / ||b+||
  long long spin_limit; // polls of a grid-wide wait before it gives up (0: the built-in 2^25)
  int dc;              // mixed 2nd stage, correction form active: correction steps between exact passes
  int bfnext;          // correction form: the next step is a correction step (else an exact pass over X)
  int dc_fell_back;    // the correction form was switched off for this run
  double step_ref;     // correction form: squared step of the last exact pass
  double step_prev;    // correction form: squared step of the exact pass before it
  int ninner;          // correction form: correction steps since the last exact pass
  unsigned char mode_hist[128];  // 2nd-stage step kind of iteration t (< 128): 0 pass over X, 1 correction step
};
static_assert(sizeof(DevState) <= 512, "the per-CTA partials of the update kernel follow the state");

// ----------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  Counter (c0..c3), key (k0, k1).
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// Draw streams (counter word c2): signs D, permutation P, sampling order sigma.
enum { STREAM_D = 0, STREAM_P = 1, STREAM_SIGMA = 2 };

// ----------------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum; FMA-based TwoProd), FP32.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// Exact FP32 -> FP64 widening on the integer pipe.  The conversion instruction runs on the FP64
// unit, which FP64-bound kernels need for their own arithmetic, so normal floats and zeros are
// widened with integer operations, without a branch: exponent re-biased by 1023 - 127 = 896
// (zero keeps only its sign), mantissa shifted up by 29 bits.  Denormals, infinities and NaNs
// are not: they set `special`, and the caller redoes those values with the conversion
// instruction (a warp-uniform, rare path).
__device__ __forceinline__ double widen(double v, bool &) { return v; }
__device__ __forceinline__ double widen(float f, bool &special) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7FFFFFFFu;
  const uint32_t e = a >> 23;
  special |= (e == 255u) | ((e == 0u) & (a != 0u));
  const uint32_t hi = (u & 0x80000000u) | (a != 0u ? (a >> 3) + 0x38000000u : 0u);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// ----------------------------------------------------------------------------------
// Bounded grid barrier for cooperative launches.  All CTAs of the grid must call it
// the same number of times.  Gives up after ~1 s and raises ST_TIMEOUT; returns false
// when the grid should stop (timeout here or in another CTA).
__device__ __forceinline__ bool grid_barrier(DevState *st, unsigned nblocks) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned *genp = &st->bar_gen;
    const unsigned g = *genp;
    __threadfence();
    const unsigned arrived = atomicAdd(&st->bar_count, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      st->bar_count = 0;
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      long long spins = 0;
      const long long lim = st->spin_limit > 0 ? st->spin_limit : (1ll << 25);
      while (*genp == g) {
        if (spins > 512) __nanosleep(32);
        if (++spins > lim) { atomicOr(&st->status, ST_TIMEOUT); ok = 0; break; }
        if ((spins & 255) == 0 && (((volatile unsigned *)&st->status)[0] & ST_TIMEOUT)) { ok = 0; break; }
      }
    }
    __threadfence();
    if (((volatile unsigned *)&st->status)[0] & ST_TIMEOUT) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ----------------------------------------------------------------------------------
// Host-side helpers and launchers implemented in the .cu files.

// api.cu: the spin limit every new DevState starts with (slse_debug_spin_limit; 0 = built-in)
long long debug_spin_limit();

constexpr int64_t kMaxPaddedRows = int64_t(1) << 24;  // largest padded row count N' the library accepts
// api.cu
bool is_host_pointer(const void *ptr);
bool valid_problem(const slse_problem *p);

// countsketch.cu: the CountSketch family (nested sizes 2^l, l1 <= l <= L, and an
// independent r-row Hessian sketch) in one sort and one pass over the rows.
struct CsPlan {
  int64_t N;
  int d, prec;
  int64_t r;        // Hessian-sketch rows (0: none)
  int L, l1;        // log2 of the largest and smallest nested sizes (-1: none)
  bool big;         // top-level buckets of >= 64 rows: one CTA per bucket
  int F;            // levels folded in registers below L by the warp kernel
  int ib, Bn, rb, Bh;
  int64_t lds;      // leading dimension of the working-precision scratch rows
  size_t o_sort0, o_sort1, o_rows0, o_rows1, o_st0, o_st1, o_scr0, o_scr1, total;
};
CsPlan cs_plan(int64_t N, int d, int prec, int64_t m_min, int64_t m_max, int64_t r);
// lvX[l] / lvY[l] (l <= 24, nullable): the 2^l-row sketch in natural bucket order (ld ldo);
// hatX / hatY (nullable when r = 0): the Hessian sketch (ld ldh).  ws: pl.total bytes.
cudaError_t launch_countsketch(const CsPlan &pl, int xdtype, const void *X, int64_t ldx, const void *Y, uint64_t seed,
                               void *const *lvX, void *const *lvY, int64_t ldo, void *hatX, void *hatY, int64_t ldh,
                               void *ws, cudaStream_t s);

// fp8.cu: the FP8 form of the sketch (E4M3 values, one power-of-two scale per 32-column
// block of a row, byte = exponent + 127; Y values in BF16).
cudaError_t launch_grad_mx(const uint8_t *U, int64_t ldq, const uint8_t *S, int64_t nsb, const __nv_bfloat16 *V,
                           int64_t nrows, int d, const double *beta_ring, const DevState *st, double *part, int nblk,
                           cudaStream_t s);
cudaError_t launch_mx_to_bf16(const uint8_t *U, int64_t ldq, const uint8_t *S, int64_t nsb, int64_t rows, int d,
                              __nv_bfloat16 *out, int64_t ldo, cudaStream_t s);
cudaError_t launch_quantize_mx(const __nv_bfloat16 *A, int64_t lda, int64_t rows, int d, uint8_t *U, int64_t ldq,
                               uint8_t *S, int64_t nsb, cudaStream_t s);

// gaussian.cu: the Gaussian sketch G [X | Y] / sqrt(m) (G m x N, entries from Philox stream 5
// and Box-Muller).  FP64: FP64 entries and products (X F64 or F32).  MIXED_BF16 (X F32): BF16
// entries and X on the tensor cores with FP32 accumulation, output BF16.
struct GaussPlan {
  int64_t N, m;
  int d, prec, nsm;
  bool with_y;
  int groups;          // column groups of <= 512 packed columns (tensor-core path)
  int ncp;             // packed columns of the widest group
  int tmem_cols, stages;
  size_t smem;
  int64_t nchunk, cps, mpad;
  int splits;
  size_t o_xt, o_part, o_status, total;  // workspace layout (o_status: one word the caller clears)
};
GaussPlan gauss_plan(int64_t N, int d, int prec, int64_t m, bool with_y, int nsm);
// SX (m x ldsx) and SY (m, nullable when the plan has no Y column) of the output precision;
// status: ST_TIMEOUT is raised there when a bounded wait gave up (the output is then NaN).
cudaError_t launch_gaussian(const GaussPlan &p, int xdtype, const void *X, int64_t ldx, const void *Y, uint64_t seed,
                            void *SX, int64_t ldsx, void *SY, double scale, unsigned *status, void *ws,
                            cudaStream_t s);

// gaussian.cu: X (F32, N x nx, ld ldx) -> BF16 chunks of 32 rows in the K-major core-matrix
// layout of the tcgen05 operands (ncp packed columns, zero beyond nx and past row N; chunks are
// written in pairs: 2 ceil(N / 64) chunks of ncp * 64 bytes).
cudaError_t launch_pack_bf16(const float *X, int64_t ldx, int64_t N, int nx, int ncp, uint8_t *xt, cudaStream_t s);

// gram.cu: G_b = Xb^T Xb (d x d, FP64, row-major) for the BF16 copy Xb of X (F32) on the tensor
// cores, through a packed copy of X and per-range FP32 partials (workspace GramPlan::total bytes).
struct GramPlan {
  int64_t N;
  int d, ncp, tmem_cols, stages, splits;
  int64_t nchunk, cps;
  size_t smem, o_xt, o_part, o_grp, total;
  // FP32 path (rows read and rounded on chip): 32-row stages, stages per range, ranges, shared memory
  int64_t nstage, cps_f;
  int splits_f, q_f;  // ranges, CTAs per range (a cluster)
  size_t smem_f;
  // tensor-core work (upper block triangle, padded rows) and DRAM bytes of each path: X read,
  // (packed path) the BF16 copy written and read, the partials written and read
  double flops_f32, flops_packed, bytes_f32, bytes_packed;
};
GramPlan gram_plan(int64_t N, int d, int nsm);
// whether launch_gram reads X directly (d and ldx multiples of 4, X 16-byte aligned) instead of
// packing it first
bool gram_fp32_path(const GramPlan &p, const float *X, int64_t ldx);
// status: ST_TIMEOUT is raised there when a bounded wait gave up (G is then NaN)
cudaError_t launch_gram(const GramPlan &p, const float *X, int64_t ldx, double *G, unsigned *status, void *ws,
                        cudaStream_t s);
// Gram matrix of a BF16 matrix B (rows x d, row stride ldb elements, a multiple of 8, 16-byte
// aligned), scaled: G = scale B^T B, through per-range FP32 partials (part_bytes at part)
struct GramWPlan {
  int64_t rows;
  int d, ncp, tmem_cols, q, splits, kr;  // kr: rows per stage
  int64_t nstage, cps;
  size_t smem, o_grp, part_bytes;  // the FP64 group sums of the reduction start at o_grp
  double flops, bytes;
};
GramWPlan gram_w_plan(int64_t rows, int d, int nsm);
bool gram_w_ok(const GramWPlan &p, const void *B, int64_t ldb);
cudaError_t launch_gram_w(const GramWPlan &p, const void *B, int64_t ldb, double scale, double *G, unsigned *status,
                          float *part, cudaStream_t s);

// draws.cu
size_t draws_ws_bytes(int64_t Np);
cudaError_t launch_draws(int64_t Np, uint64_t seed, int32_t *Psd /*N', sign-folded P*/,
                         int32_t *P /*nullable*/, int32_t *sigma, int8_t *D /*nullable*/,
                         void *ws, cudaStream_t s);
// The two permutations one at a time, so that sigma (needed from pass 2 on) can be drawn beside
// pass 1: launch_draws_perm writes Psd (ws: draws_one_ws_bytes + 4 N' bytes), launch_draws_sigma
// writes sigma (ws: draws_one_ws_bytes).  Each gives the same array as launch_draws.
size_t draws_one_ws_bytes(int64_t Np);
cudaError_t launch_draws_perm(int64_t Np, uint64_t seed, int32_t *Psd, void *ws, cudaStream_t s);
cudaError_t launch_draws_sigma(int64_t Np, uint64_t seed, int32_t *sigma, void *ws, cudaStream_t s);
// pos[idx(k)] = s for k = sigma[s], s in [s0, s1), -1 elsewhere; idx(k) = (k mod n2) n1 + k div n2
// with n2 = 2^log2 (the pass-1 group size; log2 = log2 N' for single-pass plans).
cudaError_t launch_pos_map(const int32_t *sigma, int64_t Np, int64_t s0, int64_t s1, int log2, int32_t *pos,
                           cudaStream_t s);

// srht.cu
struct SrhtPlan {
  int logN;         // log2 N'
  int log1, log2;   // pass split: n1 = 2^log1 groups-by-stride, n2 = 2^log2 rows per pass-1 group
  bool single;      // one pass (N' small)
};
SrhtPlan srht_plan(int64_t Np);
// Sketch of [X|Y] into sampled rows: out row pos[k] (if >= 0) gets scale * (H D P X_pad)[k].
// W (intermediate, N' x ldw of the output type) is unused for single-pass plans.
cudaError_t launch_srht(const SrhtPlan &pl, int prec, int xdtype, const void *X, int64_t ldx,
                        const void *Y, int64_t N, int d, const int32_t *Psd, const int32_t *pos,
                        void *W, void *WY, int64_t ldw, void *U, void *V, int64_t ldu, double scale,
                        cudaStream_t s, cudaEvent_t ev_mid /* nullable: recorded between the passes */,
                        uint8_t *Uscale = nullptr /* MIXED_FP8: block exponents of U */, int64_t ld_scale = 0,
                        __nv_bfloat16 *hat = nullptr /* MIXED_FP8: rows >= hat_row0 in BF16 here */,
                        int64_t hat_row0 = 0, int64_t hat_ld = 0,
                        void *copy_out = nullptr /* two-pass plans: X rows read by pass 1 (e.g. from
                                                    mapped host memory) are also stored here, same
                                                    element offsets (ldx); 16-byte aligned */,
                        unsigned *status = nullptr /* ST_TIMEOUT raised here if a bounded wait gave up */,
                        cudaEvent_t wait_pass2 = nullptr /* two-pass plans: s waits for it before pass 2 */);

// grad.cu
// GM_MIXED: the mixed 2nd-stage pass over X: the re-basing pass (error-free residuals) and the
// plain FP32 pass against the base point; each returns at once unless the device state selects it
// (neither runs on a correction step of the correction form).
enum GradMode { GM_F64 = 0, GM_MIXED = 1, GM_STAGE1_BF16 = 2, GM_STAGE1_F64 = 3 };
int grad_grid(int nsm);
cudaError_t launch_grad(int mode, int xdtype, const void *X, int64_t ldx, const void *Y, int64_t nrows,
                        int d, const double *beta_ring, DevState *st, const float *delta32, float *r0,
                        double *beta0, double *partials, int nblk, int check_done, cudaStream_t s);
// g = scale * (sum of the per-CTA partials).  g0 (nullable; mixed 2nd stage in correction form):
// after an exact pass (over X) g0 = g; on a correction step the reduction does nothing (the
// correction step writes g).
cudaError_t launch_reduce(const double *partials, int nblk, int d, double scale, double *g,
                          DevState *st, int check_done, cudaStream_t s, double *g0 = nullptr);
// Correction step of the correction form: g = g0 - G_b delta_e (G_b d x d FP64, delta_e =
// fl32(beta - beta_e)); runs only when the device state selects a correction step.
cudaError_t launch_gram_step(const double *Gb, const float *delta_e, const double *g0, double *g, int d,
                             DevState *st, cudaStream_t s);
// Loads the code of every kernel launch_grad (GM_F64, GM_MIXED) and launch_reduce can launch,
// so that a later first launch of one of them does not load a module (which allocates).
cudaError_t preload_grad_kernels();
struct UpdateArgs {
  const double *g;
  const double *Hinv;
  double *beta_ring;   // 3 x d
  double *beta0;       // mixed: base point
  float *delta32;      // mixed: fl32(beta - beta0)
  double *hist;        // trace, nullable
  int hist_cap;
  int d;
  double mu, eta;
  int first;           // momentum reset for this iteration
  int stage2;          // check stopping
  double thr;          // relative-step threshold (stage 2, > 0 to enable)
  int T;               // iteration cap
  int mixed;           // maintain delta32 / rebase flag
  int check_done;
  int hist_base;       // iteration index of the first 2nd-stage step (mode_hist is indexed from it)
  double rho;          // sqrt(d / r), the contraction of a plain 2nd-stage step (correction form's test)
  double *beta_e;      // correction form: the iterate of the last exact pass
  float *delta_e;      // correction form: fl32(beta - beta_e), the vector of the correction step
  double inner_cost;   // correction form: cost of a correction step in exact passes (fallback test)
};
cudaError_t launch_update(const UpdateArgs &a, DevState *st, cudaStream_t s);
cudaError_t launch_copy_beta(const double *beta_ring, DevState *st, int d, double *out, cudaStream_t s);

// linalg.cu
size_t qr_ws_bytes(int64_t r, int d, int nsm);
cudaError_t launch_gather_hessian_rows(int prec, const void *U, int64_t ldu, int64_t row0, int64_t r,
                                       int d, double scale, double *A, cudaStream_t s);
cudaError_t launch_qr(double *A, int64_t r, int d, int64_t lda, double *R, double *Hinv, void *ws,
                      DevState *st, cudaStream_t s);
// Mixed path: H-hat^{-1} = G^{-1} for G = scale2 * U[row0:row0+r]^T U[row0:row0+r] (U in BF16,
// G accumulated exactly), by the blocked sweep operator in FP64.  A non-positive pivot
// raises ST_NUMERIC (the caller then takes the Householder QR).
size_t sweep_ws_bytes(int64_t r, int d);
cudaError_t launch_gram_sweep(const void *U, int64_t ldu, int64_t row0, int64_t r, int d, double scale2, double *Hinv,
                              void *ws, DevState *st, cudaStream_t s);

}  // namespace slse
