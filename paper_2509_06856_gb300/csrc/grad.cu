// Fused one-pass residual-gradient kernels and the M-IHS update (paper Sec. 3,
// Eqs. (7) and (8); cost model "(4d+1) rows + 2d^2 + 5d" FLOPs per iteration).
//
// g = sum_i x_i^T (y_i - x_i beta) over the rows of X (2nd stage) or over the first
// m_i rows of the sampled sketch U (1st stage, scaled by N'/m_i).  One warp owns one
// row at a time: each lane holds a slice of the row (vector loads, 16 bytes per
// lane), forms its part of x_i beta, the warp reduces it with shuffles, and every
// lane then accumulates x_i r_i into its own slice of g.  Each row of X is read
// exactly once per pass.  Per-CTA partials are reduced in a fixed order (no atomics)
// so the result is deterministic.
//
// Mixed-precision 2nd stage (X stored FP32): the residual is formed against a base
// point beta_0 in FP64.  A "rebase" pass computes r0_i = y_i - x_i beta_0 with
// error-free transformations (TwoProd via FMA, TwoSum; beta_0 split into two FP32
// words) and stores r0 in FP32; later passes compute r_i = r0_i - x_i (beta - beta_0)
// in FP32, whose rounding error scales with ||beta - beta_0|| and vanishes as the
// iteration converges.  x_i r_i is accumulated in FP32 and folded every 16 rows into
// a two-word (TwoSum) accumulator.  The update kernel re-bases when the drift
// ||beta - beta_0|| exceeds both 2^-10 ||beta|| and 2^10 times the last step
// ||beta+ - beta||: the FP32 residual's error (~2^-24 of the drift) then stays below
// ~2^-14 of the step, i.e. of the iterate's current error, so passes far from the
// solution (the first steps from beta = 0) keep one base point instead of re-basing at
// every step, and the final base point lies within 2^-10 of the solution.
//
// Correction form of the mixed 2nd stage: exact passes stream X (the re-basing pass above or the
// plain FP32 pass); the reduction keeps their gradient g(beta_e).  The steps between exact ones
// use g(beta) = g(beta_e) - G_b (beta - beta_e) with the Gram matrix G_b = Xb^T Xb of the BF16 copy
// Xb of X, formed once on the tensor cores (gram.cu): a d x d product (k_gram_step) instead of a
// pass over X.  The update kernel schedules the next exact pass (a step below 1/100 of the first
// step after the last exact pass, a step above it, or one that meets the stopping test), makes it
// a re-basing pass only when the drift from beta_0 exceeds 2^-10 ||beta||, stops only on an exact
// step, and switches to the plain FP32 passes when a cycle gains less than plain steps would for
// the same cost.
#include "slse_internal.cuh"

namespace slse {
namespace {

constexpr int kGradThreads = 256;
constexpr int kWarps = kGradThreads / 32;
constexpr int kFlushRows = 16;

struct GradArgs {
  const void *X;
  int64_t ldx;
  const void *Y;
  int64_t nrows;
  int d;
  const double *beta_ring;
  DevState *st;
  const float *delta32;
  float *r0;
  double *beta0;
  double *partials;
  int check_done;
};

template <class Tx, int VW> struct Vec;
template <> struct Vec<float, 4> {
  static __device__ __forceinline__ void load(const float *p, float (&o)[4], bool stream) {
    const float4 t = stream ? __ldcs(reinterpret_cast<const float4 *>(p)) : __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
};
template <> struct Vec<float, 1> {
  static __device__ __forceinline__ void load(const float *p, float (&o)[1], bool stream) {
    o[0] = stream ? __ldcs(p) : __ldg(p);
  }
};
template <> struct Vec<double, 2> {
  static __device__ __forceinline__ void load(const double *p, double (&o)[2], bool stream) {
    const double2 t = stream ? __ldcs(reinterpret_cast<const double2 *>(p)) : __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
};
template <> struct Vec<double, 1> {
  static __device__ __forceinline__ void load(const double *p, double (&o)[1], bool stream) {
    o[0] = stream ? __ldcs(p) : __ldg(p);
  }
};
template <> struct Vec<float, 2> {  // FP32 data widened to FP64 arithmetic uses float pairs
  static __device__ __forceinline__ void load(const float *p, float (&o)[2], bool stream) {
    const float2 t = stream ? __ldcs(reinterpret_cast<const float2 *>(p)) : __ldg(reinterpret_cast<const float2 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
};

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Write the CTA partial: sum of the kWarps per-warp slices in a fixed order.
__device__ __forceinline__ void cta_partial(double (*sm)[512], int d, double *out) {
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += sm[w][c];
    out[c] = s;
  }
}

// ---------------------------------------------------------------- FP64 arithmetic
// Sums of R per-lane values (one per row) across the warp.  The first log2(R) levels are a
// transposed butterfly: at each level a lane keeps half of its rows and adds the partner's values
// of that half (one FP64 add per kept row instead of one per row), so after them lane l holds a
// partial of row rowsel(l); the remaining levels sum that one value.  FP64 adds hold this part's
// FP64 pipe for tens of cycles each, so the transposed form saves most of the reduction's cost
// (R = 4: 6 adds instead of 20).  Returns the full sum of every row to every lane (fixed order).
template <int R>
__device__ __forceinline__ void warp_sum_rows(double (&v)[R], int lane) {
  int off = 16;
#pragma unroll
  for (int n = R; n > 1; n >>= 1, off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < n / 2; ++j) {
      const double send = upper ? v[j] : v[j + n / 2];
      const double keep = upper ? v[j + n / 2] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
#pragma unroll
  for (; off > 0; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
  // lane l holds row sum((lane bit 16 >> k) * (R >> (k + 1))); broadcast each row's total
  double tot[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    int src = 0, o = 16;
#pragma unroll
    for (int n = R; n > 1; n >>= 1, o >>= 1)
      if (q % n >= n / 2) src |= o;
    tot[q] = __shfl_sync(0xffffffffu, v[0], src);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = tot[q];
}

// FP32 storage is widened by `widen` (integer pipe): the conversion instruction cost this pass
// more than its two FP64 FMAs per element (at 2^21 x 512: 6.8 ms from FP32 storage against
// 4.1 ms from FP64 storage, before the change).
// Tx = double (X F64 or U F64) or float (X F32, widened exactly).  VW = elements per lane load,
// VMAX = lane loads per row (sized to d), RPW = rows per warp iteration.
template <class Tx, int VW, int VMAX, int RPW>
__global__ void __launch_bounds__(kGradThreads) k_grad_f64(const GradArgs a) {
  __shared__ double sm[kWarps][512];
  if (a.check_done && a.st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  const int d = a.d;
  const double *beta = a.beta_ring + (size_t)(a.st->iter % 3) * d;
  const Tx *X = static_cast<const Tx *>(a.X);
  const Tx *Y = static_cast<const Tx *>(a.Y);
  double b[VMAX][VW], g[VMAX][VW];
#pragma unroll
  for (int v = 0; v < VMAX; ++v)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const int col = (v * 32 + lane) * VW + e;
      b[v][e] = col < d ? beta[col] : 0.0;
      g[v][e] = 0.0;
    }
  // The register tile wants one CTA per SM, so the rows of the next group are loaded (in their
  // storage type) before the current group's FP64 arithmetic: its latency hides behind the FMAs.
  Tx nx[RPW][VMAX][VW], ny[RPW];
  auto load_rows = [&](int64_t i0) {
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const int64_t i = i0 + q;
      const bool rv = i < a.nrows;
      const Tx *row = X + (rv ? i : 0) * a.ldx;
#pragma unroll
      for (int v = 0; v < VMAX; ++v) {
        const int col0 = (v * 32 + lane) * VW;
        if (rv && col0 < d) Vec<Tx, VW>::load(row + col0, nx[q][v], true);
        else {
#pragma unroll
          for (int e = 0; e < VW; ++e) nx[q][v][e] = Tx(0);
        }
      }
      ny[q] = rv ? Y[i] : Tx(0);
    }
  };
  const int64_t step = nw * RPW;
  if (gw * RPW < a.nrows) load_rows(gw * RPW);
  for (int64_t i0 = gw * RPW; i0 < a.nrows; i0 += step) {
    double x[RPW][VMAX][VW];
    double yv[RPW];
    bool special = false;
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
#pragma unroll
      for (int v = 0; v < VMAX; ++v)
#pragma unroll
        for (int e = 0; e < VW; ++e)
          x[q][v][e] = ((v * 32 + lane) * VW + e < d) ? widen(nx[q][v][e], special) : 0.0;
      yv[q] = widen(ny[q], special);
    }
    if (i0 + step < a.nrows) load_rows(i0 + step);
    if constexpr (sizeof(Tx) == 4) {
      // a denormal, infinity or NaN among these rows (warp-uniform, rare): convert them again
      if (__any_sync(0xffffffffu, special)) {
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
          const int64_t i = i0 + q;
          const bool rv = i < a.nrows;
          const Tx *row = X + (rv ? i : 0) * a.ldx;
#pragma unroll
          for (int v = 0; v < VMAX; ++v) {
            const int col0 = (v * 32 + lane) * VW;
#pragma unroll
            for (int e = 0; e < VW; ++e) x[q][v][e] = (rv && col0 + e < d) ? (double)row[col0 + e] : 0.0;
          }
          yv[q] = rv ? (double)Y[i] : 0.0;
        }
      }
    }
    double s[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      s[q] = 0.0;
#pragma unroll
      for (int v = 0; v < VMAX; ++v)
#pragma unroll
        for (int e = 0; e < VW; ++e) s[q] = fma(x[q][v][e], b[v][e], s[q]);
    }
    warp_sum_rows<RPW>(s, lane);
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const double r = yv[q] - s[q];  // rows past the end are zero rows: x = 0 adds nothing
#pragma unroll
      for (int v = 0; v < VMAX; ++v)
#pragma unroll
        for (int e = 0; e < VW; ++e) g[v][e] = fma(x[q][v][e], r, g[v][e]);
    }
  }
#pragma unroll
  for (int v = 0; v < VMAX; ++v)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const int col = (v * 32 + lane) * VW + e;
      if (col < d) sm[warp][col] = g[v][e];
    }
  cta_partial(sm, d, a.partials + (size_t)blockIdx.x * d);
}

// ---------------------------------------------------------------- 1st stage on BF16 sketch
// RPW consecutive rows per warp iteration (independent loads in flight); the BF16
// words stay packed in registers and are widened at use (exact).
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

template <int VMAX, int RPW>
__global__ void __launch_bounds__(kGradThreads, 2) k_grad_bf16v(const GradArgs a) {
  __shared__ double sm[kWarps][512];
  if (a.check_done && a.st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  const int d = a.d;
  const double *beta = a.beta_ring + (size_t)(a.st->iter % 3) * d;
  const __nv_bfloat16 *U = static_cast<const __nv_bfloat16 *>(a.X);
  const __nv_bfloat16 *V = static_cast<const __nv_bfloat16 *>(a.Y);
  const int64_t ldu = a.ldx;
  float b[VMAX][8], g[VMAX][8];
#pragma unroll
  for (int v = 0; v < VMAX; ++v)
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = (v * 32 + lane) * 8 + e;
      b[v][e] = col < d ? (float)beta[col] : 0.f;
      g[v][e] = 0.f;
    }
  for (int64_t i0 = gw * RPW; i0 < a.nrows; i0 += nw * RPW) {
    uint4 raw[RPW][VMAX];
    float y[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const int64_t i = i0 + q;
      const bool rv = i < a.nrows;
#pragma unroll
      for (int v = 0; v < VMAX; ++v) {
        const int col0 = (v * 32 + lane) * 8;
        raw[q][v] = (rv && col0 < d) ? __ldg(reinterpret_cast<const uint4 *>(U + i * ldu + col0))
                                     : make_uint4(0u, 0u, 0u, 0u);
      }
      y[q] = rv ? __bfloat162float(V[i]) : 0.f;
    }
    float s[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      float acc = 0.f;
#pragma unroll
      for (int v = 0; v < VMAX; ++v) {
        const uint32_t w[4] = {raw[q][v].x, raw[q][v].y, raw[q][v].z, raw[q][v].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          acc = fmaf(bf_lo(w[k]), b[v][2 * k], acc);
          acc = fmaf(bf_hi(w[k]), b[v][2 * k + 1], acc);
        }
      }
      s[q] = acc;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < RPW; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const float r = y[q] - s[q];  // padding columns are zero words, padding rows are zero
#pragma unroll
      for (int v = 0; v < VMAX; ++v) {
        const uint32_t w[4] = {raw[q][v].x, raw[q][v].y, raw[q][v].z, raw[q][v].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          g[v][2 * k] = fmaf(bf_lo(w[k]), r, g[v][2 * k]);
          g[v][2 * k + 1] = fmaf(bf_hi(w[k]), r, g[v][2 * k + 1]);
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < VMAX; ++v)
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = (v * 32 + lane) * 8 + e;
      if (col < d) sm[warp][col] = (double)g[v][e];
    }
  cta_partial(sm, d, a.partials + (size_t)blockIdx.x * d);
}

// Scalar-load variant for sketches whose rows are not 16-byte aligned.
template <int VMAX>
__global__ void __launch_bounds__(kGradThreads) k_grad_bf16s(const GradArgs a) {
  __shared__ double sm[kWarps][512];
  if (a.check_done && a.st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  const int d = a.d;
  const double *beta = a.beta_ring + (size_t)(a.st->iter % 3) * d;
  const __nv_bfloat16 *U = static_cast<const __nv_bfloat16 *>(a.X);
  const __nv_bfloat16 *V = static_cast<const __nv_bfloat16 *>(a.Y);
  float b[VMAX], g[VMAX];
#pragma unroll
  for (int v = 0; v < VMAX; ++v) {
    const int col = v * 32 + lane;
    b[v] = col < d ? (float)beta[col] : 0.f;
    g[v] = 0.f;
  }
  for (int64_t i = gw; i < a.nrows; i += nw) {
    float x[VMAX];
#pragma unroll
    for (int v = 0; v < VMAX; ++v) {
      const int col = v * 32 + lane;
      x[v] = col < d ? __bfloat162float(U[i * a.ldx + col]) : 0.f;
    }
    float s = 0.f;
#pragma unroll
    for (int v = 0; v < VMAX; ++v) s = fmaf(x[v], b[v], s);
    s = warp_sum(s);
    const float r = __bfloat162float(V[i]) - s;
#pragma unroll
    for (int v = 0; v < VMAX; ++v) g[v] = fmaf(x[v], r, g[v]);
  }
#pragma unroll
  for (int v = 0; v < VMAX; ++v) {
    const int col = v * 32 + lane;
    if (col < d) sm[warp][col] = (double)g[v];
  }
  cta_partial(sm, d, a.partials + (size_t)blockIdx.x * d);
}

// ---------------------------------------------------------------- mixed 2nd stage (X F32)
// REBASE = 1: error-free residual against beta (FP64) and r0 written; REBASE = 0:
// residual r0 - x . delta32.  The host launches both; the one whose mode does not
// match st->rebase returns at once.  The two-word accumulators (hi, lo) of each
// warp live in shared memory (float2 per column), folded every kFlushRows rows.
template <int VW, int VMAX, int REBASE, int RPW>
__global__ void __launch_bounds__(kGradThreads, 2) k_grad_mixed(const GradArgs a) {
  __shared__ __align__(16) double sm[kWarps][512];
  if (a.check_done && a.st->done) return;
  if ((a.st->rebase != 0) != (REBASE != 0)) return;
  if (!REBASE && a.st->dc && a.st->bfnext) return;  // correction form: a correction step, not a pass
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  const int d = a.d;
  const double *beta = a.beta_ring + (size_t)(a.st->iter % 3) * d;
  const float *X = static_cast<const float *>(a.X);
  const float *Y = static_cast<const float *>(a.Y);
  float2 *acc = reinterpret_cast<float2 *>(&sm[warp][0]);  // (hi, lo) per column, this warp only
  for (int c = lane; c < 512; c += 32) acc[c] = make_float2(0.f, 0.f);
  float bh[VMAX][VW], bl[REBASE ? VMAX : 1][VW];
  float gacc[VMAX][VW];
#pragma unroll
  for (int v = 0; v < VMAX; ++v)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const int col = (v * 32 + lane) * VW + e;
      if constexpr (REBASE) {
        const double bd = col < d ? beta[col] : 0.0;
        bh[v][e] = (float)bd;
        bl[v][e] = (float)(bd - (double)bh[v][e]);
      } else {
        bh[v][e] = col < d ? a.delta32[col] : 0.f;
      }
      gacc[v][e] = 0.f;
    }
  __syncwarp();
  int nacc = 0;
  for (int64_t i0 = gw * RPW; i0 < a.nrows; i0 += nw * RPW) {
    float x[RPW][VMAX][VW];
    float yr[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const int64_t i = i0 + q;
      const bool rv = i < a.nrows;
      const float *row = X + (rv ? i : 0) * a.ldx;
#pragma unroll
      for (int v = 0; v < VMAX; ++v) {
        const int col0 = (v * 32 + lane) * VW;
        float t[VW];
        if (rv && col0 < d) Vec<float, VW>::load(row + col0, t, true);
        else {
#pragma unroll
          for (int e = 0; e < VW; ++e) t[e] = 0.f;
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) x[q][v][e] = (col0 + e < d) ? t[e] : 0.f;
      }
      yr[q] = rv ? (REBASE ? __ldcs(Y + i) : __ldcs(a.r0 + i)) : 0.f;
    }
    float r[RPW];
    if constexpr (REBASE) {
      // Dot2 (Ogita, Rump, Oishi 2005): s + c = x . (bh + bl) with error-free products/sums
      float s[RPW], c[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        s[q] = 0.f;
        c[q] = 0.f;
#pragma unroll
        for (int v = 0; v < VMAX; ++v)
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            float p, pe, se;
            two_prod(x[q][v][e], bh[v][e], p, pe);
            two_sum(s[q], p, s[q], se);
            c[q] = fmaf(x[q][v][e], bl[v][e], c[q] + (pe + se));
          }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
          const float s2 = __shfl_xor_sync(0xffffffffu, s[q], off);
          const float c2 = __shfl_xor_sync(0xffffffffu, c[q], off);
          float e;
          two_sum(s[q], s2, s[q], e);
          c[q] = (c[q] + c2) + e;
        }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        float rh, re;
        two_sum(yr[q], -s[q], rh, re);
        r[q] = rh + (re - c[q]);
        if (a.r0 && lane == 0 && i0 + q < a.nrows) a.r0[i0 + q] = r[q];
      }
    } else {
      float s[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        s[q] = 0.f;
#pragma unroll
        for (int v = 0; v < VMAX; ++v)
#pragma unroll
          for (int e = 0; e < VW; ++e) s[q] = fmaf(x[q][v][e], bh[v][e], s[q]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int q = 0; q < RPW; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
#pragma unroll
      for (int q = 0; q < RPW; ++q) r[q] = yr[q] - s[q];
    }
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int v = 0; v < VMAX; ++v)
#pragma unroll
        for (int e = 0; e < VW; ++e) gacc[v][e] = fmaf(x[q][v][e], r[q], gacc[v][e]);
    nacc += RPW;
    if (nacc >= kFlushRows) {
      nacc = 0;
#pragma unroll
      for (int v = 0; v < VMAX; ++v)
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const int col = (v * 32 + lane) * VW + e;
          if (col < 512) {
            float2 h = acc[col];
            float sum, err;
            two_sum(h.x, gacc[v][e], sum, err);
            acc[col] = make_float2(sum, h.y + err);
          }
          gacc[v][e] = 0.f;
        }
    }
  }
  // fold the remainder and convert each (hi, lo) pair in place to one double
#pragma unroll
  for (int v = 0; v < VMAX; ++v)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const int col = (v * 32 + lane) * VW + e;
      if (col < 512) {
        const float2 h = acc[col];
        sm[warp][col] = ((double)h.x + (double)gacc[v][e]) + (double)h.y;
      }
    }
  if (REBASE && a.beta0 && blockIdx.x == 0) {
    for (int c = threadIdx.x; c < d; c += blockDim.x) a.beta0[c] = beta[c];
    if (threadIdx.x == 0) a.st->rebases += 1;
  }
  cta_partial(sm, d, a.partials + (size_t)blockIdx.x * d);
}

// ---------------------------------------------------------------- reduction and update
__global__ void k_reduce(const double *partials, int nblk, int d, double scale, double *g, const DevState *st,
                         int check_done, double *g0) {
  __shared__ double sm[8][33];
  if (check_done && st->done) return;
  if (g0 && st->dc && st->bfnext && !st->rebase) return;  // a correction step writes g itself
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  // four independent sums over CTAs warp, warp + 8, ... (loads overlap), combined in a fixed order
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (c < d) {
    int b = warp;
    for (; b + 24 < nblk; b += 32) {
      s0 += partials[(size_t)b * d + c];
      s1 += partials[(size_t)(b + 8) * d + c];
      s2 += partials[(size_t)(b + 16) * d + c];
      s3 += partials[(size_t)(b + 24) * d + c];
    }
    for (; b < nblk; b += 8) s0 += partials[(size_t)b * d + c];
  }
  sm[warp][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (warp == 0 && c < d) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += sm[w][lane];
    const double v = scale * t;
    if (g0) g0[c] = v;  // exact pass: keep g(beta_e)
    g[c] = v;
  }
}

struct UpdArgs {
  UpdateArgs u;
  double *part;  // 3 doubles per CTA
};

// beta+ = beta + mu H^{-1} g + eta (beta - beta_prev); one warp per row of H^{-1}.
__global__ void __launch_bounds__(256) k_update(const UpdArgs A, DevState *st) {
  const UpdateArgs &a = A.u;
  __shared__ double s_red[8][3];
  __shared__ int s_last;
  if (a.check_done && st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d = a.d;
  const int t = st->iter;
  const double *b = a.beta_ring + (size_t)(t % 3) * d;
  const double *bp = a.beta_ring + (size_t)((t + 2) % 3) * d;
  double *bn = a.beta_ring + (size_t)((t + 1) % 3) * d;
  const int i = blockIdx.x * 8 + warp;
  // correction form: whether this iteration's pass was exact (over X); read before the last block
  // of this kernel changes the state
  const bool corr_exact = a.stage2 && a.mixed && st->dc && (st->rebase || !st->bfnext);
  double ds = 0.0, nn = 0.0, dd = 0.0;
  if (i < d) {
    const double *Hrow = a.Hinv + (size_t)i * d;
    // four independent partial sums (the FP64 FMA latency is long on this part), fixed order
    double h0 = 0.0, h1 = 0.0, h2 = 0.0, h3 = 0.0;
    int k = lane;
    for (; k + 96 < d; k += 128) {
      h0 = fma(Hrow[k], a.g[k], h0);
      h1 = fma(Hrow[k + 32], a.g[k + 32], h1);
      h2 = fma(Hrow[k + 64], a.g[k + 64], h2);
      h3 = fma(Hrow[k + 96], a.g[k + 96], h3);
    }
    for (; k < d; k += 32) h0 = fma(Hrow[k], a.g[k], h0);
    double h = warp_sum((h0 + h1) + (h2 + h3));
    if (lane == 0) {
      const double mom = a.first ? 0.0 : a.eta * (b[i] - bp[i]);
      const double v = b[i] + a.mu * h + mom;
      bn[i] = v;
      ds = (v - b[i]) * (v - b[i]);
      nn = v * v;
      if (a.mixed) {
        const double del = v - a.beta0[i];
        a.delta32[i] = (float)del;
        dd = del * del;
        if (a.beta_e) {
          if (corr_exact) a.beta_e[i] = b[i];  // the gradient of this pass is g(b)
          a.delta_e[i] = (float)(v - a.beta_e[i]);
        }
      }
      if (a.hist && t < a.hist_cap) a.hist[(size_t)t * d + i] = v;
    }
  }
  if (lane == 0) { s_red[warp][0] = ds; s_red[warp][1] = nn; s_red[warp][2] = dd; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x0 = 0, x1 = 0, x2 = 0;
    for (int w = 0; w < 8; ++w) { x0 += s_red[w][0]; x1 += s_red[w][1]; x2 += s_red[w][2]; }
    A.part[3 * blockIdx.x + 0] = x0;
    A.part[3 * blockIdx.x + 1] = x1;
    A.part[3 * blockIdx.x + 2] = x2;
    __threadfence();
    const unsigned prev = atomicAdd(&st->upd_count, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || warp != 0) return;
  __threadfence();
  // the last CTA sums the per-CTA partials with its first warp: lane l takes CTAs l, l + 32, ...
  // in order, then a fixed shuffle tree (no serial chain of L2 round trips)
  double x0 = 0, x1 = 0, x2 = 0;
  for (unsigned c = lane; c < gridDim.x; c += 32) {
    x0 += __ldcg(A.part + 3 * c + 0);
    x1 += __ldcg(A.part + 3 * c + 1);
    x2 += __ldcg(A.part + 3 * c + 2);
  }
  x0 = warp_sum(x0);
  x1 = warp_sum(x1);
  x2 = warp_sum(x2);
  // correction form: a correction step more than twice the size of the cycle's first step is the
  // correction iteration diverging (an ill-conditioned X): it is not taken.  The kept iterate is
  // copied into the new slot (so the momentum of the next step is zero), the vectors of the base
  // points are formed from it, the norms are those of the kept iterate, and the next pass is exact.
  const bool reject = corr_exact == false && a.stage2 && a.mixed && st->dc && x0 > 4.0 * st->step_ref;
  if (reject) {
    double k1 = 0.0, k2 = 0.0;
    for (int i = lane; i < d; i += 32) {
      bn[i] = b[i];
      const double del = b[i] - a.beta0[i];
      a.delta32[i] = (float)del;
      if (a.beta_e) a.delta_e[i] = (float)(b[i] - a.beta_e[i]);
      if (a.hist && t < a.hist_cap) a.hist[(size_t)t * d + i] = b[i];
      k1 += b[i] * b[i];
      k2 += del * del;
    }
    x0 = 0.0;
    x1 = warp_sum(k1);
    x2 = warp_sum(k2);
  }
  if (lane != 0) return;
  st->upd_count = 0;
  const double rel = sqrt(x0) / (sqrt(x1) > 0.0 ? sqrt(x1) : 1.0);
  st->rel_step = rel;
  const int tn = t + 1;
  st->iter = tn;
  if (!isfinite(x0) || !isfinite(x1)) {
    st->status |= ST_NUMERIC;
    st->done = 1;
  }
  if (a.stage2) {
    // x2 = ||beta+ - beta_0||^2, x1 = ||beta+||^2, x0 = ||beta+ - beta||^2
    const bool corr = a.mixed && st->dc;
    const int exact = !corr || st->rebase || !st->bfnext;  // this iteration's pass was over X
    const int k2 = t - a.hist_base;
    if (k2 >= 0 && k2 < (int)sizeof(st->mode_hist)) st->mode_hist[k2] = exact ? 0 : 1;
    if (corr && exact) {
      // a cycle (exact pass + k correction steps, 1 + k c passes' worth of time for a correction
      // step costing c passes) that shrank the exact step by less than rho^(1 + k c), what plain
      // steps gain in that time, or by less than 10x: the BF16 Hessian term is too coarse for
      // these data (ill-conditioned X; its relative error, which sets a cycle's gain, is then
      // above 0.1, where the cycles, plain fixed-point steps without momentum, fall behind the
      // full form and the first cycle's gain, measured from the large first step of the 2nd
      // stage, overstates the gain in the error), so the remaining steps take the full form (its
      // next pass reads the r0 this exact pass wrote).  x0 and step_prev are squared norms.  A step
      // that meets the stopping test ends the fit either way and decides nothing.
      const double gain = fmin(0.01, pow(a.rho, 2.0 * (1.0 + a.inner_cost * st->ninner)));
      const bool stops = a.thr > 0.0 && rel <= a.thr;
      if (st->step_prev > 0.0 && x0 > st->step_prev * gain && !stops) {
        st->dc = 0;
        st->dc_fell_back = 1;
      }
      st->step_prev = x0;
      st->step_ref = x0;
      st->ninner = 0;
    } else if (corr) {
      st->ninner += 1;
    }
    const bool may_stop = !(corr && !exact);  // the correction form stops on exact steps only
    if (may_stop && a.thr > 0.0 && rel <= a.thr) st->done = 1;
    else if (tn >= a.T) {
      st->done = 1;
      if (a.thr > 0.0) st->status |= ST_NOTCONV;
    }
    if (a.mixed) {
      // next pass exact: the steps have shrunk to 1/10^4 of the cycle's first step (the correction
      // iteration has then settled at its fixed point, within ~1e-4 of the exact one on the
      // benchmark data), or one meets the stopping test (the stop itself waits for an exact step),
      // or a step grew beyond the cycle's first step (the correction iteration diverging on an
      // ill-conditioned X), or the cycle has taken 20 correction steps (twice what a contraction of
      // rho = 0.41 per step needs for 1e-4; steps count toward T); the exact pass
      // re-bases (error-free residuals) only when the drift from beta_0 exceeds 2^-10 ||beta||, so
      // that the FP32 residual r0 - X (beta - beta_0) stays within ~2^-34 ||X|| ||beta||
      if (st->dc) {
        const bool next_exact =
            !exact && (reject || x0 < 1e-8 * st->step_ref || x0 > st->step_ref || st->ninner >= 20 ||
                       (a.thr > 0.0 && rel <= a.thr));
        st->bfnext = next_exact ? 0 : 1;
        st->rebase = (next_exact && x2 > 0x1p-20 * x1) ? 1 : 0;
      } else {
        st->bfnext = 0;
        st->rebase = (x2 > 0x1p-20 * x1 && x2 > 0x1p20 * x0) ? 1 : 0;
      }
    }
  }
}

// Correction step: g = g0 - G_b delta_e, one warp per row of G_b (four independent FP64 sums, fixed
// order); only when the device state selects a correction step.
__global__ void __launch_bounds__(256) k_gram_step(const double *Gb, const float *delta_e, const double *g0, double *g,
                                                   int d, const DevState *st) {
  if (st->done || st->rebase || !st->dc || !st->bfnext) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 8 + warp;
  if (i >= d) return;
  const double *row = Gb + (size_t)i * d;
  double h0 = 0.0, h1 = 0.0, h2 = 0.0, h3 = 0.0;
  int k = lane;
  for (; k + 96 < d; k += 128) {
    h0 = fma(row[k], (double)delta_e[k], h0);
    h1 = fma(row[k + 32], (double)delta_e[k + 32], h1);
    h2 = fma(row[k + 64], (double)delta_e[k + 64], h2);
    h3 = fma(row[k + 96], (double)delta_e[k + 96], h3);
  }
  for (; k < d; k += 32) h0 = fma(row[k], (double)delta_e[k], h0);
  const double h = warp_sum((h0 + h1) + (h2 + h3));
  if (lane == 0) g[i] = g0[i] - h;
}

__global__ void k_copy_beta(const double *ring, const DevState *st, int d, double *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < d) out[c] = ring[(size_t)(st->iter % 3) * d + c];
}

template <class K>
cudaError_t launch1(K kern, int nblk, const GradArgs &a, cudaStream_t s) {
  kern<<<nblk, kGradThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// FP64 kernel with its register tile sized to d (lane loads per row) and 4 rows per warp
// iteration (2 for the widest tiles, whose rows take 32 doubles per lane)
template <class Tx, int VW>
cudaError_t launch_f64(int d, int nblk, const GradArgs &a, cudaStream_t s) {
  constexpr int per = 32 * VW;
  if (d <= per) return launch1(k_grad_f64<Tx, VW, 1, 4>, nblk, a, s);
  if (d <= 2 * per) return launch1(k_grad_f64<Tx, VW, 2, 4>, nblk, a, s);
  if (d <= 4 * per) return launch1(k_grad_f64<Tx, VW, 4, 4>, nblk, a, s);
  if (d <= 8 * per) return launch1(k_grad_f64<Tx, VW, 8, 2>, nblk, a, s);
  if constexpr (VW == 1) {
    if (d <= 16 * per) return launch1(k_grad_f64<Tx, VW, 16, 2>, nblk, a, s);
  }
  return cudaErrorInvalidValue;
}

inline bool aligned(const void *p, int64_t ld, int64_t elem_bytes, int vw) {
  return (reinterpret_cast<uintptr_t>(p) % (size_t)(vw * elem_bytes) == 0) && (ld % vw == 0);
}

}  // namespace

int grad_grid(int nsm) { return 2 * nsm; }

cudaError_t launch_grad(int mode, int xdtype, const void *X, int64_t ldx, const void *Y, int64_t nrows, int d,
                        const double *beta_ring, DevState *st, const float *delta32, float *r0, double *beta0,
                        double *partials, int nblk, int check_done, cudaStream_t s) {
  GradArgs a{X, ldx, Y, nrows, d, beta_ring, st, delta32, r0, beta0, partials, check_done};
  if (d > 512 || d < 1) return cudaErrorInvalidValue;
  switch (mode) {
    case GM_F64:
    case GM_STAGE1_F64:
      if (xdtype == SLSE_F64) {
        if (d % 2 == 0 && aligned(X, ldx, 8, 2)) return launch_f64<double, 2>(d, nblk, a, s);
        return launch_f64<double, 1>(d, nblk, a, s);
      } else {
        if (d % 2 == 0 && aligned(X, ldx, 4, 2)) return launch_f64<float, 2>(d, nblk, a, s);
        return launch_f64<float, 1>(d, nblk, a, s);
      }
    case GM_STAGE1_BF16:
      // the sketch buffer's padding columns are never written: the vector path requires
      // d % 8 == 0 so that no padding word is read
      // lanes cover 8 columns per word: one word per lane up to d = 256 (more rows in flight)
      if (d % 8 == 0 && ldx % 8 == 0 && aligned(X, ldx, 2, 8))
        return d <= 256 ? launch1(k_grad_bf16v<1, 6>, nblk, a, s) : launch1(k_grad_bf16v<2, 4>, nblk, a, s);
      return launch1(k_grad_bf16s<16>, nblk, a, s);
    case GM_MIXED: {
      if (xdtype != SLSE_F32) return cudaErrorInvalidValue;
      const bool vec = d % 4 == 0 && aligned(X, ldx, 4, 4);
      // rows in flight per warp grow as d shrinks (the same 32 x-values per lane)
      cudaError_t e;
      if (!vec) e = launch1(k_grad_mixed<1, 16, 1, 1>, nblk, a, s);
      else if (d <= 128) e = launch1(k_grad_mixed<4, 1, 1, 8>, nblk, a, s);
      else if (d <= 256) e = launch1(k_grad_mixed<4, 2, 1, 4>, nblk, a, s);
      else e = launch1(k_grad_mixed<4, 4, 1, 2>, nblk, a, s);
      if (e != cudaSuccess) return e;
      if (!vec) return launch1(k_grad_mixed<1, 16, 0, 1>, nblk, a, s);
      if (d <= 128) return launch1(k_grad_mixed<4, 1, 0, 8>, nblk, a, s);
      if (d <= 256) return launch1(k_grad_mixed<4, 2, 0, 4>, nblk, a, s);
      return launch1(k_grad_mixed<4, 4, 0, 2>, nblk, a, s);
    }
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t preload_grad_kernels() {
  // every kernel launch_grad (modes GM_F64 and GM_MIXED) and launch_reduce can pick
  const void *k[] = {
      (const void *)k_grad_f64<double, 2, 1, 4>, (const void *)k_grad_f64<double, 2, 2, 4>,
      (const void *)k_grad_f64<double, 2, 4, 4>, (const void *)k_grad_f64<double, 2, 8, 2>,
      (const void *)k_grad_f64<double, 1, 1, 4>, (const void *)k_grad_f64<double, 1, 2, 4>,
      (const void *)k_grad_f64<double, 1, 4, 4>, (const void *)k_grad_f64<double, 1, 8, 2>,
      (const void *)k_grad_f64<double, 1, 16, 2>,
      (const void *)k_grad_f64<float, 2, 1, 4>,  (const void *)k_grad_f64<float, 2, 2, 4>,
      (const void *)k_grad_f64<float, 2, 4, 4>,  (const void *)k_grad_f64<float, 2, 8, 2>,
      (const void *)k_grad_f64<float, 1, 1, 4>,  (const void *)k_grad_f64<float, 1, 2, 4>,
      (const void *)k_grad_f64<float, 1, 4, 4>,  (const void *)k_grad_f64<float, 1, 8, 2>,
      (const void *)k_grad_f64<float, 1, 16, 2>,
      (const void *)k_grad_mixed<1, 16, 1, 1>,   (const void *)k_grad_mixed<4, 1, 1, 8>,
      (const void *)k_grad_mixed<4, 2, 1, 4>,    (const void *)k_grad_mixed<4, 4, 1, 2>,
      (const void *)k_grad_mixed<1, 16, 0, 1>,   (const void *)k_grad_mixed<4, 1, 0, 8>,
      (const void *)k_grad_mixed<4, 2, 0, 4>,    (const void *)k_grad_mixed<4, 4, 0, 2>,
      (const void *)k_reduce};
  for (const void *f : k) {
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_reduce(const double *partials, int nblk, int d, double scale, double *g, DevState *st,
                          int check_done, cudaStream_t s, double *g0) {
  k_reduce<<<(d + 31) / 32, 256, 0, s>>>(partials, nblk, d, scale, g, st, check_done, g0);
  return cudaGetLastError();
}

cudaError_t launch_update(const UpdateArgs &a, DevState *st, cudaStream_t s) {
  // per-CTA partial sums live right after the DevState's own cache line block
  UpdArgs A{a, reinterpret_cast<double *>(st + 1)};
  k_update<<<(a.d + 7) / 8, 256, 0, s>>>(A, st);
  return cudaGetLastError();
}

cudaError_t launch_gram_step(const double *Gb, const float *delta_e, const double *g0, double *g, int d, DevState *st,
                             cudaStream_t s) {
  k_gram_step<<<(d + 7) / 8, 256, 0, s>>>(Gb, delta_e, g0, g, d, st);
  return cudaGetLastError();
}

cudaError_t launch_copy_beta(const double *beta_ring, DevState *st, int d, double *out, cudaStream_t s) {
  k_copy_beta<<<(d + 255) / 256, 256, 0, s>>>(beta_ring, st, d, out);
  return cudaGetLastError();
}

}  // namespace slse
