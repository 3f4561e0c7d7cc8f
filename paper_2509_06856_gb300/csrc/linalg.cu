// FP64 Householder QR of the Hessian sketch S-hat X (r x d), the explicit
// R^{-1}, and H-hat^{-1} = R^{-1} R^{-T} (paper, Appendix "implementation details":
// H-hat^{-1} v is applied through the QR of S-hat X).
//
// FP64 runs at ~1/57 of the FP32 rate on this part, so the QR is spread over every
// SM: one cooperative persistent kernel, each CTA owning a contiguous block of rows.
// Column j costs one grid-wide reduction of the d-j dot products v^T A[:, j..d)
// (which also yields ||A[j:, j]||^2), done as per-CTA partials + a sliced
// second-level sum, and a rank-1 update of each CTA's own rows.  Grid barriers are
// bounded spins (ST_TIMEOUT after ~1 s, never a hang).
#include "slse_internal.cuh"

namespace slse {
namespace {

constexpr int kQrThreads = 256;

struct QrArgs {
  double *A;
  int64_t r, lda;
  int d;
  double *R;
  double *Rt;    // R^T (d x d), nullable
  double *red;   // 2 x G x d
  double *fin;   // 2 x d
  double *piv;   // 2 x d
  DevState *st;
};

// Rows of each CTA live in shared memory for the whole factorisation (SMEM = true)
// when they fit; otherwise they stay in global memory.
template <bool SMEM>
__global__ void __launch_bounds__(kQrThreads) k_qr(const QrArgs a) {
  extern __shared__ double sA[];
  const int G = gridDim.x, b = blockIdx.x;
  const int d = a.d;
  const int64_t r = a.r;
  const int64_t rb0 = (r * b) / G, rb1 = (r * (b + 1)) / G;
  const int nr = (int)(rb1 - rb0);
  double *A = a.A;
  // own row i lives at rowp(i)[0..d)
  const int64_t ld = SMEM ? d : a.lda;
  double *own = SMEM ? sA : A + rb0 * a.lda;
  if (SMEM) {
    for (int64_t e = threadIdx.x; e < (int64_t)nr * d; e += kQrThreads)
      sA[e] = A[(rb0 + e / d) * a.lda + e % d];
    __syncthreads();
  }
  for (int j = 0; j < d; ++j) {
    const int nc = d - j;
    const int buf = j & 1;
    double *red = a.red + (size_t)buf * G * d;
    double *fin = a.fin + (size_t)buf * d;
    double *piv = a.piv + (size_t)buf * d;
    const int lo = (int)((rb0 > j ? rb0 : j) - rb0);
    const bool has_j = j >= rb0 && j < rb1;
    // phase 1: partial dot products of column j with columns j..d-1 over own rows
    for (int c = threadIdx.x; c < nc; c += kQrThreads) {
      double s = 0.0;
      for (int i = lo; i < nr; ++i) s = fma(own[i * ld + j], own[i * ld + j + c], s);
      red[(size_t)b * d + c] = s;
      if (has_j) piv[c] = own[(j - rb0) * ld + j + c];
    }
    if (!grid_barrier(a.st, G)) return;
    // phase 2: CTA b sums a slice of the columns over all CTAs; each column is summed by
    // 64 threads (strided partials, then a fixed-order shuffle/shared-memory tree)
    {
      __shared__ double s_red[kQrThreads / 32];
      const int c0 = (int)(((int64_t)nc * b) / G), c1 = (int)(((int64_t)nc * (b + 1)) / G);
      const int sub = threadIdx.x & 63, grp = threadIdx.x >> 6;
      for (int cb = c0; cb < c1; cb += kQrThreads / 64) {
        const int c = cb + grp;
        double s = 0.0;
        if (c < c1)
          for (int q = sub; q < G; q += 64) s += __ldcg(red + (size_t)q * d + c);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (sub == 0 && c < c1) fin[c] = s_red[2 * grp] + s_red[2 * grp + 1];
        __syncthreads();
      }
    }
    if (!grid_barrier(a.st, G)) return;
    // phase 3: Householder reflector from column j, applied to own rows
    const double nrm2 = __ldcg(fin);
    const double ajj = __ldcg(piv);
    if (nrm2 > 0.0) {
      const double nrm = sqrt(nrm2);
      const double alpha = ajj >= 0.0 ? -nrm : nrm;
      const double vj = ajj - alpha;
      const double tau = 1.0 / (nrm * (nrm + fabs(ajj)));  // 2 / v^T v
      for (int c = 1 + threadIdx.x; c < nc; c += kQrThreads) {
        const double tw = tau * (__ldcg(fin + c) - alpha * __ldcg(piv + c));  // tau * v^T A[:, j+c]
        for (int i = lo; i < nr; ++i) {
          const double vi = (i + rb0 == j) ? vj : own[i * ld + j];
          own[i * ld + j + c] -= vi * tw;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && has_j) own[(j - rb0) * ld + j] = alpha;
    } else if (threadIdx.x == 0 && b == 0) {
      atomicOr(&a.st->status, ST_NUMERIC);
    }
    __syncthreads();
  }
  if (SMEM) {  // rows < d hold R: write them back
    for (int64_t e = threadIdx.x; e < (int64_t)nr * d; e += kQrThreads) {
      const int64_t i = rb0 + e / d;
      if (i < d) A[i * a.lda + e % d] = sA[e];
    }
  }
  if (!grid_barrier(a.st, G)) return;
  // R = upper triangle of A[0:d, 0:d] with rows scaled to a non-negative diagonal; Rt = R^T
  for (int64_t e = (int64_t)b * kQrThreads + threadIdx.x; e < (int64_t)d * d; e += (int64_t)G * kQrThreads) {
    const int i = (int)(e / d), k = (int)(e % d);
    const double diag = __ldcg(A + (int64_t)i * a.lda + i);
    const double sgn = diag < 0.0 ? -1.0 : 1.0;
    const double v = k >= i ? sgn * __ldcg(A + (int64_t)i * a.lda + k) : 0.0;
    a.R[e] = v;
    if (a.Rt) a.Rt[(int64_t)k * d + i] = v;
  }
}

// Column k of R^{-1} by column sweep: x_i = b_i / R_ii, then b[0:i) -= x_i R[0:i, i],
// for i = k..0, one warp per column.  b is spread over the lanes (b[32t + lane] in
// register t); the critical path per step is one shuffle and one multiply.
__global__ void __launch_bounds__(256) k_tri_inv_sweep(const double *R, const double *Rt, int d, double *Rinv,
                                                       DevState *st) {
  __shared__ double s_rdiag[512];
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double rii = R[(size_t)i * d + i];
    if (rii == 0.0) atomicOr(&st->status, ST_NUMERIC);
    s_rdiag[i] = 1.0 / rii;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blockIdx.x * 8 + warp;
  if (k >= d) return;
  double bv[16], xv[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    bv[t] = (32 * t + lane == k) ? 1.0 : 0.0;
    xv[t] = 0.0;
  }
#pragma unroll
  for (int t = 15; t >= 0; --t) {
    if (32 * t > k) continue;
    const int top = (k - 32 * t) < 31 ? (k - 32 * t) : 31;
#pragma unroll 4
    for (int ln = top; ln >= 0; --ln) {
      const int i = 32 * t + ln;
      const double xi = __shfl_sync(0xffffffffu, bv[t], ln) * s_rdiag[i];
      if (lane == ln) xv[t] = xi;
      const double *col = Rt + (size_t)i * d;  // column i of R
#pragma unroll
      for (int tt = 0; tt <= t; ++tt) {
        const int l = 32 * tt + lane;
        if (l < i) bv[tt] = fma(-xi, col[l], bv[tt]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int l = 32 * t + lane;
    if (l < d) Rinv[(size_t)l * d + k] = l <= k ? xv[t] : 0.0;
  }
}

// Hinv[i][k] = sum_{l >= max(i,k)} Rinv[i][l] Rinv[k][l], 32 x 32 output tiles.
__global__ void __launch_bounds__(256) k_form_hinv(const double *Rinv, int d, double *Hinv) {
  __shared__ double sa[32][33], sb[32][33];
  const int ti = blockIdx.y, tk = blockIdx.x;
  if (tk < ti) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of threads
  double acc[4] = {0, 0, 0, 0};
  const int lstart = tk * 32;  // Rinv[k][l] = 0 for l < k, and k >= tk*32 >= i
  for (int l0 = lstart; l0 < d; l0 += 32) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int gi = ti * 32 + rr, gk = tk * 32 + rr, gl = l0 + tx;
      sa[rr][tx] = (gi < d && gl < d) ? Rinv[(size_t)gi * d + gl] : 0.0;
      sb[rr][tx] = (gk < d && gl < d) ? Rinv[(size_t)gk * d + gl] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int rr = ty + 8 * q;
      double s = acc[q];
      for (int l = 0; l < 32; ++l) s = fma(sa[rr][l], sb[tx][l], s);
      acc[q] = s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gi = ti * 32 + ty + 8 * q, gk = tk * 32 + tx;
    if (gi < d && gk < d) {
      Hinv[(size_t)gi * d + gk] = acc[q];
      Hinv[(size_t)gk * d + gi] = acc[q];
    }
  }
}

// ---------------------------------------------------------------- Gram + Cholesky route
// For the BF16 Hessian sketch (mixed path) R is obtained as the Cholesky factor of
// G = (S-hat X)^T (S-hat X) (the R of a Householder QR with non-negative diagonal is the
// same matrix).  G is accumulated from exact FP32 products of the BF16 entries with a
// two-word (TwoSum) accumulator per entry, split over row ranges, and summed in FP64 in a
// fixed order; the factorisation is FP64.

constexpr int kTile = 32;

__device__ __forceinline__ float bf16_to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// part[s][i][k] = sum over rows of split s of U[row][i] * U[row][k], upper tiles only.
__global__ void __launch_bounds__(256) k_gram_bf16(const __nv_bfloat16 *U, int64_t ldu, int64_t row0, int64_t r,
                                                   int d, int ksplit, double *part) {
  __shared__ float sa[kTile][kTile + 1], sb[kTile][kTile + 1];
  const int ti = blockIdx.y, tk = blockIdx.x, sp = blockIdx.z;
  if (tk < ti) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t lo = (r * sp) / ksplit, hi = (r * (sp + 1)) / ksplit;
  float sh[4] = {0, 0, 0, 0}, sl[4] = {0, 0, 0, 0};
  for (int64_t k0 = lo; k0 < hi; k0 += kTile) {
    for (int rr = ty; rr < kTile; rr += 8) {
      const int64_t row = k0 + rr;
      const int ci = ti * kTile + tx, ck = tk * kTile + tx;
      const bool rv = row < hi;
      sa[rr][tx] = (rv && ci < d) ? bf16_to_f(U[(row0 + row) * ldu + ci]) : 0.f;
      sb[rr][tx] = (rv && ck < d) ? bf16_to_f(U[(row0 + row) * ldu + ck]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ii = ty + 8 * q;
      float s = sh[q], c = sl[q];
#pragma unroll 8
      for (int rr = 0; rr < kTile; ++rr) {
        const float p = sa[rr][ii] * sb[rr][tx];  // exact: 8-bit x 8-bit significands
        float e;
        two_sum(s, p, s, e);
        c += e;
      }
      sh[q] = s;
      sl[q] = c;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gi = ti * kTile + ty + 8 * q, gk = tk * kTile + tx;
    if (gi < d && gk < d) part[((size_t)sp * d + gi) * d + gk] = (double)sh[q] + (double)sl[q];
  }
}

// G[i][k] = G[k][i] = scale * sum_s part[s][i][k] for i <= k.
__global__ void k_gram_reduce(const double *part, int ksplit, int d, double scale, double *G) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * d) return;
  const int i = (int)(e / d), k = (int)(e % d);
  if (k < i) return;
  double s = 0.0;
  for (int sp = 0; sp < ksplit; ++sp) s += part[((size_t)sp * d + i) * d + k];
  G[(size_t)i * d + k] = scale * s;
  G[(size_t)k * d + i] = scale * s;
}

// Diagonal block [k0, k0+nb) of the right-looking blocked Cholesky (lower, in place), and
// the inverse of that block for the panel solve.  Four warps (one per SM sub-partition:
// a warp's FP64 instruction occupies its sub-partition's FP64 pipe for many cycles on this
// part, so the work is spread over all four).  Lane i holds row i; warp w holds columns
// l = w + 4t (t < 8) in registers.  Step j: the owner of column j takes the pivot (rsqrt),
// scales the column and publishes it in shared memory; after one barrier every warp
// updates its columns l > j.  The inverse is formed by a column sweep with the same split.
// Rows past d are identity rows; a non-positive pivot raises ST_NUMERIC.
__global__ void __launch_bounds__(128) k_potrf(double *A, int d, int k0, double *Linv, DevState *st) {
  __shared__ double s_col[kTile][kTile + 1];  // s_col[j][i] = L[i][j]
  __shared__ double s_rinv[kTile];
  __shared__ int s_bad;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nb = min(kTile, d - k0);
  constexpr int TC = kTile / 4;  // columns per warp
  double a[TC];
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    const int l = w + 4 * t;
    a[t] = (lane < nb && l < nb && l <= lane) ? A[(size_t)(k0 + lane) * d + k0 + l] : (l == lane ? 1.0 : 0.0);
  }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
#pragma unroll 1
  for (int j = 0; j < kTile; ++j) {
    if (w == (j & 3)) {
      const int tj = j >> 2;
      double aj = 0.0;
#pragma unroll
      for (int t = 0; t < TC; ++t)
        if (t == tj) aj = a[t];
      const double piv = __shfl_sync(0xffffffffu, aj, j);
      const bool ok = piv > 0.0;
      const double rs = ok ? rsqrt(piv) : 0.0;
      const double lj = lane == j ? piv * rs : (lane > j ? aj * rs : 0.0);
#pragma unroll
      for (int t = 0; t < TC; ++t)
        if (t == tj) a[t] = lj;
      s_col[j][lane] = lj;
      if (lane == 0) {
        s_rinv[j] = rs;
        if (!ok) s_bad = 1;
      }
    }
    __syncthreads();
    if (s_bad) {
      if (threadIdx.x == 0) atomicOr(&st->status, ST_NUMERIC);
      return;
    }
    const double lij = s_col[j][lane];
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      const int l = w + 4 * t;
      if (l > j) a[t] = fma(-lij, s_col[j][l], a[t]);
    }
  }
  // L back to A (lower triangle of the block)
  if (lane < nb) {
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      const int l = w + 4 * t;
      if (l < nb) A[(size_t)(k0 + lane) * d + k0 + l] = l <= lane ? a[t] : 0.0;
    }
  }
  // L^{-1}: column c = w + 4t of the inverse in x[t] (lane = row); sweep i = 0..31:
  // x_i <- x_i / L_ii, then x_r <- x_r - L_ri x_i for r > i
  double x[TC];
#pragma unroll
  for (int t = 0; t < TC; ++t) x[t] = (lane == w + 4 * t) ? 1.0 : 0.0;
#pragma unroll 1
  for (int i = 0; i < kTile; ++i) {
    const double rinv = s_rinv[i], lri = s_col[i][lane];
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      const double xi = __shfl_sync(0xffffffffu, x[t], i) * rinv;
      x[t] = lane == i ? xi : (lane > i ? fma(-lri, xi, x[t]) : x[t]);
    }
  }
  if (lane < nb) {
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      const int c = w + 4 * t;
      if (c < nb) Linv[lane * kTile + c] = lane >= c ? x[t] : 0.0;
    }
  }
}

// Panel below the diagonal block: A[i0:i0+8, k0:k0+nb] <- A * Linv^T, 8 rows per CTA (one
// output per thread) so that the FP64 work spreads over many SMs.
__global__ void __launch_bounds__(256) k_trsm(double *A, int d, int k0, const double *Linv) {
  __shared__ double P[8][kTile + 1], T[kTile][kTile + 1];
  const int nb = min(kTile, d - k0);
  const int i0 = k0 + kTile + 8 * blockIdx.x;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  P[ty][tx] = (i0 + ty < d && tx < nb) ? A[(size_t)(i0 + ty) * d + k0 + tx] : 0.0;
  for (int rr = ty; rr < kTile; rr += 8) T[rr][tx] = (rr < nb && tx < nb) ? Linv[rr * kTile + tx] : 0.0;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int l = 0; l < kTile; ++l) s = fma(P[ty][l], T[tx][l], s);  // (P Linv^T)[ty][tx]
  if (i0 + ty < d && tx < nb) A[(size_t)(i0 + ty) * d + k0 + tx] = s;
}

// Trailing update of the lower triangle: A[rows, cols] -= L[rows, k] L[cols, k]^T for the
// 8-row slice blockIdx.y of the trailing part against the 32-column block blockIdx.x
// (lower triangle only), one output per thread.
__global__ void __launch_bounds__(256) k_syrk(double *A, int d, int k0) {
  __shared__ double Li[8][kTile + 1], Lj[kTile][kTile + 1];
  const int nb = min(kTile, d - k0);
  const int base = k0 + kTile;
  const int i0 = base + 8 * blockIdx.y, j0 = base + kTile * blockIdx.x;
  if (j0 > i0 + 7) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  Li[ty][tx] = (i0 + ty < d && tx < nb) ? A[(size_t)(i0 + ty) * d + k0 + tx] : 0.0;
  for (int rr = ty; rr < kTile; rr += 8) Lj[rr][tx] = (j0 + rr < d && tx < nb) ? A[(size_t)(j0 + rr) * d + k0 + tx] : 0.0;
  __syncthreads();
  const int gi = i0 + ty, gj = j0 + tx;
  if (gi < d && gj < d && gj <= gi) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < kTile; ++l) s = fma(Li[ty][l], Lj[tx][l], s);
    A[(size_t)gi * d + gj] -= s;
  }
}

// R = L^T (upper, positive diagonal) and Rt = L (lower with zeros above).
__global__ void k_chol_to_r(const double *A, int d, double *R, double *Rt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * d) return;
  const int i = (int)(e / d), k = (int)(e % d);
  const double l = k <= i ? A[e] : 0.0;  // L[i][k]
  Rt[e] = l;
  R[(size_t)k * d + i] = l;
}

template <class T> __device__ __forceinline__ double to_d(T v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <class T>
__global__ void k_gather(const T *U, int64_t ldu, int64_t row0, int64_t r, int d, double scale, double *A) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * d) return;
  const int64_t i = e / d;
  const int c = (int)(e % d);
  A[e] = scale * to_d(U[(row0 + i) * ldu + c]);
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int qr_grid(int64_t r, int nsm) {
  int64_t g = (r + 7) / 8;  // at least ~8 rows per CTA
  if (g > nsm) g = nsm;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

size_t qr_ws_bytes(int64_t r, int d, int nsm) {
  const int G = qr_grid(r, nsm);
  return align256(2 * (size_t)G * d * 8) + 2 * align256(2 * (size_t)d * 8) + 2 * align256((size_t)d * d * 8);
}

cudaError_t launch_gather_hessian_rows(int prec, const void *U, int64_t ldu, int64_t row0, int64_t r, int d,
                                       double scale, double *A, cudaStream_t s) {
  const int64_t n = r * d;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (prec == SLSE_PREC_FP64)
    k_gather<double><<<grid, 256, 0, s>>>(static_cast<const double *>(U), ldu, row0, r, d, scale, A);
  else
    k_gather<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(U), ldu, row0, r, d, scale, A);
  return cudaGetLastError();
}

// A is overwritten (it must be a scratch copy).  ws: qr_ws_bytes(r, d).
cudaError_t launch_qr(double *A, int64_t r, int d, int64_t lda, double *R, double *Hinv, void *ws, DevState *st,
                      cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int G = qr_grid(r, nsm);
  const int64_t nr_max = (r + G - 1) / G;
  const size_t smem = (size_t)nr_max * d * sizeof(double);
  const bool use_smem = smem <= (size_t)200 * 1024;
  auto kern = use_smem ? k_qr<true> : k_qr<false>;
  const size_t dyn = use_smem ? smem : 0;
  if (use_smem) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kQrThreads, dyn);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  char *p = static_cast<char *>(ws);
  size_t off = 0;
  QrArgs a;
  a.A = A;
  a.r = r;
  a.lda = lda;
  a.d = d;
  a.R = R;
  a.red = reinterpret_cast<double *>(p + off); off += align256(2 * (size_t)G * d * 8);
  a.fin = reinterpret_cast<double *>(p + off); off += align256(2 * (size_t)d * 8);
  a.piv = reinterpret_cast<double *>(p + off); off += align256(2 * (size_t)d * 8);
  double *Rinv = reinterpret_cast<double *>(p + off); off += align256((size_t)d * d * 8);
  a.Rt = reinterpret_cast<double *>(p + off); off += align256((size_t)d * d * 8);
  a.st = st;
  void *args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(kQrThreads), args, dyn, s);
  if (e != cudaSuccess) return e;
  if (Hinv) {
    k_tri_inv_sweep<<<(d + 7) / 8, 256, 0, s>>>(R, a.Rt, d, Rinv, st);
    const int nt = (d + 31) / 32;
    k_form_hinv<<<dim3(nt, nt), 256, 0, s>>>(Rinv, d, Hinv);
  }
  return cudaGetLastError();
}

size_t chol_ws_bytes(int64_t r, int d) {
  const int ksplit = (int)((r + 255) / 256 < 8 ? (r + 255) / 256 : 8);
  return align256((size_t)(ksplit > 0 ? ksplit : 1) * d * d * 8) + align256((size_t)d * d * 8) +
         align256((size_t)kTile * kTile * 8) + 2 * align256((size_t)d * d * 8);
}

cudaError_t launch_gram_chol(const void *U, int64_t ldu, int64_t row0, int64_t r, int d, double scale2, double *R,
                             double *Hinv, void *ws, DevState *st, cudaStream_t s) {
  int ksplit = (int)((r + 255) / 256);
  if (ksplit > 8) ksplit = 8;
  if (ksplit < 1) ksplit = 1;
  char *p = static_cast<char *>(ws);
  size_t off = 0;
  double *part = reinterpret_cast<double *>(p + off); off += align256((size_t)ksplit * d * d * 8);
  double *G = reinterpret_cast<double *>(p + off); off += align256((size_t)d * d * 8);
  double *Linv = reinterpret_cast<double *>(p + off); off += align256((size_t)kTile * kTile * 8);
  double *Rinv = reinterpret_cast<double *>(p + off); off += align256((size_t)d * d * 8);
  double *Rt = reinterpret_cast<double *>(p + off); off += align256((size_t)d * d * 8);
  const int nt = (d + kTile - 1) / kTile;
  k_gram_bf16<<<dim3(nt, nt, ksplit), 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(U), ldu, row0, r, d, ksplit, part);
  const int64_t dd = (int64_t)d * d;
  k_gram_reduce<<<(unsigned)((dd + 255) / 256), 256, 0, s>>>(part, ksplit, d, scale2, G);
  for (int kb = 0; kb < nt; ++kb) {
    const int k0 = kb * kTile;
    k_potrf<<<1, 128, 0, s>>>(G, d, k0, Linv, st);
    const int below = nt - kb - 1;
    if (below > 0) {
      const int rows = d - k0 - kTile;  // rows below the diagonal block
      const int slices = (rows + 7) / 8;
      k_trsm<<<slices, 256, 0, s>>>(G, d, k0, Linv);
      k_syrk<<<dim3(below, slices), 256, 0, s>>>(G, d, k0);
    }
  }
  k_chol_to_r<<<(unsigned)((dd + 255) / 256), 256, 0, s>>>(G, d, R, Rt);
  if (Hinv) {
    k_tri_inv_sweep<<<(d + 7) / 8, 256, 0, s>>>(R, Rt, d, Rinv, st);
    k_form_hinv<<<dim3(nt, nt), 256, 0, s>>>(Rinv, d, Hinv);
  }
  return cudaGetLastError();
}

}  // namespace slse
