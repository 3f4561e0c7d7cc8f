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

// ---------------------------------------------------------------- Gram + sweep route
// For the BF16 Hessian sketch (mixed path) H-hat^{-1} is formed directly from
// G = (S-hat X)^T (S-hat X), which equals R^T R for the R of a Householder QR of S-hat X.
// G is accumulated from exact FP32 products of the BF16 entries with a two-word (TwoSum)
// accumulator per entry, split over row ranges, and summed in FP64 in a fixed order.
// G^{-1} then comes from the sweep operator (Goodnight 1979) applied block by block in FP64:
// sweeping the diagonal block P = A_kk of a symmetric matrix A gives
//   A_kk <- -P^{-1},  A_ik <- A_ik P^{-1},  A_kj <- P^{-1} A_kj,  A_ij <- A_ij - A_ik P^{-1} A_kj,
// and sweeping every block leaves -G^{-1}.  Each pivot P is a Schur complement of the
// positive definite G, hence positive definite; a non-positive scalar pivot inside it
// raises ST_NUMERIC (the caller then takes the Householder QR of the rows).  Rows and
// columns past d are padded with the identity.

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

// A (dp x dp, dp = d rounded up to 32): A[i][k] = A[k][i] = scale * sum_s part[s][i][k] for
// i <= k < d, the identity outside the d x d block.
__global__ void k_sweep_load(const double *part, int ksplit, int d, int dp, double scale, double *A) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)dp * dp) return;
  const int i = (int)(e / dp), k = (int)(e % dp);
  double v;
  if (i < d && k < d) {
    const int a = i < k ? i : k, b = i < k ? k : i;
    double s = 0.0;
    for (int sp = 0; sp < ksplit; ++sp) s += part[((size_t)sp * d + a) * d + b];
    v = scale * s;
  } else {
    v = i == k ? 1.0 : 0.0;
  }
  A[e] = v;
}

// 1 / v from the FP32 reciprocal refined by one FP64 Newton step (relative error ~2^-46),
// the exact quotient when v is outside the FP32 range.
__device__ __forceinline__ double recip_fast(double v) {
  const float f = (float)v;
  if (!(fabsf(f) > 0x1p-120f) || !(fabsf(f) < 0x1p120f)) return 1.0 / v;
  const double x0 = (double)__frcp_rn(f);
  return fma(x0, fma(-v, x0, 1.0), x0);
}

// Pivot step k, CTA (b, q4): sweeps its own copy of P = A_kk (32 scalar sweeps in shared
// memory) into S = -P^{-1}; CTA (k, q4) stores columns 8 q4 .. 8 q4 + 7 of S in W_k, every
// other CTA the same columns of C_b = A_bk (the column block before the step) and of
// W_b = A_bk P^{-1} = -A_bk S.  Only the lower triangle of A is kept: A_bk for b < k is read
// as (A_kb)^T.  In the sweep, thread t owns entries (t div 8, t mod 8 + 8q), q < 4; the
// thread that writes the next pivot also forms its reciprocal.
__global__ void __launch_bounds__(256) k_sweep_pivot(const double *A, int dp, int k, double *W, double *C,
                                                     DevState *st) {
  __shared__ double P[kTile][kTile + 1];
  __shared__ double T[kTile][kTile + 1];
  __shared__ double s_inv[2];
  __shared__ int s_bad;
  const int t = threadIdx.x, b = blockIdx.x, q4 = blockIdx.y;
  const int r = t >> 3, c0 = t & 7;
  const double *Akk = A + (size_t)k * kTile * dp + (size_t)k * kTile;
  for (int e = t; e < kTile * kTile; e += 256) {
    const int er = e >> 5, ec = e & 31;
    P[er][ec] = er >= ec ? Akk[(size_t)er * dp + ec] : Akk[(size_t)ec * dp + er];
    if (b > k) T[er][ec] = A[(size_t)(b * kTile + er) * dp + k * kTile + ec];
    else if (b < k) T[er][ec] = A[(size_t)(k * kTile + ec) * dp + b * kTile + er];
  }
  if (t == 0) s_bad = 0;
  __syncthreads();
  if (t == 0) {
    const double p0 = P[0][0];
    if (!(p0 > 0.0)) s_bad = 1;
    s_inv[0] = recip_fast(p0);
  }
  __syncthreads();
  // One FMA per entry: v = h - f_r g_c with f_r = P[r][j]/p (r != j) or -1/p (r == j),
  // g_c = P[j][c] (c != j) or -1 (c == j), and h = P[r][c] off row and column j, else 0;
  // this gives P[r][c] - P[r][j] P[j][c]/p, P[j][c]/p, P[r][j]/p and -1/p in the four cases.
  for (int j = 0; j < kTile; ++j) {
    const double inv = s_inv[j & 1];
    const double prj = P[r][j];
    double g[4], h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + 8 * q;
      g[q] = c == j ? -1.0 : P[j][c];
      h[q] = (c == j || r == j) ? 0.0 : P[r][c];
    }
    __syncthreads();
    const double f = r == j ? -inv : prj * inv;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + 8 * q;
      const double v = fma(-f, g[q], h[q]);
      P[r][c] = v;
      if (r == j + 1 && c == j + 1) {  // the next pivot
        if (!(v > 0.0)) s_bad = 1;
        s_inv[(j + 1) & 1] = recip_fast(v);
      }
    }
    __syncthreads();
  }
  if (s_bad && t == 0 && q4 == 0) atomicOr(&st->status, ST_NUMERIC);
  // columns 8 q4 .. 8 q4 + 7: one output per thread
  const int c = 8 * q4 + c0;
  double *Wb = W + (size_t)b * kTile * kTile;
  if (b == k) {
    Wb[r * kTile + c] = P[r][c];
    return;
  }
  double acc = 0.0;
#pragma unroll 8
  for (int l = 0; l < kTile; ++l) acc = fma(T[r][l], P[l][c], acc);
  Wb[r * kTile + c] = -acc;
  C[(size_t)b * kTile * kTile + r * kTile + c] = T[r][c];
}

// Update of lower tile (i, j), i >= j, for pivot step k (tile index from the linear block id):
//   (k, k): -P^{-1};  (i, k): W_i;  (k, j): W_j^T;  otherwise A_ij - W_i C_j^T.
__global__ void __launch_bounds__(256) k_sweep_update(double *A, int dp, int k, const double *W, const double *C) {
  __shared__ double Ws[kTile][kTile + 1], Cs[kTile][kTile + 1];
  int i = 0, rem = blockIdx.x;
  while (rem > i) { rem -= i + 1; ++i; }
  const int j = rem;
  const int t = threadIdx.x, r = t >> 3, c0 = t & 7;
  double *Aij = A + (size_t)i * kTile * dp + (size_t)j * kTile;
  if (i == k || j == k) {
    const double *src = W + (size_t)(j == k ? i : j) * kTile * kTile;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + 8 * q;
      Aij[(size_t)r * dp + c] = j == k ? src[r * kTile + c] : src[c * kTile + r];
    }
    return;
  }
  const double *Wi = W + (size_t)i * kTile * kTile, *Cj = C + (size_t)j * kTile * kTile;
  for (int e = t; e < kTile * kTile; e += 256) {
    Ws[e >> 5][e & 31] = Wi[e];
    Cs[e >> 5][e & 31] = Cj[e];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = c0 + 8 * q;
    double acc = Aij[(size_t)r * dp + c];
#pragma unroll 8
    for (int l = 0; l < kTile; ++l) acc = fma(-Ws[r][l], Cs[c][l], acc);
    Aij[(size_t)r * dp + c] = acc;
  }
}

// Hinv = -G^{-1} read from the lower triangle of the swept matrix (leading d x d block).
__global__ void k_sweep_final(const double *A, int d, int dp, double *Hinv) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * d) return;
  const int i = (int)(e / d), k = (int)(e % d);
  Hinv[e] = i >= k ? -A[(size_t)i * dp + k] : -A[(size_t)k * dp + i];
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

size_t sweep_ws_bytes(int64_t r, int d) {
  const int ksplit = (int)((r + 255) / 256 < 8 ? (r + 255) / 256 : 8);
  const size_t dp = (size_t)(d + kTile - 1) / kTile * kTile;
  return align256((size_t)(ksplit > 0 ? ksplit : 1) * d * d * 8) + align256(dp * dp * 8) + 2 * align256(dp * kTile * 8);
}

cudaError_t launch_gram_sweep(const void *U, int64_t ldu, int64_t row0, int64_t r, int d, double scale2,
                              double *Hinv, void *ws, DevState *st, cudaStream_t s) {
  int ksplit = (int)((r + 255) / 256);
  if (ksplit > 8) ksplit = 8;
  if (ksplit < 1) ksplit = 1;
  const int nb = (d + kTile - 1) / kTile, dp = nb * kTile;
  char *p = static_cast<char *>(ws);
  size_t off = 0;
  double *part = reinterpret_cast<double *>(p + off); off += align256((size_t)ksplit * d * d * 8);
  double *A = reinterpret_cast<double *>(p + off); off += align256((size_t)dp * dp * 8);
  double *W = reinterpret_cast<double *>(p + off); off += align256((size_t)dp * kTile * 8);
  double *C = reinterpret_cast<double *>(p + off);
  k_gram_bf16<<<dim3(nb, nb, ksplit), 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(U), ldu, row0, r, d, ksplit, part);
  const int64_t ee = (int64_t)dp * dp;
  k_sweep_load<<<(unsigned)((ee + 255) / 256), 256, 0, s>>>(part, ksplit, d, dp, scale2, A);
  for (int k = 0; k < nb; ++k) {
    k_sweep_pivot<<<dim3(nb, 4), 256, 0, s>>>(A, dp, k, W, C, st);
    k_sweep_update<<<nb * (nb + 1) / 2, 256, 0, s>>>(A, dp, k, W, C);
  }
  const int64_t dd = (int64_t)d * d;
  k_sweep_final<<<(unsigned)((dd + 255) / 256), 256, 0, s>>>(A, d, dp, Hinv);
  return cudaGetLastError();
}

}  // namespace slse
