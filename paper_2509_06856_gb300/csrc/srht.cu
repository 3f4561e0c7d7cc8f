// SRHT of the tall data [X | Y] (paper Sec. 3): Z = H D P X_pad, followed by the
// row sampling B.  H is the Sylvester-order Walsh-Hadamard matrix
// H[k, j] = (-1)^popcount(k & j); the 1/sqrt(N') normalisation and the sampling
// scale are one scalar applied at the output.
//
// Structure (GB300): the N'-point transform along rows is split by the Kronecker
// identity H_{N'} = H_{n1} (x) H_{n2} (row index j = j1 n2 + j2) into two streaming
// passes over HBM:
//   pass 1: for each block j1 of n2 consecutive rows of D P X_pad (a row gather
//           through the sign-folded permutation), apply H_{n2} down every column;
//           write the intermediate W (row-major, N' rows);
//   pass 2: for each k2, apply H_{n1} to the n1 rows W[j1 n2 + k2] (stride n2),
//           scale, and write only the rows the sketch keeps, compacted in sampling
//           order (pos[k] = position of row k in sigma, or -1).
// Small N' (<= 2^9) uses one pass.
//
// One transform "group" (n rows x C columns) is held on chip: a cluster of
// Q = 2^LOGQ CTAs each keeps 2^LOGM consecutive rows x C columns in shared memory
// (64 KB).  Each CTA applies the butterflies of the low LOGM row bits in registers
// (two register stages with one shared-memory exchange); the top LOGQ bits are
// combined across the cluster through distributed shared memory.  Global loads and
// stores move whole row segments (C = 32 FP32 or 16 FP64 columns = 128 bytes) so
// every warp access is coalesced.  The work is adds/subtracts only: HBM-bound in
// FP32, FP64-ALU-bound in FP64 on this part.
#include <cooperative_groups.h>

#include "slse_internal.cuh"

namespace cg = cooperative_groups;

namespace slse {
namespace {

struct GroupArgs {
  const void *in;       // X (pass 1 / single) or W (pass 2)
  int64_t ldin;
  const void *in_y;     // Y or WY
  int64_t N;            // gather mode: rows >= N are the zero padding
  const int32_t *Psd;   // non-null: gather mode (sign-folded permutation)
  int64_t istride, igstride;  // input row j = rho * istride + g * igstride
  void *out;
  int64_t ldout;
  void *out_y;
  const int32_t *pos;   // non-null: output row = pos[k], skipped when < 0
  int64_t ostride, ogstride;  // output index k = kappa * ostride + g * ogstride
  int d;
  int nslab;
  int logq;
  double scale;
};

template <class T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class Ts, class Tin> __device__ __forceinline__ Ts load_cvt(const Tin *p) {
  if constexpr (sizeof(Ts) == 8) return (Ts)(*p);
  else return to_f<Tin>(*p);
}
template <> __device__ __forceinline__ double load_cvt<double, __nv_bfloat16>(const __nv_bfloat16 *p) {
  return (double)__bfloat162float(*p);
}

template <class Tout, class Ts> __device__ __forceinline__ void store_cvt(Tout *p, Ts v) {
  if constexpr (sizeof(Tout) == 2) *p = __float2bfloat16_rn((float)v);
  else *p = (Tout)v;
}

template <class Ts, class Tin>
__device__ __forceinline__ Ts load_elem(const GroupArgs &a, int64_t g, int64_t rho, int col) {
  const int64_t j = rho * a.istride + g * a.igstride;
  int64_t src = j;
  bool neg = false;
  if (a.Psd) {
    const int32_t v = __ldg(a.Psd + j);
    neg = v < 0;
    src = neg ? (int64_t)(~v) : (int64_t)v;
    if (src >= a.N) return Ts(0);
  }
  Ts x;
  if (col < a.d) x = load_cvt<Ts>(static_cast<const Tin *>(a.in) + src * a.ldin + col);
  else if (col == a.d) x = load_cvt<Ts>(static_cast<const Tin *>(a.in_y) + src);
  else x = Ts(0);
  return neg ? -x : x;
}

template <class Tout, class Ts>
__device__ __forceinline__ void store_elem(const GroupArgs &a, int64_t g, int64_t kappa, int col, Ts v) {
  if (col > a.d) return;
  const int64_t k = kappa * a.ostride + g * a.ogstride;
  int64_t dst = k;
  if (a.pos) {
    dst = __ldg(a.pos + k);
    if (dst < 0) return;
  }
  v = v * (Ts)a.scale;
  if (col < a.d) store_cvt(static_cast<Tout *>(a.out) + dst * a.ldout + col, v);
  else store_cvt(static_cast<Tout *>(a.out_y) + dst, v);
}

template <int R, class T> __device__ __forceinline__ void fwht_regs(T (&v)[R]) {
#pragma unroll
  for (int h = 1; h < R; h <<= 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if ((i & h) == 0) {
        const T x = v[i], y = v[i + h];
        v[i] = x + y;
        v[i + h] = x - y;
      }
    }
  }
}

// Group transform: 2^LOGM rows x C columns per CTA, Q = 2^logq CTAs per cluster.
template <class Tin, class Ts, class Tout, int LOGM, int C, int NT>
__global__ void __launch_bounds__(NT) k_group(const GroupArgs a) {
  constexpr int M = 1 << LOGM;
  constexpr int S1 = LOGM <= 5 ? 0 : LOGM / 2;   // low-bit stage
  constexpr int S0 = LOGM - S1;                  // high-bit stage (first, loads from HBM)
  constexpr int RA = 1 << S0, RB = 1 << S1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Ts *tile = reinterpret_cast<Ts *>(smem_raw);

  const int Q = 1 << a.logq;
  const int rank = (int)(blockIdx.x & (unsigned)(Q - 1));
  const int64_t item = (int64_t)(blockIdx.x >> a.logq);
  const int slab = (int)(item % a.nslab);
  const int64_t g = item / a.nslab;
  const int col0 = slab * C;
  const int64_t rho0 = (int64_t)rank * M;
  const bool direct_out = (Q == 1) && (S1 == 0);

  // stage A: bits [S1, LOGM) of the local row index; loads the group rows from HBM
  for (int it = threadIdx.x; it < (C << S1); it += NT) {
    const int c = it % C, b = it / C;
    Ts v[RA];
#pragma unroll
    for (int k = 0; k < RA; ++k) v[k] = load_elem<Ts, Tin>(a, g, rho0 + b + (k << S1), col0 + c);
    fwht_regs<RA, Ts>(v);
    if (direct_out) {
#pragma unroll
      for (int k = 0; k < RA; ++k) store_elem<Tout, Ts>(a, g, rho0 + b + (k << S1), col0 + c, v[k]);
    } else {
#pragma unroll
      for (int k = 0; k < RA; ++k) tile[(b + (k << S1)) * C + c] = v[k];
    }
  }
  if constexpr (S1 > 0) {
    __syncthreads();
    // stage B: bits [0, S1)
    for (int it = threadIdx.x; it < (C << S0); it += NT) {
      const int c = it % C, b = it / C;
      Ts v[RB];
#pragma unroll
      for (int k = 0; k < RB; ++k) v[k] = tile[((b << S1) + k) * C + c];
      fwht_regs<RB, Ts>(v);
      if (Q == 1) {
#pragma unroll
        for (int k = 0; k < RB; ++k) store_elem<Tout, Ts>(a, g, rho0 + (b << S1) + k, col0 + c, v[k]);
      } else {
#pragma unroll
        for (int k = 0; k < RB; ++k) tile[((b << S1) + k) * C + c] = v[k];
      }
    }
  }
  if (Q > 1) {
    // cluster stage: the top logq bits of the group row index live in different CTAs
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const int MQ = M >> a.logq;
    for (int it = threadIdx.x; it < MQ * C; it += NT) {
      const int c = it % C;
      const int l = rank * MQ + it / C;
      Ts v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q < Q) v[q] = cl.map_shared_rank(tile, q)[l * C + c];
      }
#pragma unroll
      for (int hh = 0; hh < 3; ++hh) {
        const int h = 1 << hh;
        if (h < Q) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (q + h < 8 && (q & h) == 0 && q + h < Q) {
              const Ts x = v[q], y = v[q + h];
              v[q] = x + y;
              v[q + h] = x - y;
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q < Q) store_elem<Tout, Ts>(a, g, (int64_t)q * M + l, col0 + c, v[q]);
      }
    }
    cl.sync();
  }
}

// Small transforms (N' <= 2^9): one CTA per column slab holds all N' rows; the
// butterflies run level by level in shared memory.
template <class Tin, class Ts, class Tout, int C, int NT>
__global__ void __launch_bounds__(NT) k_small(const GroupArgs a, int logn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Ts *tile = reinterpret_cast<Ts *>(smem_raw);
  const int n = 1 << logn;
  const int slab = blockIdx.x;
  const int col0 = slab * C;
  for (int it = threadIdx.x; it < n * C; it += NT) {
    const int c = it % C, rho = it / C;
    tile[rho * C + c] = load_elem<Ts, Tin>(a, 0, rho, col0 + c);
  }
  __syncthreads();
  for (int h = 1; h < n; h <<= 1) {
    for (int it = threadIdx.x; it < (n / 2) * C; it += NT) {
      const int c = it % C, p = it / C;
      const int i = (p / h) * 2 * h + (p % h);
      const Ts x = tile[i * C + c], y = tile[(i + h) * C + c];
      tile[i * C + c] = x + y;
      tile[(i + h) * C + c] = x - y;
    }
    __syncthreads();
  }
  for (int it = threadIdx.x; it < n * C; it += NT) {
    const int c = it % C, kappa = it / C;
    store_elem<Tout, Ts>(a, 0, kappa, col0 + c, tile[kappa * C + c]);
  }
}

template <class Tin, class Ts, class Tout, int LOGM, int C>
cudaError_t launch_group_t(const GroupArgs &a, int64_t ngroups, cudaStream_t s) {
  constexpr int NT = 256;
  const size_t smem = (size_t)(1 << LOGM) * C * sizeof(Ts);
  auto kern = k_group<Tin, Ts, Tout, LOGM, C, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int Q = 1 << a.logq;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ngroups * a.nslab * Q));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class Tin, class Ts, class Tout, int C>
cudaError_t launch_pass_t(const GroupArgs &a0, int L, int64_t ngroups, cudaStream_t s) {
  // L = log2 of the group size; LOGM = min(L, 9) (10 for L = 13), LOGQ = L - LOGM <= 3
  GroupArgs a = a0;
  int logm = L <= 9 ? L : (L >= 13 ? 10 : 9);
  a.logq = L - logm;
  switch (logm) {
    case 5: return launch_group_t<Tin, Ts, Tout, 5, C>(a, ngroups, s);
    case 6: return launch_group_t<Tin, Ts, Tout, 6, C>(a, ngroups, s);
    case 7: return launch_group_t<Tin, Ts, Tout, 7, C>(a, ngroups, s);
    case 8: return launch_group_t<Tin, Ts, Tout, 8, C>(a, ngroups, s);
    case 9: return launch_group_t<Tin, Ts, Tout, 9, C>(a, ngroups, s);
    case 10: return launch_group_t<Tin, Ts, Tout, 10, C>(a, ngroups, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class Tin, class Ts, class Tout, int C>
cudaError_t launch_small_t(const GroupArgs &a, int logn, cudaStream_t s) {
  constexpr int NT = 256;
  const size_t smem = (size_t)(1 << logn) * C * sizeof(Ts);
  auto kern = k_small<Tin, Ts, Tout, C, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<a.nslab, NT, smem, s>>>(a, logn);
  return cudaGetLastError();
}

// Dispatch on (input type, working type, output type).
template <class Tin, class Ts, class Tout, int C>
cudaError_t run_plan(const SrhtPlan &pl, const void *X, int64_t ldx, const void *Y, int64_t N, int d,
                     const int32_t *Psd, const int32_t *pos, void *W, void *WY, int64_t ldw, void *U,
                     void *V, int64_t ldu, double scale, cudaStream_t s,
                     cudaError_t (*pass2)(const GroupArgs &, int, int64_t, cudaStream_t)) {
  GroupArgs a = {};
  a.d = d;
  a.nslab = (d + 1 + C - 1) / C;
  a.N = N;
  a.Psd = Psd;
  a.in = X;
  a.ldin = ldx;
  a.in_y = Y;
  if (pl.single) {
    a.istride = 1; a.igstride = 0;
    a.out = U; a.ldout = ldu; a.out_y = V; a.pos = pos;
    a.ostride = 1; a.ogstride = 0;
    a.scale = scale;
    a.logq = 0;
    return launch_small_t<Tin, Ts, Tout, C>(a, pl.logN, s);
  }
  const int64_t n1 = int64_t(1) << pl.log1, n2 = int64_t(1) << pl.log2;
  // pass 1: groups g = j1 (n1 of them), rows rho = j2 (n2 per group)
  a.istride = 1; a.igstride = n2;
  a.out = W; a.ldout = ldw; a.out_y = WY; a.pos = nullptr;
  a.ostride = 1; a.ogstride = n2;
  a.scale = 1.0;
  cudaError_t e = launch_pass_t<Tin, Ts, Tout, C>(a, pl.log2, n1, s);
  if (e != cudaSuccess) return e;
  // pass 2: groups g = k2 (n2 of them), rows rho = j1 at stride n2, outputs kappa = k1
  GroupArgs b = a;
  b.Psd = nullptr;
  b.N = 0;
  b.in = W; b.ldin = ldw; b.in_y = WY;
  b.istride = n2; b.igstride = 1;
  b.out = U; b.ldout = ldu; b.out_y = V; b.pos = pos;
  b.ostride = n2; b.ogstride = 1;
  b.scale = scale;
  return pass2(b, pl.log1, n2, s);
}

}  // namespace

SrhtPlan srht_plan(int64_t Np) {
  SrhtPlan p{};
  int l = 0;
  while ((int64_t(1) << l) < Np) ++l;
  p.logN = l;
  p.single = l <= 9;
  p.log2 = (l + 1) / 2;  // pass-1 group (inner, contiguous rows)
  p.log1 = l - p.log2;
  return p;
}

cudaError_t launch_srht(const SrhtPlan &pl, int prec, int xdtype, const void *X, int64_t ldx, const void *Y,
                        int64_t N, int d, const int32_t *Psd, const int32_t *pos, void *W, void *WY,
                        int64_t ldw, void *U, void *V, int64_t ldu, double scale, cudaStream_t s) {
  using bf16 = __nv_bfloat16;
  if (prec == SLSE_PREC_FP64) {
    auto p2 = &launch_pass_t<double, double, double, 16>;
    if (xdtype == SLSE_F64)
      return run_plan<double, double, double, 16>(pl, X, ldx, Y, N, d, Psd, pos, W, WY, ldw, U, V, ldu, scale, s, p2);
    return run_plan<float, double, double, 16>(pl, X, ldx, Y, N, d, Psd, pos, W, WY, ldw, U, V, ldu, scale, s, p2);
  }
  if (prec == SLSE_PREC_MIXED_BF16 && xdtype == SLSE_F32) {
    auto p2 = &launch_pass_t<bf16, float, bf16, 32>;
    return run_plan<float, float, bf16, 32>(pl, X, ldx, Y, N, d, Psd, pos, W, WY, ldw, U, V, ldu, scale, s, p2);
  }
  return cudaErrorInvalidValue;
}

}  // namespace slse
