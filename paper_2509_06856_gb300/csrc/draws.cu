// Random draws of the SRHT (paper Sec. 3): Rademacher signs D, the uniform
// permutation P and the sampling order sigma, all from Philox4x32-10 keyed by the
// seed.  A permutation is the stable argsort of one 64-bit Philox key per index;
// ties (probability ~ N'^2 / 2^65) go to the smaller index.
//
// GPU argsort of uniform keys, both permutations (P and sigma) in the same launches
// (blockIdx.y = which one): bucket by the top B = max(0, log2 N' - 10) key bits
// (counting sort: histogram, scan, scatter of the indices), then order each bucket
// (about 1024 entries) in shared memory by a second counting sort on the next 8 key
// bits followed by an insertion sort of each sub-bucket (about 4 entries) on the full
// (key, index) pair.  Keys are recomputed from the index (Philox is cheaper than a
// round trip through HBM).  A bucket larger than the shared-memory capacity is ordered
// by exact ranks instead, so the result is the unique (key, index) order for every input.
#include "slse_internal.cuh"

namespace slse {
namespace {

constexpr int kSortCap = 2048;  // entries per bucket ordered in shared memory
constexpr int kSortThreads = 256;
constexpr int kSubBits = 8;
constexpr int kSub = 1 << kSubBits;

__host__ __device__ inline int bucket_bits(int logNp) { return logNp > 10 ? logNp - 10 : 0; }

__device__ __forceinline__ unsigned long long sort_key(int64_t i, int stream, uint32_t k0, uint32_t k1) {
  const U4 r = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)stream, 0u, k0, k1);
  return ((unsigned long long)r.y << 32) | r.x;
}

// Per-sort arrays: the two sorts (y = 0: P, y = 1: sigma) use separate copies.
struct SortArrays {
  uint32_t *tidx[2];
  unsigned *counts[2], *offsets[2], *cursor[2];
  int32_t *out[2];
};

__device__ __forceinline__ int sort_stream_id(int y) { return y == 0 ? STREAM_P : STREAM_SIGMA; }
// Select one of the two per-sort pointers without indexing the kernel parameter at run time.
template <class T> __device__ __forceinline__ T pick(T const (&a)[2], int y) { return y ? a[1] : a[0]; }

__global__ void k_keys_hist(int64_t Np, uint32_t k0, uint32_t k1, int B, SortArrays w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const int y = blockIdx.y;
  const unsigned long long key = sort_key(i, sort_stream_id(y), k0, k1);
  const unsigned b = B > 0 ? (unsigned)(key >> (64 - B)) : 0u;
  atomicAdd(&pick(w.counts, y)[b], 1u);
}

// Exclusive scan of nb counts by one CTA per sort; writes offsets and cursor (= offsets).
__global__ void k_scan(int nb, SortArrays w) {
  __shared__ unsigned s_part[1024];
  __shared__ unsigned s_carry;
  const int y = blockIdx.x;
  const unsigned *counts = pick(w.counts, y);
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const unsigned v = i < nb ? counts[i] : 0u;
    s_part[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const unsigned t = threadIdx.x >= off ? s_part[threadIdx.x - off] : 0u;
      __syncthreads();
      s_part[threadIdx.x] += t;
      __syncthreads();
    }
    const unsigned incl = s_part[threadIdx.x] + s_carry;
    if (i < nb) { pick(w.offsets, y)[i] = incl - v; pick(w.cursor, y)[i] = incl - v; }
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
    __syncthreads();
  }
}

__global__ void k_scatter(int64_t Np, uint32_t k0, uint32_t k1, int B, SortArrays w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const int y = blockIdx.y;
  const unsigned long long key = sort_key(i, sort_stream_id(y), k0, k1);
  const unsigned b = B > 0 ? (unsigned)(key >> (64 - B)) : 0u;
  const unsigned slot = atomicAdd(&pick(w.cursor, y)[b], 1u);
  pick(w.tidx, y)[slot] = (uint32_t)i;
}

__device__ __forceinline__ bool pair_gt(unsigned long long ka, uint32_t ia, unsigned long long kb, uint32_t ib) {
  return ka > kb || (ka == kb && ia > ib);
}

// One CTA per bucket (blockIdx.x) and sort (blockIdx.y); writes the ordered indices to
// out[offset .. offset + count).
__global__ void __launch_bounds__(kSortThreads) k_bucket_sort(uint32_t k0, uint32_t k1, int B, SortArrays w) {
  static_assert(kSub == kSortThreads, "one sub-bucket per thread");
  __shared__ unsigned long long s_k1[kSortCap];
  __shared__ uint32_t s_i0[kSortCap], s_i1[kSortCap];
  __shared__ unsigned s_cnt[kSub], s_start[kSub], s_cur[kSub];
  const int y = blockIdx.y;
  const int stream = sort_stream_id(y);
  const unsigned cnt = pick(w.counts, y)[blockIdx.x];
  const unsigned off = pick(w.offsets, y)[blockIdx.x];
  const uint32_t *tidx = pick(w.tidx, y);
  int32_t *out = pick(w.out, y);
  if (cnt == 0) return;
  if (cnt > (unsigned)kSortCap) {
    // exact rank of each entry among the bucket's distinct (key, index) pairs
    for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) {
      const uint32_t it = tidx[off + t];
      const unsigned long long kt = sort_key(it, stream, k0, k1);
      unsigned rank = 0;
      for (unsigned u = 0; u < cnt; ++u) {
        const uint32_t iu = tidx[off + u];
        rank += pair_gt(kt, it, sort_key(iu, stream, k0, k1), iu) ? 1u : 0u;
      }
      out[off + rank] = (int32_t)it;
    }
    return;
  }
  const int shift = 64 - B - kSubBits;
  for (int s = threadIdx.x; s < kSub; s += blockDim.x) s_cnt[s] = 0;
  __syncthreads();
  for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) {
    const uint32_t i = tidx[off + t];
    const unsigned long long key = sort_key(i, stream, k0, k1);
    s_i0[t] = i;
    atomicAdd(&s_cnt[(unsigned)(key >> shift) & (kSub - 1)], 1u);
  }
  __syncthreads();
  // exclusive scan of the sub-bucket counts (kSub = kSortThreads entries, one per thread)
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned v = s_cnt[threadIdx.x];
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    __shared__ unsigned s_wsum[kSortThreads / 32];
    if (lane == 31) s_wsum[wid] = incl;
    __syncthreads();
    unsigned base = 0;
    for (int k = 0; k < wid; ++k) base += s_wsum[k];
    s_start[threadIdx.x] = base + incl - v;
    s_cur[threadIdx.x] = base + incl - v;
  }
  __syncthreads();
  for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) {
    const uint32_t i = s_i0[t];
    const unsigned long long key = sort_key(i, stream, k0, k1);
    const unsigned slot = atomicAdd(&s_cur[(unsigned)(key >> shift) & (kSub - 1)], 1u);
    s_k1[slot] = key;
    s_i1[slot] = i;
  }
  __syncthreads();
  // insertion sort of sub-bucket s by one thread
  {
    const unsigned lo = s_start[threadIdx.x], n = s_cnt[threadIdx.x];
    for (unsigned a = 1; a < n; ++a) {
      const unsigned long long ka = s_k1[lo + a];
      const uint32_t ia = s_i1[lo + a];
      unsigned b = a;
      while (b > 0 && pair_gt(s_k1[lo + b - 1], s_i1[lo + b - 1], ka, ia)) {
        s_k1[lo + b] = s_k1[lo + b - 1];
        s_i1[lo + b] = s_i1[lo + b - 1];
        --b;
      }
      s_k1[lo + b] = ka;
      s_i1[lo + b] = ia;
    }
  }
  __syncthreads();
  for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) out[off + t] = (int32_t)s_i1[t];
}

// Sign-folded permutation: Psd[j] = P[j] if D_j = +1, ~P[j] if D_j = -1.
__global__ void k_fold_signs(int64_t Np, uint32_t k0, uint32_t k1, const int32_t *perm, int32_t *Psd,
                             int32_t *P_out, int8_t *D_out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Np) return;
  const U4 r = philox4x32_10((uint32_t)j, (uint32_t)(j >> 32), (uint32_t)STREAM_D, 0u, k0, k1);
  const bool neg = (r.x & 1u) != 0u;
  const int32_t p = perm[j];
  if (Psd) Psd[j] = neg ? ~p : p;
  if (P_out) P_out[j] = p;
  if (D_out) D_out[j] = neg ? (int8_t)-1 : (int8_t)1;
}

// pos is stored "pass-2-major": output row k = k1 n2 + k2 lives at index k2 n1 + k1, so
// the rows one pass-2 group writes are contiguous.  log2 = log2 n2 (= log2 N' for one pass).
__global__ void k_pos_scatter(const int32_t *sigma, int64_t s0, int64_t s1, int log1, int log2, int32_t *pos) {
  const int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= s1) return;
  const int64_t k = sigma[s];
  const int64_t idx = ((k & ((int64_t(1) << log2) - 1)) << log1) | (k >> log2);
  pos[idx] = (int32_t)s;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int log2_exact(int64_t Np) {
  int l = 0;
  while ((int64_t(1) << l) < Np) ++l;
  return l;
}

// Workspace: per sort the scattered indices (N') and three bucket arrays; the
// permutation P before sign folding (N').
SortArrays carve(void *ws, int64_t Np, int nb, int32_t *sigma_out) {
  char *p = static_cast<char *>(ws);
  SortArrays w;
  size_t off = 0;
  for (int y = 0; y < 2; ++y) {
    w.tidx[y] = reinterpret_cast<uint32_t *>(p + off); off = align256(off + 4 * (size_t)Np);
    w.counts[y] = reinterpret_cast<unsigned *>(p + off); off = align256(off + 4 * (size_t)nb);
    w.offsets[y] = reinterpret_cast<unsigned *>(p + off); off = align256(off + 4 * (size_t)nb);
    w.cursor[y] = reinterpret_cast<unsigned *>(p + off); off = align256(off + 4 * (size_t)nb);
  }
  w.out[0] = reinterpret_cast<int32_t *>(p + off);
  w.out[1] = sigma_out;
  return w;
}

}  // namespace

size_t draws_ws_bytes(int64_t Np) {
  const int nb = 1 << bucket_bits(log2_exact(Np));
  return 2 * (align256(4 * (size_t)Np) + 3 * align256(4 * (size_t)nb)) + align256(4 * (size_t)Np) + 256;
}

cudaError_t launch_draws(int64_t Np, uint64_t seed, int32_t *Psd, int32_t *P, int32_t *sigma, int8_t *D,
                         void *ws, cudaStream_t s) {
  const int logNp = log2_exact(Np);
  const int B = bucket_bits(logNp);
  const int nb = 1 << B;
  SortArrays w = carve(ws, Np, nb, sigma);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int T = 256;
  const unsigned grid = (unsigned)((Np + T - 1) / T);
  cudaError_t e;
  for (int y = 0; y < 2; ++y)
    if ((e = cudaMemsetAsync(w.counts[y], 0, 4 * (size_t)nb, s)) != cudaSuccess) return e;
  k_keys_hist<<<dim3(grid, 2), T, 0, s>>>(Np, k0, k1, B, w);
  k_scan<<<2, 1024, 0, s>>>(nb, w);
  k_scatter<<<dim3(grid, 2), T, 0, s>>>(Np, k0, k1, B, w);
  k_bucket_sort<<<dim3(nb, 2), kSortThreads, 0, s>>>(k0, k1, B, w);
  k_fold_signs<<<grid, T, 0, s>>>(Np, k0, k1, w.out[0], Psd, P, D);
  return cudaGetLastError();
}

cudaError_t launch_pos_map(const int32_t *sigma, int64_t Np, int64_t s0, int64_t s1, int log2, int32_t *pos,
                           cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pos, 0xFF, 4 * (size_t)Np, s);
  if (e != cudaSuccess || s1 <= s0) return e;
  const int T = 256;
  const int log1 = log2_exact(Np) - log2;
  k_pos_scatter<<<(unsigned)((s1 - s0 + T - 1) / T), T, 0, s>>>(sigma, s0, s1, log1, log2, pos);
  return cudaGetLastError();
}

}  // namespace slse
