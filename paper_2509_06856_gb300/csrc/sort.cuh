// Argsort of row indices by a 64-bit key computed from the index, two sorts per launch
// (blockIdx.y selects the sort).  Used for the SRHT permutations (Philox keys) and for
// the CountSketch bucket lists (keys built from the row's hash and its index).
//
// Method: bucket by the top B key bits (counting sort: histogram, scan, scatter of the
// indices), then order each bucket (about 1024 entries when B is chosen for that) in
// shared memory by a second counting sort on the next 8 key bits followed by an
// insertion sort of each sub-bucket on the full (key, index) pair.  Keys are recomputed
// from the index rather than stored.  A bucket larger than the shared-memory capacity is
// ordered by exact ranks instead, so the result is the unique (key, index) order for
// every input.
#pragma once
#include "slse_internal.cuh"

namespace slse {
namespace sortk {

constexpr int kSortCap = 2048;  // entries per bucket ordered in shared memory
constexpr int kSortThreads = 256;
constexpr int kSubBits = 8;
constexpr int kSub = 1 << kSubBits;

enum KeyKind { KEY_PHILOX = 0, KEY_CS_NESTED = 1, KEY_CS_HAT = 2 };

// How a row index i becomes its sort key.
//   KEY_PHILOX:    (w1 << 32) | w0 of Philox(counter (i, stream), key (k0, k1)).
//   KEY_CS_NESTED: CountSketch hash h = w0 of Philox stream `stream`; the key holds the
//                  bit-reversed low L bits of h on top and the index below, so rows are
//                  ordered by bucket of every nested size 2^l <= 2^L at once (a bucket of
//                  size 2^l is a run of keys), and by index inside a bucket.
//   KEY_CS_HAT:    bucket floor(w0 r / 2^32) on top, the index below.
struct RowKey {
  int kind;
  int stream;
  uint32_t k0, k1;
  int L;        // KEY_CS_NESTED: bits of the hash kept
  uint32_t r;   // KEY_CS_HAT: number of buckets
  int rb;       // KEY_CS_HAT: bits of r - 1
  int ib;       // bits of the largest index (N - 1)
};

__device__ __forceinline__ uint32_t bitrev_low(uint32_t x, int L) {
  return L > 0 ? (__brev(x) >> (32 - L)) : 0u;
}

__device__ __forceinline__ unsigned long long row_key(const RowKey &k, int64_t i) {
  const U4 w = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)k.stream, 0u, k.k0, k.k1);
  if (k.kind == KEY_PHILOX) return ((unsigned long long)w.y << 32) | w.x;
  const unsigned long long ii = (unsigned long long)i;
  if (k.kind == KEY_CS_NESTED) {
    const unsigned long long top = (unsigned long long)bitrev_low(w.x, k.L);
    return (k.L > 0 ? top << (64 - k.L) : 0ull) | (k.ib > 0 ? ii << (64 - k.L - k.ib) : 0ull);
  }
  const unsigned long long hb = ((unsigned long long)w.x * k.r) >> 32;
  return (k.rb > 0 ? hb << (64 - k.rb) : 0ull) | (k.ib > 0 ? ii << (64 - k.rb - k.ib) : 0ull);
}

// Per-sort arrays (y = 0, 1).
struct SortArrays {
  RowKey key[2];
  int B[2];        // bucket bits of each sort
  int64_t n[2];    // rows of each sort
  uint32_t *tidx[2];
  unsigned *counts[2], *offsets[2], *cursor[2];
  int32_t *out[2];
};

// Select one of the two per-sort entries without indexing the kernel parameter at run time.
template <class T> __device__ __forceinline__ const T &pick(T const (&a)[2], int y) { return y ? a[1] : a[0]; }

// Kernels have internal linkage: every translation unit that includes this header gets
// its own copy.
namespace {

__device__ __forceinline__ unsigned bucket_of(unsigned long long key, int B) {
  return B > 0 ? (unsigned)(key >> (64 - B)) : 0u;
}

__global__ void k_keys_hist(SortArrays w) {
  const int y = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pick(w.n, y)) return;
  const unsigned long long key = row_key(pick(w.key, y), i);
  atomicAdd(&pick(w.counts, y)[bucket_of(key, pick(w.B, y))], 1u);
}

// Exclusive scan of the 2^B counts by one CTA per sort; writes offsets and cursor.
__global__ void k_scan(SortArrays w) {
  __shared__ unsigned s_part[1024];
  __shared__ unsigned s_carry;
  const int y = blockIdx.x;
  const int nb = 1 << pick(w.B, y);
  const unsigned *counts = pick(w.counts, y);
  unsigned *offsets = pick(w.offsets, y), *cursor = pick(w.cursor, y);
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
    if (i < nb) { offsets[i] = incl - v; cursor[i] = incl - v; }
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
    __syncthreads();
  }
}

__global__ void k_scatter(SortArrays w) {
  const int y = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pick(w.n, y)) return;
  const unsigned long long key = row_key(pick(w.key, y), i);
  const unsigned slot = atomicAdd(&pick(w.cursor, y)[bucket_of(key, pick(w.B, y))], 1u);
  pick(w.tidx, y)[slot] = (uint32_t)i;
}

__device__ __forceinline__ bool pair_gt(unsigned long long ka, uint32_t ia, unsigned long long kb, uint32_t ib) {
  return ka > kb || (ka == kb && ia > ib);
}

// One CTA per bucket (blockIdx.x) and sort (blockIdx.y); writes the ordered indices to
// out[offset .. offset + count).
__global__ void __launch_bounds__(kSortThreads) k_bucket_sort(SortArrays w) {
  static_assert(kSub == kSortThreads, "one sub-bucket per thread");
  __shared__ unsigned long long s_k1[kSortCap];
  __shared__ uint32_t s_i0[kSortCap], s_i1[kSortCap];
  __shared__ unsigned s_cnt[kSub], s_start[kSub], s_cur[kSub];
  __shared__ unsigned s_wsum[kSortThreads / 32];
  const int y = blockIdx.y;
  const int B = pick(w.B, y);
  if (blockIdx.x >= (1u << B)) return;
  const RowKey key = pick(w.key, y);
  const unsigned cnt = pick(w.counts, y)[blockIdx.x];
  const unsigned off = pick(w.offsets, y)[blockIdx.x];
  const uint32_t *tidx = pick(w.tidx, y);
  int32_t *out = pick(w.out, y);
  if (cnt == 0) return;
  if (cnt > (unsigned)kSortCap) {
    // exact rank of each entry among the bucket's distinct (key, index) pairs
    for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) {
      const uint32_t it = tidx[off + t];
      const unsigned long long kt = row_key(key, it);
      unsigned rank = 0;
      for (unsigned u = 0; u < cnt; ++u) {
        const uint32_t iu = tidx[off + u];
        rank += pair_gt(kt, it, row_key(key, iu), iu) ? 1u : 0u;
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
    s_i0[t] = i;
    atomicAdd(&s_cnt[(unsigned)(row_key(key, i) >> shift) & (kSub - 1)], 1u);
  }
  __syncthreads();
  // exclusive scan of the sub-bucket counts (one per thread)
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned v = s_cnt[threadIdx.x];
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
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
    const unsigned long long k = row_key(key, i);
    const unsigned slot = atomicAdd(&s_cur[(unsigned)(k >> shift) & (kSub - 1)], 1u);
    s_k1[slot] = k;
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

}  // namespace

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

inline int bits_for(int64_t n) {  // number of bits of n - 1 (0 for n <= 1)
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

// Workspace of one sort of n rows with 2^B buckets.
inline size_t sort_ws_bytes(int64_t n, int B) {
  return align256(4 * (size_t)n) + 3 * align256(4 * ((size_t)1 << B));
}

inline void carve_sort(SortArrays &w, int y, void *ws, int64_t n, int B) {
  char *p = static_cast<char *>(ws);
  size_t off = 0;
  w.n[y] = n;
  w.B[y] = B;
  w.tidx[y] = reinterpret_cast<uint32_t *>(p + off); off += align256(4 * (size_t)n);
  w.counts[y] = reinterpret_cast<unsigned *>(p + off); off += align256(4 * ((size_t)1 << B));
  w.offsets[y] = reinterpret_cast<unsigned *>(p + off); off += align256(4 * ((size_t)1 << B));
  w.cursor[y] = reinterpret_cast<unsigned *>(p + off);
}

// Runs both sorts of `w` (keys, sizes, bucket bits, arrays and outputs filled in).
inline cudaError_t launch_sort_pair(const SortArrays &w, cudaStream_t s) {
  cudaError_t e;
  for (int y = 0; y < 2; ++y)
    if ((e = cudaMemsetAsync(w.counts[y], 0, 4 * ((size_t)1 << w.B[y]), s)) != cudaSuccess) return e;
  const int T = 256;
  const int64_t nmax = w.n[0] > w.n[1] ? w.n[0] : w.n[1];
  const unsigned grid = (unsigned)((nmax + T - 1) / T);
  const int Bmax = w.B[0] > w.B[1] ? w.B[0] : w.B[1];
  if (grid > 0) k_keys_hist<<<dim3(grid, 2), T, 0, s>>>(w);
  k_scan<<<2, 1024, 0, s>>>(w);
  if (grid > 0) k_scatter<<<dim3(grid, 2), T, 0, s>>>(w);
  k_bucket_sort<<<dim3(1u << Bmax, 2), kSortThreads, 0, s>>>(w);
  return cudaGetLastError();
}

// Runs sort y of `w` alone (its entry copied to slot 0; the other sort is not touched).
inline cudaError_t launch_sort_one(const SortArrays &w, int y, cudaStream_t s) {
  SortArrays v = w;
  v.key[0] = w.key[y]; v.B[0] = w.B[y]; v.n[0] = w.n[y]; v.tidx[0] = w.tidx[y];
  v.counts[0] = w.counts[y]; v.offsets[0] = w.offsets[y]; v.cursor[0] = w.cursor[y]; v.out[0] = w.out[y];
  v.key[1] = v.key[0]; v.B[1] = v.B[0]; v.n[1] = v.n[0]; v.tidx[1] = v.tidx[0];
  v.counts[1] = v.counts[0]; v.offsets[1] = v.offsets[0]; v.cursor[1] = v.cursor[0]; v.out[1] = v.out[0];
  cudaError_t e;
  if ((e = cudaMemsetAsync(v.counts[0], 0, 4 * ((size_t)1 << v.B[0]), s)) != cudaSuccess) return e;
  const int T = 256;
  const unsigned grid = (unsigned)((v.n[0] + T - 1) / T);
  if (grid > 0) k_keys_hist<<<dim3(grid, 1), T, 0, s>>>(v);
  k_scan<<<1, 1024, 0, s>>>(v);
  if (grid > 0) k_scatter<<<dim3(grid, 1), T, 0, s>>>(v);
  k_bucket_sort<<<dim3(1u << v.B[0], 1), kSortThreads, 0, s>>>(v);
  return cudaGetLastError();
}

}  // namespace sortk
}  // namespace slse
