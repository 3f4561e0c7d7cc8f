// Random draws of the SRHT (paper Sec. 3): Rademacher signs D, the uniform
// permutation P and the sampling order sigma, all from Philox4x32-10 keyed by the
// seed.  A permutation is the stable argsort of one 64-bit Philox key per index;
// ties (probability ~ N'^2 / 2^65) go to the smaller index.
//
// GPU argsort of uniform keys: bucket by the top B = max(0, log2 N' - 10) key bits
// (counting sort: histogram, scan, scatter), then sort each bucket (about 1024
// entries) on (key, index) in shared memory with a bitonic network.  A bucket
// larger than the shared-memory capacity is sorted by exact ranks instead, so the
// result is the unique (key, index) order for every input.
#include "slse_internal.cuh"

namespace slse {
namespace {

constexpr int kSortCap = 4096;  // entries per bucket sorted in shared memory (48 KB)
constexpr int kSortThreads = 512;

__host__ __device__ inline int bucket_bits(int logNp) { return logNp > 10 ? logNp - 10 : 0; }

__global__ void k_keys_hist(int64_t Np, uint32_t k0, uint32_t k1, int stream, int B,
                            unsigned long long *keys, unsigned *counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const U4 r = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)stream, 0u, k0, k1);
  const unsigned long long key = ((unsigned long long)r.y << 32) | r.x;
  keys[i] = key;
  const unsigned b = B > 0 ? (unsigned)(key >> (64 - B)) : 0u;
  atomicAdd(&counts[b], 1u);
}

// Exclusive scan of nb counts by one CTA; writes offsets and cursor (= offsets).
__global__ void k_scan(const unsigned *counts, int nb, unsigned *offsets, unsigned *cursor) {
  __shared__ unsigned s_part[1024];
  __shared__ unsigned s_carry;
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

__global__ void k_scatter(int64_t Np, int B, const unsigned long long *keys, unsigned *cursor,
                          unsigned long long *tkeys, uint32_t *tidx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const unsigned long long key = keys[i];
  const unsigned b = B > 0 ? (unsigned)(key >> (64 - B)) : 0u;
  const unsigned slot = atomicAdd(&cursor[b], 1u);
  tkeys[slot] = key;
  tidx[slot] = (uint32_t)i;
}

__device__ __forceinline__ bool pair_gt(unsigned long long ka, uint32_t ia, unsigned long long kb, uint32_t ib) {
  return ka > kb || (ka == kb && ia > ib);
}

// One CTA per bucket; writes the sorted indices to out[offset .. offset + count).
__global__ void __launch_bounds__(kSortThreads) k_bucket_sort(const unsigned *counts, const unsigned *offsets,
                                                              const unsigned long long *tkeys,
                                                              const uint32_t *tidx, int32_t *out) {
  extern __shared__ unsigned char smem_raw[];
  unsigned long long *sk = reinterpret_cast<unsigned long long *>(smem_raw);
  uint32_t *si = reinterpret_cast<uint32_t *>(sk + kSortCap);
  const unsigned cnt = counts[blockIdx.x];
  const unsigned off = offsets[blockIdx.x];
  if (cnt == 0) return;
  if (cnt <= (unsigned)kSortCap) {
    unsigned n = 1;
    while (n < cnt) n <<= 1;
    for (unsigned t = threadIdx.x; t < n; t += blockDim.x) {
      if (t < cnt) { sk[t] = tkeys[off + t]; si[t] = tidx[off + t]; }
      else { sk[t] = ~0ull; si[t] = 0xFFFFFFFFu; }
    }
    __syncthreads();
    for (unsigned k = 2; k <= n; k <<= 1) {
      for (unsigned j = k >> 1; j > 0; j >>= 1) {
        for (unsigned t = threadIdx.x; t < n; t += blockDim.x) {
          const unsigned l = t ^ j;
          if (l > t) {
            const bool up = (t & k) == 0;
            const bool gt = pair_gt(sk[t], si[t], sk[l], si[l]);
            if (gt == up) {
              const unsigned long long tk = sk[t]; sk[t] = sk[l]; sk[l] = tk;
              const uint32_t ti = si[t]; si[t] = si[l]; si[l] = ti;
            }
          }
        }
        __syncthreads();
      }
    }
    for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) out[off + t] = (int32_t)si[t];
  } else {
    // exact rank of each entry among the bucket's distinct (key, index) pairs
    for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) {
      const unsigned long long kt = tkeys[off + t];
      const uint32_t it = tidx[off + t];
      unsigned rank = 0;
      for (unsigned u = 0; u < cnt; ++u) rank += pair_gt(kt, it, tkeys[off + u], tidx[off + u]) ? 1u : 0u;
      out[off + rank] = (int32_t)it;
    }
  }
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

struct DrawsWs {
  unsigned long long *keys, *tkeys;
  uint32_t *tidx;
  unsigned *counts, *offsets, *cursor;
  int32_t *perm;
};

DrawsWs carve(void *ws, int64_t Np, int nb) {
  char *p = static_cast<char *>(ws);
  DrawsWs w;
  size_t off = 0;
  w.keys = reinterpret_cast<unsigned long long *>(p + off); off = align256(off + 8 * (size_t)Np);
  w.tkeys = reinterpret_cast<unsigned long long *>(p + off); off = align256(off + 8 * (size_t)Np);
  w.tidx = reinterpret_cast<uint32_t *>(p + off); off = align256(off + 4 * (size_t)Np);
  w.perm = reinterpret_cast<int32_t *>(p + off); off = align256(off + 4 * (size_t)Np);
  w.counts = reinterpret_cast<unsigned *>(p + off); off = align256(off + 4 * (size_t)nb);
  w.offsets = reinterpret_cast<unsigned *>(p + off); off = align256(off + 4 * (size_t)nb);
  w.cursor = reinterpret_cast<unsigned *>(p + off); off = align256(off + 4 * (size_t)nb);
  return w;
}

int log2_exact(int64_t Np) {
  int l = 0;
  while ((int64_t(1) << l) < Np) ++l;
  return l;
}

cudaError_t sort_stream(int64_t Np, uint64_t seed, int stream, const DrawsWs &w, int32_t *out, cudaStream_t s) {
  const int logNp = log2_exact(Np);
  const int B = bucket_bits(logNp);
  const int nb = 1 << B;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int T = 256;
  const unsigned grid = (unsigned)((Np + T - 1) / T);
  cudaError_t e = cudaMemsetAsync(w.counts, 0, 4 * (size_t)nb, s);
  if (e != cudaSuccess) return e;
  k_keys_hist<<<grid, T, 0, s>>>(Np, k0, k1, stream, B, w.keys, w.counts);
  k_scan<<<1, 1024, 0, s>>>(w.counts, nb, w.offsets, w.cursor);
  k_scatter<<<grid, T, 0, s>>>(Np, B, w.keys, w.cursor, w.tkeys, w.tidx);
  const size_t smem = (size_t)kSortCap * (sizeof(unsigned long long) + sizeof(uint32_t));
  k_bucket_sort<<<nb, kSortThreads, smem, s>>>(w.counts, w.offsets, w.tkeys, w.tidx, out);
  return cudaGetLastError();
}

}  // namespace

size_t draws_ws_bytes(int64_t Np) {
  const int nb = 1 << bucket_bits(log2_exact(Np));
  return align256(8 * (size_t)Np) * 2 + align256(4 * (size_t)Np) * 2 + 3 * align256(4 * (size_t)nb) + 256;
}

cudaError_t launch_draws(int64_t Np, uint64_t seed, int32_t *Psd, int32_t *P, int32_t *sigma, int8_t *D,
                         void *ws, cudaStream_t s) {
  const int nb = 1 << bucket_bits(log2_exact(Np));
  DrawsWs w = carve(ws, Np, nb);
  cudaError_t e = sort_stream(Np, seed, STREAM_P, w, w.perm, s);
  if (e != cudaSuccess) return e;
  const int T = 256;
  const unsigned grid = (unsigned)((Np + T - 1) / T);
  k_fold_signs<<<grid, T, 0, s>>>(Np, (uint32_t)seed, (uint32_t)(seed >> 32), w.perm, Psd, P, D);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sort_stream(Np, seed, STREAM_SIGMA, w, sigma, s);
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
