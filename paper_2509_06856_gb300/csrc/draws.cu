// Random draws of the SRHT (paper Sec. 3): Rademacher signs D, the uniform
// permutation P and the sampling order sigma, all from Philox4x32-10 keyed by the
// seed.  A permutation is the stable argsort of one 64-bit Philox key per index;
// ties (probability ~ N'^2 / 2^65) go to the smaller index.
//
// Both permutations are argsorts of 64-bit Philox keys, run together by sort.cuh.
#include "sort.cuh"

namespace slse {
namespace {

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

int log2_exact(int64_t Np) { return sortk::bits_for(Np); }

}  // namespace

// Workspace: per permutation the scattered indices and the bucket arrays; P before sign
// folding.
size_t draws_ws_bytes(int64_t Np) {
  const int B = sortk::bits_for(Np) > 10 ? sortk::bits_for(Np) - 10 : 0;
  return 2 * sortk::align256(sortk::sort_ws_bytes(Np, B)) + sortk::align256(4 * (size_t)Np) + 256;
}

cudaError_t launch_draws(int64_t Np, uint64_t seed, int32_t *Psd, int32_t *P, int32_t *sigma, int8_t *D,
                         void *ws, cudaStream_t s) {
  const int B = sortk::bits_for(Np) > 10 ? sortk::bits_for(Np) - 10 : 0;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  char *p = static_cast<char *>(ws);
  const size_t one = sortk::align256(sortk::sort_ws_bytes(Np, B));
  sortk::SortArrays w{};
  w.key[0] = sortk::RowKey{sortk::KEY_PHILOX, STREAM_P, k0, k1, 0, 0u, 0, 0};
  w.key[1] = sortk::RowKey{sortk::KEY_PHILOX, STREAM_SIGMA, k0, k1, 0, 0u, 0, 0};
  sortk::carve_sort(w, 0, p, Np, B);
  sortk::carve_sort(w, 1, p + one, Np, B);
  int32_t *perm = reinterpret_cast<int32_t *>(p + 2 * one);
  w.out[0] = perm;
  w.out[1] = sigma;
  cudaError_t e = sortk::launch_sort_pair(w, s);
  if (e != cudaSuccess) return e;
  const int T = 256;
  k_fold_signs<<<(unsigned)((Np + T - 1) / T), T, 0, s>>>(Np, k0, k1, perm, Psd, P, D);
  return cudaGetLastError();
}

size_t draws_one_ws_bytes(int64_t Np) {
  const int B = sortk::bits_for(Np) > 10 ? sortk::bits_for(Np) - 10 : 0;
  return sortk::align256(sortk::sort_ws_bytes(Np, B));
}

cudaError_t launch_draws_perm(int64_t Np, uint64_t seed, int32_t *Psd, void *ws, cudaStream_t s) {
  const int B = sortk::bits_for(Np) > 10 ? sortk::bits_for(Np) - 10 : 0;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  char *p = static_cast<char *>(ws);
  sortk::SortArrays w{};
  w.key[0] = sortk::RowKey{sortk::KEY_PHILOX, STREAM_P, k0, k1, 0, 0u, 0, 0};
  sortk::carve_sort(w, 0, p, Np, B);
  int32_t *perm = reinterpret_cast<int32_t *>(p + sortk::align256(sortk::sort_ws_bytes(Np, B)));
  w.out[0] = perm;
  cudaError_t e = sortk::launch_sort_one(w, 0, s);
  if (e != cudaSuccess) return e;
  const int T = 256;
  k_fold_signs<<<(unsigned)((Np + T - 1) / T), T, 0, s>>>(Np, k0, k1, perm, Psd, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_draws_sigma(int64_t Np, uint64_t seed, int32_t *sigma, void *ws, cudaStream_t s) {
  const int B = sortk::bits_for(Np) > 10 ? sortk::bits_for(Np) - 10 : 0;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  sortk::SortArrays w{};
  w.key[0] = sortk::RowKey{sortk::KEY_PHILOX, STREAM_SIGMA, k0, k1, 0, 0u, 0, 0};
  sortk::carve_sort(w, 0, ws, Np, B);
  w.out[0] = sigma;
  return sortk::launch_sort_one(w, 0, s);
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
