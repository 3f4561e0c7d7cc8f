// Gaussian sketch (Sec. 2: S in R^{m x N} with i.i.d. N(0, 1/m) entries), used as the
// Hessian sketch S-hat X = G X / sqrt(m).  Forming it is a dense (m x N)(N x d) product, so
// the mixed-precision path runs it on the tensor cores.
//
// Entries: G[i, k] from Philox4x32-10 at counter (q mod 2^32, q div 2^32, 5, i), q = k div 8,
// key = seed; output word j feeds Box-Muller with u1 = (w mod 2^16 + 1/2) 2^-16 and
// u2 = (w div 2^16 + 1/2) 2^-16: G[i, 8q + 2j] = sqrt(-2 ln u1) cos(2 pi u2),
// G[i, 8q + 2j + 1] = sqrt(-2 ln u1) sin(2 pi u2).
//
// MIXED_BF16 (X F32): X is packed once into BF16 chunks of 32 rows laid out as the K-major
// operand of tcgen05.mma (8 x 16-byte core matrices); k_gauss_tc gives each CTA 128 rows of
// G and a range of chunks, in a pipeline of up to 8 stages.  Sixteen producer warps draw the
// G tile in FP32 (hardware log2, sin, cos, rsqrt; the Philox words of the next chunk are drawn
// beside the Box-Muller step of the current one), round it to BF16 and store it in the same
// layout; one thread copies the X chunk with cp.async.bulk; one thread issues the
// 128 x ncp x 32 MMAs into an FP32 accumulator in tensor memory; four warps read it back
// (tcgen05.ld) into per-split partial sums, which k_gauss_reduce adds in a fixed order.
// FP64: the same entries in double precision (log, sincospi) and an FP64 CUDA-core product.
#include "tc_common.cuh"

namespace slse {
namespace {

constexpr int kStreamG = 5;

// ------------------------------------------------------------------ normals
// single-instruction approximations (the operands here are normal numbers: ftz changes nothing)
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void box_muller_f64(uint32_t w, double &a, double &b) {
  const double u1 = ((double)(w & 0xFFFFu) + 0.5) * 0x1p-16;
  const double u2 = ((double)(w >> 16) + 0.5) * 0x1p-16;
  const double rad = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  a = rad * cs;
  b = rad * sn;
}

// Philox4x32-10 with the round keys precomputed (they are the same for every call of a
// thread): per round two 32x32->64-bit products and two three-input XORs.
struct RoundKeys {
  uint32_t k0[10], k1[10];
};
__device__ __forceinline__ RoundKeys round_keys(uint32_t k0, uint32_t k1) {
  RoundKeys r;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    r.k0[i] = k0 + (uint32_t)i * 0x9E3779B9u;
    r.k1[i] = k1 + (uint32_t)i * 0xBB67AE85u;
  }
  return r;
}
__device__ __forceinline__ U4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const RoundKeys &K) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[i], n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[i];
    c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
  }
  return U4{c0, c1, c2, c3};
}

// Box-Muller pairs of two words at once, rounded to BF16 (word -> (cos entry, sin entry)),
// with the FP32 additions and multiplications in the packed two-lane instructions:
//   u = (h + 1/2) 2^-16 exactly, as the float 1 + h 2^-16 minus (1 - 2^-17) (both in [1/2, 2]);
//   t = -2 ln u1 >= -2 ln(1 - 2^-17) = 1.5e-5, far above the 2^-22 absolute error of lg2 near 1,
//     so t > 0 and the reciprocal square root is finite;
//   theta = 2 pi u2 - pi lies in (-pi, pi), where the hardware sine and cosine are accurate, and
//     cos(2 pi u2) = -cos(theta), sin(2 pi u2) = -sin(theta): the radius is carried negated.
__device__ __forceinline__ uint2 box_muller_bf16x2_pair(uint32_t wa, uint32_t wb) {
  const float2 one_m = make_float2(-0.99999237060546875f, -0.99999237060546875f);
  const float2 u1 = __fadd2_rn(make_float2(__uint_as_float(((wa << 7) & 0x007FFF80u) | 0x3F800000u),
                                           __uint_as_float(((wb << 7) & 0x007FFF80u) | 0x3F800000u)),
                               one_m);
  const float2 u2 = __fadd2_rn(make_float2(__uint_as_float(((wa >> 9) & 0x007FFF80u) | 0x3F800000u),
                                           __uint_as_float(((wb >> 9) & 0x007FFF80u) | 0x3F800000u)),
                               one_m);
  const float2 t = __fmul2_rn(make_float2(-1.3862943611198906f, -1.3862943611198906f),
                              make_float2(lg2_approx(u1.x), lg2_approx(u1.y)));
  const float2 nrad = __fmul2_rn(make_float2(-t.x, -t.y), make_float2(rsqrt_approx(t.x), rsqrt_approx(t.y)));
  const float2 th = __ffma2_rn(u2, make_float2(6.2831853071795865f, 6.2831853071795865f),
                               make_float2(-3.1415926535897932f, -3.1415926535897932f));
  const float2 ca = __fmul2_rn(nrad, make_float2(cos_approx(th.x), cos_approx(th.y)));
  const float2 sa = __fmul2_rn(nrad, make_float2(sin_approx(th.x), sin_approx(th.y)));
  const __nv_bfloat162 ha = __floats2bfloat162_rn(ca.x, sa.x), hb = __floats2bfloat162_rn(ca.y, sa.y);
  return make_uint2(*reinterpret_cast<const uint32_t *>(&ha), *reinterpret_cast<const uint32_t *>(&hb));
}

// ------------------------------------------------------------------ tensor-core path
// A chunk is 32 rows of X (two MMAs of K = 16).  Operands sit in shared memory as K-major
// core matrices (8 rows x 16 bytes): element (row, k) of a tile at byte
// (row div 8) 512 + (k div 8) 128 + (row mod 8) 16 + (k mod 8) 2, so the descriptors use a
// leading byte offset of 128 (next core matrix along K) and a stride byte offset of 512
// (next group of 8 rows).
constexpr int kBM = 128;               // rows of G per CTA (MMA M)
constexpr int kBK = 32;                // rows of X per chunk
constexpr int kSBO = kBK * 16;         // bytes between 8-row groups of a tile
constexpr int kTileA = kBM * kBK * 2;  // 8 KiB
constexpr int kProdWarps = 16;         // 512 producer threads: one Philox call (8 entries) each per chunk
constexpr int kLoadWarp = kProdWarps, kMmaWarp = kProdWarps + 1;
constexpr int kTcThreads = (kProdWarps + 2) * 32;
constexpr int kMaxStages = 8;
static_assert(kProdWarps * 32 == kBM * (kBK / 8), "one 8-entry octet per producer thread and chunk");

struct TcArgs {
  const uint8_t *xt;   // nchunk packed X chunks of ncp * 64 bytes
  float *part;         // [splits][mpad][ncp]
  unsigned *status;
  int64_t nchunk, cps; // chunks, chunks per split
  int64_t m;           // rows of G
  int ncp;             // packed columns: a multiple of 16, <= 512
  int tmem_cols;       // power of two >= max(ncp, 32)
  int stages;
  uint32_t seed_lo, seed_hi;
};

// Pipeline per CTA (rows m0 .. m0 + 127 of G, chunks c0 .. c1 - 1): stage s of S holds one G
// tile (producer warps) and one X chunk (bulk copy); the MMA thread waits for both, issues the
// chunk's MMAs and commits them to empty[s], which frees the stage for both producers.
__global__ void __launch_bounds__(kTcThreads, 1) k_gauss_tc(const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = a.stages;
  const uint32_t bB = (uint32_t)a.ncp * (kBK * 2);
  uint8_t *sA = sm;
  uint8_t *sB = sm + (size_t)S * kTileA;
  uint64_t *full_g = reinterpret_cast<uint64_t *>(sB + (size_t)S * bB);
  uint64_t *full_x = full_g + S;
  uint64_t *empty = full_x + S;
  uint64_t *accum = empty + S;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(accum + 1);
  volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_g[s], kProdWarps);  // one arrival per producer warp
      mbar_init(&full_x[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort_f = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kLoadWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int64_t c0 = (int64_t)blockIdx.y * a.cps;
  const int64_t c1 = c0 + a.cps < a.nchunk ? c0 + a.cps : a.nchunk;
  const int nk = (int)(c1 - c0);
  const int64_t m0 = (int64_t)blockIdx.x * kBM;

  if (warp < kProdWarps) {
    // producers: row = thread mod 128, octet (8 entries along K) = thread div 128
    const int row = threadIdx.x & (kBM - 1);
    const int oct = threadIdx.x >> 7;
    const int64_t gi = m0 + row;
    const bool live = gi < a.m;
    uint8_t *dst0 = sA + (row >> 3) * kSBO + (row & 7) * 16 + oct * 128;
    // the Philox words of chunk k + 1 are drawn beside the Box-Muller step of chunk k (two
    // independent dependency chains per thread)
    const RoundKeys K = round_keys(a.seed_lo, a.seed_hi);
    uint64_t q = (uint64_t)c0 * (kBK / 8) + (uint64_t)oct;  // octet index of chunk k along K
    U4 wn = philox_rk((uint32_t)q, (uint32_t)(q >> 32), kStreamG, (uint32_t)gi, K);
    int s = 0;
    uint32_t ph = 0;
    for (int k = 0; k < nk; ++k) {
      // warp-uniform: a lane that gave up takes its whole warp out of the loop
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(&empty[s], ph ^ 1u, abort_f, a.status))) break;
      const U4 w = wn;
      if (k + 1 < nk) q += kBK / 8;
      wn = philox_rk((uint32_t)q, (uint32_t)(q >> 32), kStreamG, (uint32_t)gi, K);
      const uint2 v01 = box_muller_bf16x2_pair(w.x, w.y), v23 = box_muller_bf16x2_pair(w.z, w.w);
      uint4 v = make_uint4(v01.x, v01.y, v23.x, v23.y);
      if (!live) v = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4 *>(dst0 + (size_t)s * kTileA) = v;
      // each thread orders its own store before the MMA's (async-proxy) read; the warp then
      // arrives once
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_g[s]);
      if (++s == S) { s = 0; ph ^= 1u; }
    }
    if (warp < 4) {
      // epilogue: TMEM lanes 32 warp .. 32 warp + 31 hold rows m0 + 32 warp + lane
      const bool ok = mbar_wait(accum, 0u, abort_f, a.status);
      tc_fence_after();
      if (__all_sync(0xFFFFFFFFu, ok && !*abort_f)) {
        float *dst = a.part + (((int64_t)blockIdx.y * gridDim.x * kBM) + m0 + 32 * warp + lane) * a.ncp;
        for (int c = 0; c < a.ncp; c += 32) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
          const int nv = a.ncp - c < 32 ? a.ncp - c : 32;  // ncp is a multiple of 16
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (j < nv) *reinterpret_cast<uint4 *>(dst + c + j) = make_uint4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
      }
      tc_fence_before();
    }
  } else if (warp == kLoadWarp) {
    if (lane == 0) {
      int issued = 0, s = 0;
      uint32_t ph = 0;
      for (int k = 0; k < nk; ++k) {
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_f, a.status)) break;
        mbar_arrive_expect_tx(&full_x[s], bB);
        bulk_g2s(sB + (size_t)s * bB, a.xt + (size_t)(c0 + k) * bB, bB, &full_x[s]);
        issued = k + 1;
        if (++s == S) { s = 0; ph ^= 1u; }
      }
      // copies in flight land before the CTA exits: the last use of each stage completes
      // (on the normal path the MMA thread has already seen every one of them)
      const int first = issued > S ? issued - S : 0;
      for (int k = first; k < issued; ++k) {
        volatile int never = 0;
        mbar_wait(&full_x[k % S], (uint32_t)(k / S) & 1u, &never, a.status);
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      const int n0 = a.ncp < 256 ? a.ncp : 256;
      const uint32_t id0 = umma_idesc_bf16(kBM, n0);
      const uint32_t id1 = a.ncp > 256 ? umma_idesc_bf16(kBM, a.ncp - 256) : 0u;
      int s = 0;
      uint32_t ph = 0;
      for (int k = 0; k < nk; ++k) {
        if (!mbar_wait(&full_x[s], ph, abort_f, a.status)) break;
        if (!mbar_wait(&full_g[s], ph, abort_f, a.status)) break;
        tc_fence_after();
        const uint32_t ab = smem_u32(sA + (size_t)s * kTileA);
        const uint32_t bb = smem_u32(sB + (size_t)s * bB);
#pragma unroll
        for (int ks = 0; ks < kBK / 16; ++ks) {
          // K step ks covers core-matrix columns 2 ks, 2 ks + 1 (128 bytes apart)
          const uint64_t ad = umma_desc(ab + ks * 256, 128, kSBO);
          const uint32_t acc = (k > 0 || ks > 0) ? 1u : 0u;
          umma_bf16(tmem, ad, umma_desc(bb + ks * 256, 128, kSBO), id0, acc);
          if (a.ncp > 256) umma_bf16(tmem + 256, ad, umma_desc(bb + 32 * kSBO + ks * 256, 128, kSBO), id1, acc);
        }
        umma_commit(&empty[s]);
        if (++s == S) { s = 0; ph ^= 1u; }
      }
      umma_commit(accum);  // arrives once every MMA issued above has completed
    }
  }
  __syncthreads();
  if (warp == kLoadWarp) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// X (F32) -> BF16 chunks of 32 rows in the K-major core-matrix layout of the MMA's B operand:
// element (n, k) of chunk c (k = row - 32 c) at byte (n div 8) 512 + (k div 8) 128 + (n mod 8) 16
// + (k mod 8) 2.  Packed column n is X column c0 + n for n < nx, Y for n == ycol, zero otherwise;
// rows >= N are zero.  One CTA per 64 rows (two chunks): each warp reads 8 whole rows
// (float4 loads when VEC), rounds them to BF16 and stores them transposed in shared memory,
// word (n, kw) (rows 2 kw, 2 kw + 1 of column n) at n 32 + (kw + n div 4) mod 32 so that the
// 32 lanes of a store hit 32 banks; then 16-byte units are written out contiguously.
template <bool VEC>
__global__ void __launch_bounds__(256) k_pack_xt(const float *__restrict__ X, int64_t ldx, const float *__restrict__ Y,
                                                 int64_t N, int c0, int nx, int ycol, int ncp,
                                                 uint8_t *__restrict__ xt) {
  extern __shared__ uint32_t s32[];  // ncp x 32 words
  uint16_t *s16 = reinterpret_cast<uint16_t *>(s32);
  const int64_t k0 = (int64_t)blockIdx.x * 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; idx < ncp * 32; idx += 256) s32[idx] = 0u;
  __syncthreads();
  auto put = [&](int n, int r, float f) {
    const int w = n * 32 + (((r >> 1) + (n >> 2)) & 31);
    const __nv_bfloat16 b = __float2bfloat16_rn(f);
    s16[2 * w + (r & 1)] = *reinterpret_cast<const uint16_t *>(&b);
  };
  for (int rr = 0; rr < 8; ++rr) {
    const int r = warp * 8 + rr;
    const int64_t k = k0 + r;
    if (k >= N) break;
    const float *xr = X + k * ldx + c0;
    if (VEC) {
      const int ng4 = nx >> 2;  // nx <= 512: at most 4 float4 per lane
      float4 v[4];
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int g = lane + 32 * it;
        v[it] = g < ng4 ? __ldg(reinterpret_cast<const float4 *>(xr) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        const int g = lane + 32 * it;
        if (g < ng4) {
          put(4 * g, r, v[it].x);
          put(4 * g + 1, r, v[it].y);
          put(4 * g + 2, r, v[it].z);
          put(4 * g + 3, r, v[it].w);
        }
      }
      if (lane < nx - 4 * ng4) put(4 * ng4 + lane, r, xr[4 * ng4 + lane]);
    } else {
      for (int n = lane; n < nx; n += 32) put(n, r, xr[n]);
    }
    if (ycol >= 0 && lane == 0) put(ycol, r, Y[k]);
  }
  __syncthreads();
  // unit v of chunk half hc: column n = (v div 32) 8 + v mod 8, row octet k8 = 4 hc + (v div 8) mod 4
  const int per = ncp * 4;
  for (int u = threadIdx.x; u < 2 * per; u += 256) {
    const int hc = u >= per ? 1 : 0;
    const int v = u - hc * per;
    const int n = (v >> 5) * 8 + (v & 7);
    const int k8 = 4 * hc + ((v >> 3) & 3);
    uint32_t p[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = s32[n * 32 + ((4 * k8 + j + (n >> 2)) & 31)];
    *reinterpret_cast<uint4 *>(xt + ((size_t)(2 * blockIdx.x + hc) * ncp * 64) + (size_t)v * 16) =
        make_uint4(p[0], p[1], p[2], p[3]);
  }
}

// out[i, j] = scale * sum over splits of part[split][i][j] (fixed order); NaN after a timeout
template <typename TP, typename TO>
__global__ void k_gauss_reduce(const TP *__restrict__ part, int splits, int64_t mpad, int ncp, int64_t m, int nx,
                               int ycol, double scale, const unsigned *status, TO *SX, int64_t ldsx, TO *SY) {
  const bool bad = (*(volatile const unsigned *)status & ST_TIMEOUT) != 0;
  const int64_t total = m * ncp;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / ncp;
    const int j = (int)(idx - i * ncp);
    if (j >= nx && j != ycol) continue;
    double v = 0.0;
    for (int s = 0; s < splits; ++s) v += (double)part[((int64_t)s * mpad + i) * ncp + j];
    v *= scale;
    if (bad) v = __longlong_as_double(0x7FF8000000000000ll);
    if (j < nx) SX[i * ldsx + j] = (TO)v;
    else if (SY) SY[i] = (TO)v;
  }
}

// ------------------------------------------------------------------ FP64 path
constexpr int kF64M = 64, kF64N = 128, kF64K = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_gauss_f64(const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y,
                                                   int64_t N, int nx, int ycol, int64_t m, int64_t nchunk,
                                                   int64_t cps, uint32_t slo, uint32_t shi, double *part,
                                                   int64_t mpad, int ncpad) {
  extern __shared__ double sh[];
  double *sG = sh;                       // [64][33]
  double *sX = sh + kF64M * (kF64K + 1); // [32][129]
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * kF64M;
  const int n0 = blockIdx.y * kF64N;
  const int64_t ca = (int64_t)blockIdx.z * cps;
  const int64_t cb = ca + cps < nchunk ? ca + cps : nchunk;
  double acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
  for (int64_t c = ca; c < cb; ++c) {
    const int64_t k0 = c * kF64K;
    {  // G tile: row t / 4, octet t mod 4 (8 entries per Philox call)
      const int r = t >> 2, o = t & 3;
      const int64_t gi = m0 + r;
      double g[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (gi < m) {
        const uint64_t q = (uint64_t)(k0 >> 3) + o;
        const U4 w = philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), kStreamG, (uint32_t)gi, slo, shi);
        box_muller_f64(w.x, g[0], g[1]);
        box_muller_f64(w.y, g[2], g[3]);
        box_muller_f64(w.z, g[4], g[5]);
        box_muller_f64(w.w, g[6], g[7]);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) sG[r * (kF64K + 1) + o * 8 + e] = g[e];
    }
    for (int idx = t; idx < kF64K * kF64N; idx += 256) {
      const int r = idx / kF64N, j = idx - r * kF64N;
      const int64_t k = k0 + r;
      const int col = n0 + j;
      double v = 0.0;
      if (k < N) {
        if (col < nx) v = (double)X[k * ldx + col];
        else if (col == ycol) v = (double)Y[k];
      }
      sX[r * (kF64N + 1) + j] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kF64K; ++kk) {
      double av[4], bv[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sG[(ty * 4 + i) * (kF64K + 1) + kk];
#pragma unroll
      for (int j = 0; j < 8; ++j) bv[j] = sX[kk * (kF64N + 1) + tx * 8 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
      part[((int64_t)blockIdx.z * mpad + m0 + ty * 4 + i) * ncpad + n0 + tx * 8 + j] = acc[i][j];
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// ------------------------------------------------------------------ host side
GaussPlan gauss_plan(int64_t N, int d, int prec, int64_t m, bool with_y, int nsm) {
  GaussPlan p{};
  p.N = N; p.d = d; p.prec = prec; p.m = m; p.with_y = with_y;
  p.nsm = nsm > 0 ? nsm : 152;
  const int ncols = d + (with_y ? 1 : 0);
  if (prec == SLSE_PREC_FP64) {
    p.groups = 1;
    p.ncp = (int)cdiv(ncols, kF64N) * kF64N;
    p.nchunk = cdiv(N, kF64K);
    const int64_t mt = cdiv(m, kF64M), nt = p.ncp / kF64N;
    int64_t splits = (4 * (int64_t)p.nsm) / (mt * nt);
    if (splits < 1) splits = 1;
    if (splits > p.nchunk) splits = p.nchunk;
    p.cps = cdiv(p.nchunk, splits);
    p.splits = (int)cdiv(p.nchunk, p.cps);
    p.mpad = mt * kF64M;
    p.o_part = 0;
    p.total = al256((size_t)p.splits * p.mpad * p.ncp * 8) + 256;
    p.o_status = p.total - 256;
    return p;
  }
  p.groups = (ncols + 511) / 512;
  const int wmax = ncols < 512 ? ncols : 512;
  p.ncp = (wmax + 15) & ~15;
  int tc = 32;
  while (tc < p.ncp) tc <<= 1;
  p.tmem_cols = tc;
  const size_t bB = (size_t)p.ncp * kBK * 2;
  int S = (int)((232448 - 2048) / (kTileA + bB));
  if (S > kMaxStages) S = kMaxStages;
  p.stages = S;
  size_t smem = (size_t)S * (kTileA + bB) + (3 * S + 1) * 8 + 8 + 1024;
  // at most 512 / tmem_cols CTAs may share an SM (their TMEM allocations must all fit)
  const size_t floor_smem = 233472 / (512 / tc + 1) - 1024 + 1;
  if (smem < floor_smem) smem = floor_smem;
  p.smem = smem;
  const int per_sm = (int)(233472 / (smem + 1024)) < 512 / tc ? (int)(233472 / (smem + 1024)) : 512 / tc;
  p.nchunk = cdiv(N, kBK);
  const int64_t mt = cdiv(m, kBM);
  int64_t splits = ((int64_t)p.nsm * (per_sm > 0 ? per_sm : 1)) / mt;
  if (splits < 1) splits = 1;
  if (splits > p.nchunk) splits = p.nchunk;
  p.cps = cdiv(p.nchunk, splits);
  p.splits = (int)cdiv(p.nchunk, p.cps);
  p.mpad = mt * kBM;
  p.o_xt = 0;
  p.o_part = al256((size_t)cdiv(N, 2 * kBK) * 2 * bB);  // the pack writes chunks in pairs
  p.total = p.o_part + al256((size_t)p.splits * p.mpad * p.ncp * 4) + 256;
  p.o_status = p.total - 256;
  return p;
}

cudaError_t launch_pack_bf16(const float *X, int64_t ldx, int64_t N, int nx, int ncp, uint8_t *xt, cudaStream_t s) {
  if (ncp % 16 != 0 || ncp > 512 || nx > ncp) return cudaErrorInvalidValue;
  const bool vec = ldx % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0;
  const size_t psm = (size_t)ncp * 128;
  const unsigned pgrid = (unsigned)cdiv(N, 2 * kBK);
  cudaError_t e;
  if (vec) {
    if ((e = cudaFuncSetAttribute(k_pack_xt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm))) return e;
    k_pack_xt<true><<<pgrid, 256, psm, s>>>(X, ldx, nullptr, N, 0, nx, -1, ncp, xt);
  } else {
    if ((e = cudaFuncSetAttribute(k_pack_xt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm))) return e;
    k_pack_xt<false><<<pgrid, 256, psm, s>>>(X, ldx, nullptr, N, 0, nx, -1, ncp, xt);
  }
  return cudaGetLastError();
}

cudaError_t launch_gaussian(const GaussPlan &p, int xdtype, const void *X, int64_t ldx, const void *Y, uint64_t seed,
                            void *SX, int64_t ldsx, void *SY, double scale, unsigned *status, void *ws,
                            cudaStream_t s) {
  uint8_t *base = static_cast<uint8_t *>(ws);
  const uint32_t slo = (uint32_t)seed, shi = (uint32_t)(seed >> 32);
  cudaError_t e;
  if (p.prec == SLSE_PREC_FP64) {
    double *part = reinterpret_cast<double *>(base + p.o_part);
    const size_t smem = (size_t)(kF64M * (kF64K + 1) + kF64K * (kF64N + 1)) * 8;
    const dim3 grid((unsigned)(p.mpad / kF64M), (unsigned)(p.ncp / kF64N), (unsigned)p.splits);
    const int ycol = p.with_y ? p.d : -1;
    if (xdtype == SLSE_F64) {
      if ((e = cudaFuncSetAttribute(k_gauss_f64<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
      k_gauss_f64<double><<<grid, 256, smem, s>>>(static_cast<const double *>(X), ldx, static_cast<const double *>(Y),
                                                   p.N, p.d, ycol, p.m, p.nchunk, p.cps, slo, shi, part, p.mpad,
                                                   p.ncp);
    } else {
      if ((e = cudaFuncSetAttribute(k_gauss_f64<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
      k_gauss_f64<float><<<grid, 256, smem, s>>>(static_cast<const float *>(X), ldx, static_cast<const float *>(Y),
                                                 p.N, p.d, ycol, p.m, p.nchunk, p.cps, slo, shi, part, p.mpad, p.ncp);
    }
    if ((e = cudaGetLastError())) return e;
    const int64_t tot = p.m * p.ncp;
    const int rb = (int)(cdiv(tot, 256) < 8 * p.nsm ? cdiv(tot, 256) : 8 * p.nsm);
    k_gauss_reduce<double, double><<<rb, 256, 0, s>>>(part, p.splits, p.mpad, p.ncp, p.m, p.d, ycol, scale, status,
                                                      static_cast<double *>(SX), ldsx, static_cast<double *>(SY));
    return cudaGetLastError();
  }
  if (xdtype != SLSE_F32) return cudaErrorInvalidValue;
  uint8_t *xt = base + p.o_xt;
  float *part = reinterpret_cast<float *>(base + p.o_part);
  if ((e = cudaFuncSetAttribute(k_gauss_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem))) return e;
  const int ncols = p.d + (p.with_y ? 1 : 0);
  for (int g = 0; g < p.groups; ++g) {
    const int c0 = 512 * g;
    const int w = ncols - c0 < 512 ? ncols - c0 : 512;
    const int nx = p.d - c0 < w ? (p.d - c0 > 0 ? p.d - c0 : 0) : w;
    const int ycol = p.with_y && p.d >= c0 && p.d < c0 + w ? p.d - c0 : -1;
    const int ncp = (w + 15) & ~15;
    const bool vec = ldx % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0;
    const size_t psm = (size_t)ncp * 128;
    const unsigned pgrid = (unsigned)cdiv(p.N, 2 * kBK);
    if (vec) {
      if ((e = cudaFuncSetAttribute(k_pack_xt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm))) return e;
      k_pack_xt<true><<<pgrid, 256, psm, s>>>(static_cast<const float *>(X), ldx, static_cast<const float *>(Y), p.N,
                                             c0, nx, ycol, ncp, xt);
    } else {
      if ((e = cudaFuncSetAttribute(k_pack_xt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm))) return e;
      k_pack_xt<false><<<pgrid, 256, psm, s>>>(static_cast<const float *>(X), ldx, static_cast<const float *>(Y), p.N,
                                              c0, nx, ycol, ncp, xt);
    }
    if ((e = cudaGetLastError())) return e;
    TcArgs a{};
    a.xt = xt; a.part = part; a.status = status; a.nchunk = p.nchunk; a.cps = p.cps; a.m = p.m; a.ncp = ncp;
    int tc = 32;
    while (tc < ncp) tc <<= 1;
    a.tmem_cols = tc <= p.tmem_cols ? tc : p.tmem_cols;
    a.stages = p.stages;
    a.seed_lo = slo; a.seed_hi = shi;
    k_gauss_tc<<<dim3((unsigned)(p.mpad / kBM), (unsigned)p.splits), kTcThreads, p.smem, s>>>(a);
    if ((e = cudaGetLastError())) return e;
    const int64_t tot = p.m * ncp;
    const int rb = (int)(cdiv(tot, 256) < 8 * p.nsm ? cdiv(tot, 256) : 8 * p.nsm);
    k_gauss_reduce<float, __nv_bfloat16><<<rb, 256, 0, s>>>(
        part, p.splits, p.mpad, ncp, p.m, nx, ycol, scale, status, static_cast<__nv_bfloat16 *>(SX) + c0, ldsx,
        static_cast<__nv_bfloat16 *>(SY));
    if ((e = cudaGetLastError())) return e;
  }
  return cudaSuccess;
}

}  // namespace slse
