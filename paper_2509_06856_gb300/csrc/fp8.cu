// FP8 form of the sketch (an extension: the paper stores its sketches in double
// precision).  U holds E4M3 values with one power-of-two scale 2^k per 32-column block of
// a row (byte k + 127); V stays BF16.  The 1st-stage subproblems read U at one byte per
// element, half the traffic of the BF16 form.  The Hessian-sketch rows are kept in BF16
// (the SRHT's second pass writes them there); where they share rows with the 1st-stage
// sketches they are widened from the FP8 form (exactly: an E4M3 value times a power of two
// is a BF16 value) for the exact Gram matrix.
//   k_grad_mx:     1st-stage residual-gradient partials on MXFP8 rows (FP32 accumulation,
//                  per-CTA FP64 partials reduced by launch_reduce);
//   k_mx_to_bf16:  rows of the FP8 form widened to BF16;
//   k_quantize_mx: BF16 rows to the FP8 form (single-pass sketch sizes).
#include <cuda_fp8.h>

#include "slse_internal.cuh"

namespace slse {
namespace {

constexpr int kThreads = 256, kWarps = kThreads / 32;

__device__ __forceinline__ float e4m3_to_float(uint8_t q) {
  const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3);
  return __half2float(__half(h));
}

__device__ __forceinline__ float exp2i(int k) { return ldexpf(1.f, k); }

// Sixteen E4M3 values (one 16-byte word) widened to FP32.
__device__ __forceinline__ void unpack16(const uint4 w, float (&f)[16]) {
  const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(ww[i] & 0xFFFFu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(ww[i] >> 16), __NV_E4M3);
    const float2 a = __half22float2(__half2(lo)), b = __half22float2(__half2(hi));
    f[4 * i + 0] = a.x; f[4 * i + 1] = a.y; f[4 * i + 2] = b.x; f[4 * i + 3] = b.y;
  }
}

// g partials = sum_i u_i (v_i - u_i . beta) over rows [0, nrows) of the FP8 form.  Lane l
// holds columns 16 l .. 16 l + 15 (block l / 2); RPW rows per warp step.
template <int RPW>
__global__ void __launch_bounds__(kThreads, 2) k_grad_mx(const uint8_t *U, int64_t ldq, const uint8_t *S, int64_t nsb,
                                                         const __nv_bfloat16 *V, int64_t nrows, int d,
                                                         const double *beta_ring, const DevState *st, double *part) {
  __shared__ double sm[kWarps][512];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  const double *beta = beta_ring + (size_t)(st->iter % 3) * d;
  const int c0 = lane * 16;
  const bool live = c0 < d;
  float b[16], g[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    b[e] = (live && c0 + e < d) ? (float)beta[c0 + e] : 0.f;
    g[e] = 0.f;
  }
  for (int64_t i0 = gw * RPW; i0 < nrows; i0 += nw * RPW) {
    uint4 raw[RPW];
    float sc[RPW], y[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const int64_t i = i0 + q;
      const bool rv = i < nrows && live;
      raw[q] = rv ? __ldg(reinterpret_cast<const uint4 *>(U + i * ldq + c0)) : make_uint4(0u, 0u, 0u, 0u);
      sc[q] = rv ? exp2i((int)S[i * nsb + (lane >> 1)] - 127) : 0.f;
      y[q] = i < nrows ? __bfloat162float(V[i]) : 0.f;
    }
    // a lane's 16 columns share one block scale: u . beta = 2^k (q . beta), u r = q (2^k r)
    float u[RPW][16], s[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      unpack16(raw[q], u[q]);
      float acc = 0.f;
#pragma unroll
      for (int e = 0; e < 16; ++e) acc = fmaf(u[q][e], b[e], acc);
      s[q] = acc * sc[q];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < RPW; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const float r = (y[q] - s[q]) * sc[q];
#pragma unroll
      for (int e = 0; e < 16; ++e) g[e] = fmaf(u[q][e], r, g[e]);
    }
  }
  if (live)
#pragma unroll
    for (int e = 0; e < 16; ++e)
      if (c0 + e < d) sm[warp][c0 + e] = (double)g[e];
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += kThreads) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += sm[w][c];
    part[(size_t)blockIdx.x * d + c] = t;
  }
}

// Scalar form for d not a multiple of 16 (one element per lane step).
__global__ void __launch_bounds__(kThreads) k_grad_mx_s(const uint8_t *U, int64_t ldq, const uint8_t *S, int64_t nsb,
                                                        const __nv_bfloat16 *V, int64_t nrows, int d,
                                                        const double *beta_ring, const DevState *st, double *part) {
  __shared__ double sm[kWarps][512];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  const double *beta = beta_ring + (size_t)(st->iter % 3) * d;
  float g[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) g[q] = 0.f;
  for (int64_t i = gw; i < nrows; i += nw) {
    float u[16], acc = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int c = lane + 32 * q;
      u[q] = c < d ? e4m3_to_float(U[i * ldq + c]) * exp2i((int)S[i * nsb + c / 32] - 127) : 0.f;
      acc = fmaf(u[q], c < d ? (float)beta[c] : 0.f, acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    const float r = __bfloat162float(V[i]) - acc;
#pragma unroll
    for (int q = 0; q < 16; ++q) g[q] = fmaf(u[q], r, g[q]);
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int c = lane + 32 * q;
    if (c < d) sm[warp][c] = (double)g[q];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += kThreads) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += sm[w][c];
    part[(size_t)blockIdx.x * d + c] = t;
  }
}

__global__ void k_mx_to_bf16(const uint8_t *U, int64_t ldq, const uint8_t *S, int64_t nsb, int64_t rows, int d,
                             __nv_bfloat16 *out, int64_t ldo) {
  const int64_t n = rows * (int64_t)d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / d;
    const int c = (int)(t - i * d);
    const float v = e4m3_to_float(U[i * ldq + c]) * exp2i((int)S[i * nsb + c / 32] - 127);
    out[i * ldo + c] = __float2bfloat16_rn(v);  // exact: 4 significant bits in the BF16 range
  }
}

// One warp per (row, 32-column block): block exponent from the block's largest magnitude,
// then E4M3 rounding of value / 2^k.
__global__ void k_quantize_mx(const __nv_bfloat16 *A, int64_t lda, int64_t rows, int d, uint8_t *U, int64_t ldq,
                              uint8_t *S, int64_t nsb) {
  const int lane = threadIdx.x & 31;
  const int64_t nblk = rows * nsb;
  for (int64_t wb = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wb < nblk;
       wb += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t i = wb / nsb;
    const int blk = (int)(wb - i * nsb);
    const int c = blk * 32 + lane;
    const float x = c < d ? __bfloat162float(A[i * lda + c]) : 0.f;
    float am = fabsf(x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
    const uint32_t bits = __float_as_uint(am);
    const int E = (int)((bits >> 23) & 0xFFu);
    int k = -127;
    if (am > 0.f && E != 0) k = (bits & 0x7FFFFFu) <= 0x600000u ? (E - 127) - 8 : (E - 127) - 7;
    k = k < -127 ? -127 : (k > 127 ? 127 : k);
    if (c < d) U[i * ldq + c] = (uint8_t)__nv_cvt_float_to_fp8(x * ldexpf(1.f, -k), __NV_SATFINITE, __NV_E4M3);
    if (lane == 0) S[i * nsb + blk] = (uint8_t)(k + 127);
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 65535LL * 64) g = 65535LL * 64;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_grad_mx(const uint8_t *U, int64_t ldq, const uint8_t *S, int64_t nsb, const __nv_bfloat16 *V,
                           int64_t nrows, int d, const double *beta_ring, const DevState *st, double *part, int nblk,
                           cudaStream_t s) {
  if (d < 1 || d > 512) return cudaErrorInvalidValue;
  const bool vec = d % 16 == 0 && ldq % 16 == 0 && reinterpret_cast<uintptr_t>(U) % 16 == 0;
  if (vec) k_grad_mx<4><<<nblk, kThreads, 0, s>>>(U, ldq, S, nsb, V, nrows, d, beta_ring, st, part);
  else k_grad_mx_s<<<nblk, kThreads, 0, s>>>(U, ldq, S, nsb, V, nrows, d, beta_ring, st, part);
  return cudaGetLastError();
}

cudaError_t launch_mx_to_bf16(const uint8_t *U, int64_t ldq, const uint8_t *S, int64_t nsb, int64_t rows, int d,
                              __nv_bfloat16 *out, int64_t ldo, cudaStream_t s) {
  if (rows < 1) return cudaSuccess;
  k_mx_to_bf16<<<grid_for(rows * d, 256), 256, 0, s>>>(U, ldq, S, nsb, rows, d, out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_quantize_mx(const __nv_bfloat16 *A, int64_t lda, int64_t rows, int d, uint8_t *U, int64_t ldq,
                               uint8_t *S, int64_t nsb, cudaStream_t s) {
  if (rows < 1) return cudaSuccess;
  k_quantize_mx<<<grid_for(rows * nsb * 32, 256), 256, 0, s>>>(A, lda, rows, d, U, ldq, S, nsb);
  return cudaGetLastError();
}

}  // namespace slse
