// Differentiation through the least-squares estimate beta-hat = (X^T X)^{-1} X^T Y that
// SLSE-FRS converges to (its 2nd-stage fixed point satisfies X^T (Y - X beta) = 0).
// For a loss L(beta-hat) with v = dL/d(beta-hat):
//   w       = (X^T X)^{-1} v
//   dL/dY   = X w
//   dL/dX   = r w^T - (X w) beta-hat^T,  r = Y - X beta-hat (recomputed, not stored).
// The normal-equation solve is the M-IHS iteration of the 2nd stage with the gradient
// replaced by v - X^T X w, preconditioned by the H-hat^{-1} of the fit (paper Eqs. (7),
// (8)), so it converges at the fit's rate: w+ = w + mu H^{-1}(v - X^T X w) + eta (w - w_prev).
// Each iteration is one pass over X (the residual-gradient kernels with Y = 0).
#include <cmath>
#include <type_traits>

#include "slse_internal.cuh"

namespace slse {
namespace {

constexpr size_t kStateBytesA = 4096;

inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void k_init_adj(DevState *st, int rebase) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    DevState z = {};
    z.rebase = rebase;
    *st = z;
  }
}

// g <- v + g (g holds X^T (0 - X w) = -X^T X w); skipped once the stop flag is set.
__global__ void k_add_rhs(double *g, const double *v, int d, const DevState *st) {
  if (st->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d) g[i] = v[i] + g[i];
}

// One warp per row: a = x.w, p = x.beta (FP32 inputs: compensated products and sums with
// w and beta split into float head + tail, so both dot products carry about twice the
// working precision), then dY = a and dX = (y - p) w - a beta.  Lane l holds columns
// l + 32 q, q < MQ (MQ = ceil(d / 32) rounded up to 4, 8 or 16).
template <class T, int MQ>
__global__ void __launch_bounds__(256) k_vjp_rows(const T *X, int64_t ldx, const T *Y, int64_t N, int d,
                                                  const double *beta, const double *w, T *dX, int64_t lddx, T *dY) {
  using Tw = std::conditional_t<sizeof(T) == 8, double, float>;
  const int lane = threadIdx.x & 31;
  Tw bh[MQ], bl[MQ], wh[MQ], wl[MQ];
#pragma unroll
  for (int q = 0; q < MQ; ++q) {
    const int c = lane + 32 * q;
    const double bv = c < d ? beta[c] : 0.0, wv = c < d ? w[c] : 0.0;
    bh[q] = (Tw)bv; bl[q] = (Tw)(bv - (double)bh[q]);
    wh[q] = (Tw)wv; wl[q] = (Tw)(wv - (double)wh[q]);
  }
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += nw) {
    const T *x = X + i * ldx;
    T xv[MQ];
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const int c = lane + 32 * q;
      xv[q] = c < d ? x[c] : T(0);
    }
    Tw rf, af;
    if constexpr (sizeof(T) == 8) {
      double a = 0.0, p = 0.0;
#pragma unroll
      for (int q = 0; q < MQ; ++q) {
        a = fma(xv[q], wh[q], a);
        p = fma(xv[q], bh[q], p);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        p += __shfl_xor_sync(0xffffffffu, p, o);
      }
      af = a;
      rf = Y[i] - p;
    } else {
      // head/tail float pairs throughout (no FP64 arithmetic, which is slow on this part)
      float as = 0.f, ae = 0.f, ps = 0.f, pe = 0.f;
#pragma unroll
      for (int q = 0; q < MQ; ++q) {
        float pr, er, s, e2;
        two_prod(xv[q], wh[q], pr, er);
        two_sum(as, pr, s, e2);
        as = s;
        ae += e2 + er + xv[q] * wl[q];
        two_prod(xv[q], bh[q], pr, er);
        two_sum(ps, pr, s, e2);
        ps = s;
        pe += e2 + er + xv[q] * bl[q];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float as2 = __shfl_xor_sync(0xffffffffu, as, o), ae2 = __shfl_xor_sync(0xffffffffu, ae, o);
        const float ps2 = __shfl_xor_sync(0xffffffffu, ps, o), pe2 = __shfl_xor_sync(0xffffffffu, pe, o);
        float t, e;
        two_sum(as, as2, t, e);
        as = t; ae = (ae + ae2) + e;
        two_sum(ps, ps2, t, e);
        ps = t; pe = (pe + pe2) + e;
      }
      float rh, re;
      two_sum((float)Y[i], -ps, rh, re);
      rf = rh + (re - pe);
      af = as + ae;
    }
    if (lane == 0) dY[i] = (T)af;
    T *o = dX + i * lddx;
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const int c = lane + 32 * q;
      if (c < d) o[c] = (T)fma(rf, wh[q], -af * bh[q]);
    }
  }
}

// Packed FP32 pairs: one instruction does both halves.  a - b is fma(b, -1, a), which
// rounds once, exactly as the subtraction does.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// Knuth's TwoSum on each half: s + e = a + b exactly.
__device__ __forceinline__ void p_two_sum(float2 a, float2 b, float2 &s, float2 &e) {
  s = p_add(a, b);
  const float2 bb = p_sub(s, a);
  e = p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb));
}

template <int VMAX, int RPW>
__device__ __forceinline__ void vjp_load(const float *X, int64_t ldx, int64_t N, int d, int lane, int64_t i0,
                                         float4 (&x)[RPW][VMAX]) {
#pragma unroll
  for (int q = 0; q < RPW; ++q)
#pragma unroll
    for (int v = 0; v < VMAX; ++v) {
      const int c = 4 * lane + 128 * v;
      const int64_t i = i0 + q;
      x[q][v] = (i < N && c < d) ? __ldcs(reinterpret_cast<const float4 *>(X + i * ldx + c))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// FP32 rows, 16-byte aligned, d % 4 == 0: lane l holds columns 4 l + 128 v .. + 3
// (v < VMAX) of RPW rows at once (RPW * VMAX = 4), and the next RPW rows are loaded while
// this group is written.  Both dot products run as one Dot2 sum (error-free products and
// sums, the vector split into FP32 head + tail, as in the mixed gradient) on packed FP32
// pairs: the .x half accumulates -x . beta and the .y half -x . w, so a = x . w is as
// accurate as the residual (a row whose a cancels still gets a to ~2^-24 |a|).  The RPW
// sums of a warp are reduced together: each of the first log2(RPW) butterfly steps hands
// half of the rows to the partner lane, so that lane l ends with row l / (32 / RPW) after
// a plain butterfly over the remaining lanes; r = y - p is formed there and broadcast with
// a.  dX = r w - a beta needs no x.
template <int VMAX, int RPW, int MINB>
__global__ void __launch_bounds__(256, MINB) k_vjp_rows_f32v(const float *X, int64_t ldx, const float *Y, int64_t N,
                                                            int d, const double *beta, const double *w, float *dX,
                                                            int64_t lddx, float *dY) {
  constexpr int LR = RPW == 8 ? 3 : RPW == 4 ? 2 : RPW == 2 ? 1 : 0;  // log2 RPW
  constexpr int GL = 32 >> LR;                                         // lanes per row at the end
  static_assert((1 << LR) == RPW && RPW * VMAX == 4, "RPW must be 4 / VMAX, a power of two");
  const int lane = threadIdx.x & 31;
  // per column: (beta, w) heads, their negations, and the negated tails
  float2 b2[VMAX][4], nb2[VMAX][4], nl2[VMAX][4];
#pragma unroll
  for (int v = 0; v < VMAX; ++v)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = 4 * lane + 128 * v + e;
      const double bv = c < d ? beta[c] : 0.0, wv = c < d ? w[c] : 0.0;
      b2[v][e] = make_float2((float)bv, (float)wv);
      nb2[v][e] = make_float2(-b2[v][e].x, -b2[v][e].y);
      nl2[v][e] = make_float2(-(float)(bv - (double)b2[v][e].x), -(float)(wv - (double)b2[v][e].y));
    }
  const int64_t step = (((int64_t)gridDim.x * blockDim.x) >> 5) * RPW;
  int64_t i0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW;
  float4 x[RPW][VMAX];
  vjp_load<VMAX, RPW>(X, ldx, N, d, lane, i0, x);
  for (; i0 < N; i0 += step) {
    const int64_t iy = i0 + (lane / GL);  // the row this lane holds after the reduction
    const float y = iy < N ? __ldcs(Y + iy) : 0.f;
    float2 ns[RPW], nc[RPW];  // (-x . beta, -x . w) = ns + nc
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      float2 sum = make_float2(0.f, 0.f), cor = sum;
#pragma unroll
      for (int v = 0; v < VMAX; ++v)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float xv = e == 0 ? x[q][v].x : e == 1 ? x[q][v].y : e == 2 ? x[q][v].z : x[q][v].w;
          const float2 xx = make_float2(xv, xv);
          const float2 qn = p_mul(xx, nb2[v][e]);     // -fl(x head)
          const float2 ee = p_fma(xx, b2[v][e], qn);  // x head - fl(x head), exact
          float2 t, err;
          p_two_sum(sum, qn, t, err);
          sum = t;
          cor = p_fma(xx, nl2[v][e], p_add(cor, p_sub(err, ee)));
        }
      ns[q] = sum;
      nc[q] = cor;
    }
#pragma unroll
    for (int sp = 0; sp < LR; ++sp) {
      const int off = 16 >> sp, half = RPW >> (sp + 1);
      const bool up = (lane & off) != 0;  // keeps the upper half of the rows left
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float2 s_send = up ? ns[k] : ns[k + half], c_send = up ? nc[k] : nc[k + half];
        const float2 s_keep = up ? ns[k + half] : ns[k], c_keep = up ? nc[k + half] : nc[k];
        const float2 s_r = make_float2(__shfl_xor_sync(0xffffffffu, s_send.x, off),
                                       __shfl_xor_sync(0xffffffffu, s_send.y, off));
        const float2 c_r = make_float2(__shfl_xor_sync(0xffffffffu, c_send.x, off),
                                       __shfl_xor_sync(0xffffffffu, c_send.y, off));
        float2 t, err;
        p_two_sum(s_keep, s_r, t, err);
        ns[k] = t;
        nc[k] = p_add(p_add(c_keep, c_r), err);
      }
    }
#pragma unroll
    for (int off = GL / 2; off > 0; off >>= 1) {
      const float2 s_r = make_float2(__shfl_xor_sync(0xffffffffu, ns[0].x, off),
                                     __shfl_xor_sync(0xffffffffu, ns[0].y, off));
      const float2 c_r = make_float2(__shfl_xor_sync(0xffffffffu, nc[0].x, off),
                                     __shfl_xor_sync(0xffffffffu, nc[0].y, off));
      float2 t, err;
      p_two_sum(ns[0], s_r, t, err);
      ns[0] = t;
      nc[0] = p_add(p_add(nc[0], c_r), err);
    }
    vjp_load<VMAX, RPW>(X, ldx, N, d, lane, i0 + step, x);
    float rh, re;
    two_sum(y, ns[0].x, rh, re);
    const float r = rh + (re + nc[0].x);
    const float a = -(ns[0].y + nc[0].y);
    if ((lane & (GL - 1)) == 0 && iy < N) dY[iy] = a;
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const float rq = __shfl_sync(0xffffffffu, r, q * GL), aq = __shfl_sync(0xffffffffu, a, q * GL);
      const int64_t i = i0 + q;
      const float2 r2 = make_float2(rq, rq), na2 = make_float2(-aq, -aq);
#pragma unroll
      for (int v = 0; v < VMAX; ++v) {
        const int col = 4 * lane + 128 * v;
        if (i < N && col < d) {
          const float2 o0 = p_fma(r2, make_float2(b2[v][0].y, b2[v][1].y), p_mul(na2, make_float2(b2[v][0].x, b2[v][1].x)));
          const float2 o1 = p_fma(r2, make_float2(b2[v][2].y, b2[v][3].y), p_mul(na2, make_float2(b2[v][2].x, b2[v][3].x)));
          __stcs(reinterpret_cast<float4 *>(dX + i * lddx + col), make_float4(o0.x, o0.y, o1.x, o1.y));
        }
      }
    }
  }
}

// Pinned mailbox for the stop flag (one per host thread).
struct MailboxA {
  DevState *h = nullptr;
  ~MailboxA() {
    if (h) cudaFreeHost(h);
  }
  DevState *get() {
    if (!h && cudaHostAlloc((void **)&h, 4 * sizeof(DevState), cudaHostAllocDefault) != cudaSuccess) h = nullptr;
    return h;
  }
};
thread_local MailboxA t_mbox;

struct AdjLayout {
  int nblk;
  size_t o_state, o_part, o_g, o_ring, o_b0, o_d32, o_r0, o_y0, total;
};

AdjLayout adj_layout(const slse_problem *p, int prec, int nsm) {
  AdjLayout L{};
  const int d = p->d;
  L.nblk = 2 * (nsm > 0 ? nsm : 152);
  size_t o = 0;
  auto take = [&](size_t b) { const size_t r = o; o += al(b); return r; };
  L.o_state = take(kStateBytesA);
  L.o_part = take((size_t)L.nblk * d * 8);
  L.o_g = take((size_t)d * 8);
  L.o_ring = take((size_t)3 * d * 8);
  L.o_b0 = take((size_t)d * 8);
  L.o_d32 = take((size_t)d * 4);
  L.o_r0 = take(prec == SLSE_PREC_MIXED_BF16 ? (size_t)p->N * 4 : 0);
  L.o_y0 = take((size_t)p->N * (p->dtype == SLSE_F64 ? 8 : 4));
  L.total = o;
  return L;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

slse_status from_bits(unsigned bits) {
  if (bits & ST_TIMEOUT) return SLSE_ETIMEOUT;
  if (bits & ST_NUMERIC) return SLSE_ENUMERIC;
  if (bits & ST_NOTCONV) return SLSE_ENOTCONV;
  return SLSE_OK;
}

#define CKA(call)                              \
  do {                                         \
    if ((call) != cudaSuccess) {               \
      cudaGetLastError();                      \
      return SLSE_ECUDA;                       \
    }                                          \
  } while (0)

}  // namespace
}  // namespace slse

using namespace slse;

extern "C" size_t slse_solve_normal_workspace(const slse_problem *prob, int32_t prec) {
  if (!valid_problem(prob)) return 0;
  return adj_layout(prob, prec, sm_count()).total;
}

extern "C" slse_status slse_solve_normal(const slse_problem *prob, const double *Hinv, const double *v, double *w_out,
                                         const slse_schedule *sched, slse_report *report, void *workspace,
                                         size_t ws_bytes, slse_stream_t stream) {
  if (report) *report = slse_report{};
  if (!valid_problem(prob) || !Hinv || !v || !w_out || !sched) return SLSE_EINVAL;
  if (is_host_pointer(prob->X) || is_host_pointer(Hinv) || is_host_pointer(v) || is_host_pointer(w_out))
    return SLSE_EINVAL;
  const int prec = sched->prec;
  if (prec != SLSE_PREC_FP64 && prec != SLSE_PREC_MIXED_BF16) return SLSE_EINVAL;
  if (prec == SLSE_PREC_MIXED_BF16 && prob->dtype != SLSE_F32) return SLSE_EINVAL;
  if (sched->T < 1 || sched->r < prob->d || !std::isfinite(sched->mu) || !std::isfinite(sched->eta)) return SLSE_EINVAL;
  const int nsm = sm_count();
  if (nsm <= 0) return SLSE_ECUDA;
  const AdjLayout L = adj_layout(prob, prec, nsm);
  void *ws = workspace;
  bool owned = false;
  cudaStream_t s = (cudaStream_t)stream;
  if (!ws) {
    if (cudaMallocAsync(&ws, L.total, s) != cudaSuccess) {
      cudaGetLastError();
      return SLSE_ENOMEM;
    }
    owned = true;
  } else if (ws_bytes < L.total) {
    return SLSE_ENOMEM;
  }
  struct Free {
    void *p;
    bool own;
    cudaStream_t s;
    ~Free() {
      if (own) cudaFreeAsync(p, s);
    }
  } guard{ws, owned, s};
  char *base = static_cast<char *>(ws);
  DevState *st = reinterpret_cast<DevState *>(base + L.o_state);
  double *part = reinterpret_cast<double *>(base + L.o_part);
  double *g = reinterpret_cast<double *>(base + L.o_g);
  double *ring = reinterpret_cast<double *>(base + L.o_ring);
  double *b0 = reinterpret_cast<double *>(base + L.o_b0);
  float *d32 = reinterpret_cast<float *>(base + L.o_d32);
  float *r0 = prec == SLSE_PREC_MIXED_BF16 ? reinterpret_cast<float *>(base + L.o_r0) : nullptr;
  void *y0 = base + L.o_y0;
  const int d = prob->d;
  const bool mixed = prec == SLSE_PREC_MIXED_BF16;

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CKA(cudaEventCreate(&e0));
  CKA(cudaEventCreate(&e1));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{e0, e1};
  CKA(cudaEventRecord(e0, s));
  k_init_adj<<<1, 32, 0, s>>>(st, mixed ? 1 : 0);
  CKA(cudaGetLastError());
  CKA(cudaMemsetAsync(ring, 0, (size_t)3 * d * 8, s));
  CKA(cudaMemsetAsync(y0, 0, (size_t)prob->N * (prob->dtype == SLSE_F64 ? 8 : 4), s));

  UpdateArgs ua{};
  ua.g = g; ua.Hinv = Hinv; ua.beta_ring = ring; ua.beta0 = b0; ua.delta32 = d32;
  ua.hist = nullptr; ua.hist_cap = 0; ua.d = d; ua.mu = sched->mu; ua.eta = sched->eta; ua.T = sched->T;
  const double rho = std::sqrt((double)d / (double)sched->r);
  ua.thr = sched->tol > 0.0 ? sched->tol * (1.0 - rho) / rho : 0.0;
  ua.stage2 = 1; ua.mixed = mixed ? 1 : 0; ua.check_done = 1;
  DevState *mb = t_mbox.get();
  if (!mb) return SLSE_ECUDA;
  cudaEvent_t flag[2];
  CKA(cudaEventCreateWithFlags(&flag[0], cudaEventDisableTiming));
  CKA(cudaEventCreateWithFlags(&flag[1], cudaEventDisableTiming));
  struct Ev2 {
    cudaEvent_t *f;
    ~Ev2() {
      cudaEventDestroy(f[0]);
      cudaEventDestroy(f[1]);
    }
  } evf{flag};
  int launches = 3;
  for (int k = 0; k < sched->T; ++k) {
    if (launch_grad(mixed ? GM_MIXED : GM_F64, prob->dtype, prob->X, prob->ldx, y0, prob->N, d, ring, st, d32, r0, b0,
                    part, L.nblk, 1, s) != cudaSuccess)
      return SLSE_ECUDA;
    if (launch_reduce(part, L.nblk, d, 1.0, g, st, 1, s) != cudaSuccess) return SLSE_ECUDA;
    k_add_rhs<<<(d + 255) / 256, 256, 0, s>>>(g, v, d, st);
    CKA(cudaGetLastError());
    ua.first = k == 0;
    if (launch_update(ua, st, s) != cudaSuccess) return SLSE_ECUDA;
    launches += mixed ? 5 : 4;
    // iteration k+1 is enqueued before the stop flag of iteration k is read back
    CKA(cudaMemcpyAsync(&mb[k & 1], st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CKA(cudaEventRecord(flag[k & 1], s));
    if (k > 0) {
      CKA(cudaEventSynchronize(flag[(k - 1) & 1]));
      if (((volatile DevState *)&mb[(k - 1) & 1])->done) break;
    }
  }
  if (launch_copy_beta(ring, st, d, w_out, s) != cudaSuccess) return SLSE_ECUDA;
  CKA(cudaMemcpyAsync(&mb[2], st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CKA(cudaEventRecord(e1, s));
  CKA(cudaEventSynchronize(e1));
  const volatile DevState *fv = &mb[2];
  DevState fin{};
  fin.iter = fv->iter;
  fin.status = fv->status;
  fin.rel_step = fv->rel_step;
  fin.rebases = fv->rebases;
  const slse_status status = from_bits(fin.status);
  if (report) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    report->ms_total = ms;
    report->ms_stage2 = ms;
    report->iters_stage2 = fin.iter;
    report->final_rel_step = fin.rel_step;
    report->rebases = fin.rebases;
    report->kernels = launches;
    report->status = status;
  }
  return status;
}

extern "C" slse_status slse_ols_vjp(const slse_problem *prob, const double *beta, const double *w, void *dX,
                                    int64_t lddx, void *dY, slse_stream_t stream) {
  if (!valid_problem(prob) || !beta || !w || !dX || !dY || lddx < prob->d) return SLSE_EINVAL;
  if (is_host_pointer(prob->X) || is_host_pointer(prob->Y) || is_host_pointer(beta) || is_host_pointer(w) ||
      is_host_pointer(dX) || is_host_pointer(dY))
    return SLSE_EINVAL;
  const int nsm = sm_count();
  if (nsm <= 0) return SLSE_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)(8 * nsm);
  auto run = [&](auto tag, auto mq) {
    using T = decltype(tag);
    constexpr int MQ = decltype(mq)::value;
    k_vjp_rows<T, MQ><<<grid, 256, 0, s>>>(static_cast<const T *>(prob->X), prob->ldx,
                                           static_cast<const T *>(prob->Y), prob->N, prob->d, beta, w,
                                           static_cast<T *>(dX), lddx, static_cast<T *>(dY));
  };
  const int d = prob->d;
  if (prob->dtype == SLSE_F64) {
    if (d <= 128) run(double{}, std::integral_constant<int, 4>{});
    else if (d <= 256) run(double{}, std::integral_constant<int, 8>{});
    else run(double{}, std::integral_constant<int, 16>{});
  } else if (d % 4 == 0 && prob->ldx % 4 == 0 && lddx % 4 == 0 && ((uintptr_t)prob->X & 15) == 0 &&
             ((uintptr_t)dX & 15) == 0) {
    // 3 CTAs per SM with the next rows in flight (0.81 of the HBM copy rate at d = 128, where
    // the packed Dot2 arithmetic sets the pace); 2 above d = 128, where 3 would spill
    auto runv = [&](auto vmax) {
      constexpr int V = decltype(vmax)::value, MB = V == 1 ? 3 : 2;
      k_vjp_rows_f32v<V, 4 / V, MB><<<(unsigned)(MB * nsm), 256, 0, s>>>(
          static_cast<const float *>(prob->X), prob->ldx, static_cast<const float *>(prob->Y), prob->N, d, beta, w,
          static_cast<float *>(dX), lddx, static_cast<float *>(dY));
    };
    if (d <= 128) runv(std::integral_constant<int, 1>{});
    else if (d <= 256) runv(std::integral_constant<int, 2>{});
    else runv(std::integral_constant<int, 4>{});
  } else {
    if (d <= 128) run(float{}, std::integral_constant<int, 4>{});
    else if (d <= 256) run(float{}, std::integral_constant<int, 8>{});
    else run(float{}, std::integral_constant<int, 16>{});
  }
  if (cudaGetLastError() != cudaSuccess) return SLSE_ECUDA;
  return SLSE_OK;
}
