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
  } else {
    if (d <= 128) run(float{}, std::integral_constant<int, 4>{});
    else if (d <= 256) run(float{}, std::integral_constant<int, 8>{});
    else run(float{}, std::integral_constant<int, 16>{});
  }
  if (cudaGetLastError() != cudaSuccess) return SLSE_ECUDA;
  return SLSE_OK;
}
