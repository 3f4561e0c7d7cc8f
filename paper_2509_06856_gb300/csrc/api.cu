// C ABI of the SLSE-FRS library: argument validation, workspace layout, and the
// host-side stage loop of Algorithm 2 (paper Sec. 3).  All arithmetic runs in the
// kernels of draws.cu, srht.cu, grad.cu and linalg.cu.
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "slse_internal.cuh"

using namespace slse;

// Host memory (pinned or pageable) as opposed to device or managed memory.
bool slse::is_host_pointer(const void *ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

namespace {
std::atomic<long long> g_spin_limit{0};
}
long long slse::debug_spin_limit() { return g_spin_limit.load(std::memory_order_relaxed); }

bool slse::valid_problem(const slse_problem *p) {
  if (!p || !p->X || !p->Y) return false;
  if (p->N < 1 || p->d < 1 || p->d > 512 || p->d > p->N) return false;
  if (p->ldx < p->d) return false;
  if (p->dtype != SLSE_F64 && p->dtype != SLSE_F32) return false;
  int64_t np = 1;
  while (np < p->N) np <<= 1;
  if (np > kMaxPaddedRows) return false;
  return true;
}


namespace {

// slse_gram: F32 X, or BF16 X with a row stride that is a multiple of 8 (Y unused but non-null)
bool valid_gram_problem(const slse_problem *p) {
  if (!p) return false;
  if (p->dtype == SLSE_BF16) {
    slse_problem q = *p;
    q.dtype = SLSE_F32;
    return slse::valid_problem(&q) && p->ldx % 8 == 0;
  }
  return slse::valid_problem(p) && p->dtype == SLSE_F32;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kStateBytes = 4096;  // DevState + per-CTA partials of the update kernel
constexpr int64_t kMaxNp = kMaxPaddedRows;

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

int64_t padded(int64_t N) {
  int64_t p = 1;
  while (p < N) p <<= 1;
  return p;
}

struct Sched {
  std::vector<int64_t> m;
  std::vector<int32_t> a;
  int64_t r;
  double mu, eta, tol;
  int T, prec, momentum_reset;
  int kind = SLSE_SRHT;
  int stage2 = SLSE_STAGE2_CORRECTION;
};

bool is_pow2(int64_t m) { return m >= 1 && (m & (m - 1)) == 0; }

bool make_sched(const slse_problem *p, const slse_schedule *s, Sched &o) {
  const int64_t Np = padded(p->N);
  if (!s) {
    int64_t mb[64];
    int32_t ab[64];
    slse_schedule d;
    const int K = slse_default_schedule(p->N, p->d, &d, mb, ab, 64);
    if (K > 64) return false;
    o.m.assign(mb, mb + K);
    o.a.assign(ab, ab + K);
    o.r = d.r; o.mu = d.mu; o.eta = d.eta; o.tol = d.tol; o.T = d.T; o.prec = d.prec;
    o.momentum_reset = d.momentum_reset;
    o.kind = SLSE_SRHT;
    o.stage2 = d.stage2;
    return true;
  }
  if (s->stage2 != SLSE_STAGE2_FULL && s->stage2 != SLSE_STAGE2_CORRECTION) return false;
  if (s->K < 0 || (s->K > 0 && (!s->m || !s->a))) return false;
  if (s->kind != SLSE_SRHT && s->kind != SLSE_COUNTSKETCH && s->kind != SLSE_GAUSSIAN) return false;
  if (s->prec != SLSE_PREC_FP64 && s->prec != SLSE_PREC_MIXED_BF16 && s->prec != SLSE_PREC_MIXED_FP8) return false;
  if (s->prec != SLSE_PREC_FP64 && p->dtype != SLSE_F32) return false;
  if (s->prec == SLSE_PREC_MIXED_FP8 && s->kind != SLSE_SRHT) return false;  // FP8 form: SRHT only
  if (s->r < p->d || s->r > Np || s->T < 0) return false;
  if (!std::isfinite(s->mu) || !std::isfinite(s->eta) || !std::isfinite(s->tol)) return false;
  o.m.assign(s->m, s->m + s->K);
  o.a.assign(s->a, s->a + s->K);
  for (int i = 0; i < s->K; ++i) {
    if (o.m[i] < 1 || o.m[i] > Np || o.a[i] < 0) return false;
    if (i > 0 && o.m[i] <= o.m[i - 1]) return false;
  }
  if (s->kind == SLSE_COUNTSKETCH)
    for (int i = 0; i < s->K; ++i)
      if (!is_pow2(o.m[i])) return false;  // the nested CountSketch family has sizes 2^l
  o.r = s->r; o.mu = s->mu; o.eta = s->eta; o.tol = s->tol; o.T = s->T; o.prec = s->prec;
  o.momentum_reset = s->momentum_reset;
  o.kind = s->kind;
  o.stage2 = s->stage2;
  return true;
}

// ------------------------------------------------------------------ workspace layout
struct Layout {
  size_t total = 0;
  size_t take(size_t bytes) {
    const size_t o = align256(total);
    total = o + align256(bytes);
    return o;
  }
};

struct FitLayout {
  int64_t Np, n_samp, h0, ldu;
  int64_t ld16, nsb;        // FP8 form: BF16 leading dimension, scale bytes per row
  SrhtPlan sp;
  bool cs;                  // CountSketch family instead of the SRHT
  CsPlan csp;
  bool gauss;               // SRHT subproblems, Gaussian Hessian sketch
  GaussPlan gp;
  std::vector<int64_t> lvl_off;  // CountSketch: first row in U of the sketch of each schedule size
  int nblk;
  bool host_in;
  bool dc;                  // mixed 2nd stage in correction form (its Gram workspace in the big region)
  GramPlan grp;
  bool gw;                  // correction form: G_b from the SRHT intermediate W (W^T W = n2 X^T X)
  GramWPlan gwp;
  size_t o_gpart;           // its partial sums, inside the big region after W and its Y column
  size_t o_xin, o_yin, o_g0, o_be, o_de, o_gb, o_gst;
  bool sig_side;            // two-pass SRHT: sigma and pos drawn on a side stream beside pass 1
  size_t o_sigws;           // the temporaries of that sort (the big region is W by then)
  size_t o_state, o_psd, o_sigma, o_pos, o_big, o_wy, o_u, o_v, o_A, o_R, o_Hinv, o_qr, o_chol, o_part, o_g,
      o_ring, o_b0, o_d32, o_out, o_r0, o_us, o_hat16;
  size_t total;
};

// bytes per element of the sketch rows U, of the pass-1 intermediate W and of V
size_t elem_bytes_u(int prec) { return prec == SLSE_PREC_FP64 ? 8 : (prec == SLSE_PREC_MIXED_FP8 ? 1 : 2); }
size_t elem_bytes_w(int prec) { return prec == SLSE_PREC_FP64 ? 8 : 2; }
int64_t mx_blocks(int d) { return (d + 31) / 32; }

FitLayout fit_layout(const slse_problem *p, const Sched &s, int nsm) {
  FitLayout L{};
  const int d = p->d;
  L.Np = padded(p->N);
  L.sp = srht_plan(L.Np);
  L.cs = s.kind == SLSE_COUNTSKETCH;
  const int64_t mK = s.m.empty() ? 0 : s.m.back();
  if (L.cs) {
    // U holds the sketch of every schedule size, in schedule order, then the r rows of S-hat
    int64_t off = 0;
    for (int64_t m : s.m) { L.lvl_off.push_back(off); off += m; }
    L.h0 = off;
    L.n_samp = off + s.r;
    L.csp = cs_plan(p->N, d, s.prec, s.m.empty() ? 0 : s.m.front(), mK, s.r);
  } else if (s.kind == SLSE_GAUSSIAN) { L.h0 = mK; L.n_samp = mK; }  // S-hat is not sampled
  else if (mK + s.r <= L.Np) { L.h0 = mK; L.n_samp = mK + s.r; }
  else { L.h0 = 0; L.n_samp = mK > s.r ? mK : s.r; }
  const bool fp8 = s.prec == SLSE_PREC_MIXED_FP8;
  L.ld16 = (d + 7) & ~int64_t(7);
  L.ldu = fp8 ? ((d + 15) & ~int64_t(15)) : L.ld16;
  L.nsb = mx_blocks(d);
  const size_t eu = elem_bytes_u(s.prec), ew = elem_bytes_w(s.prec), ev = fp8 ? 2 : eu;
  L.nblk = 2 * (nsm > 0 ? nsm : 152);
  Layout w;
  L.o_state = w.take(kStateBytes);
  const size_t nperm = L.cs ? 0 : 4 * (size_t)L.Np;
  L.o_psd = w.take(nperm);
  L.o_sigma = w.take(nperm);
  L.o_pos = w.take(nperm);
  L.sig_side = !L.cs && !L.sp.single && L.n_samp > 0;
  L.o_sigws = w.take(L.sig_side ? draws_one_ws_bytes(L.Np) : 0);
  size_t big = L.cs ? L.csp.total : draws_ws_bytes(L.Np);
  const size_t wbytes = (L.sp.single || L.cs) ? 0 : (size_t)L.Np * L.ld16 * ew;
  const size_t wybytes = (L.sp.single || L.cs) ? 0 : (size_t)L.Np * ew;
  if (wbytes + align256(wybytes) + 256 > big) big = align256(wbytes) + align256(wybytes);
  // FP8 form at single-pass sizes: the BF16 rows are formed in this region, then quantised
  if (fp8 && L.sp.single && (size_t)L.n_samp * L.ld16 * 2 > big) big = (size_t)L.n_samp * L.ld16 * 2;
  // Gaussian Hessian sketch: its packed X and partial sums reuse this region after the SRHT
  L.gauss = s.kind == SLSE_GAUSSIAN;
  if (L.gauss) {
    L.gp = gauss_plan(p->N, d, s.prec, s.r, false, nsm);
    if (L.gp.total > big) big = L.gp.total;
  }
  // correction form of the mixed 2nd stage: the packed BF16 copy of X and the partial sums of its
  // Gram matrix take the big region, whose SRHT, CountSketch or Gaussian temporaries are dead by then
  L.host_in = is_host_pointer(p->X);
  L.dc = s.prec != SLSE_PREC_FP64 && s.stage2 == SLSE_STAGE2_CORRECTION;
  // with a two-pass SRHT, G_b is formed from the pass-1 intermediate W (BF16, kept until the 2nd
  // stage) instead of X: its partial sums follow W in the big region
  L.gw = L.dc && !L.cs && !L.gauss && !L.sp.single && L.n_samp > 0;
  if (L.gw) {
    L.gwp = gram_w_plan(L.Np, d, nsm);
    L.o_gpart = align256(wbytes) + align256(wybytes);
    if (L.o_gpart + L.gwp.part_bytes > big) big = L.o_gpart + L.gwp.part_bytes;
  } else if (L.dc) {
    L.grp = gram_plan(p->N, d, nsm);
    if (L.grp.total > big) big = L.grp.total;
  }
  L.o_big = w.take(big);
  L.o_wy = L.o_big + align256(wbytes);
  L.o_u = w.take((size_t)L.n_samp * L.ldu * eu);
  L.o_v = w.take((size_t)L.n_samp * ev);
  L.o_us = w.take(fp8 ? (size_t)L.n_samp * L.nsb : 0);
  L.o_hat16 = w.take((fp8 || (L.gauss && s.prec != SLSE_PREC_FP64)) ? (size_t)s.r * L.ld16 * 2 : 0);
  L.o_A = w.take((size_t)s.r * d * 8);
  L.o_R = w.take((size_t)d * d * 8);
  L.o_Hinv = w.take((size_t)d * d * 8);
  L.o_qr = w.take(qr_ws_bytes(s.r, d, nsm > 0 ? nsm : 152));
  L.o_chol = w.take(s.prec != SLSE_PREC_FP64 ? sweep_ws_bytes(s.r, d) : 0);
  L.o_part = w.take((size_t)L.nblk * d * 8);
  L.o_g = w.take((size_t)d * 8);
  L.o_ring = w.take((size_t)3 * d * 8);
  L.o_b0 = w.take((size_t)d * 8);
  L.o_d32 = w.take((size_t)d * 4);
  L.o_out = w.take((size_t)d * 8);
  L.o_r0 = w.take(s.prec != SLSE_PREC_FP64 ? (size_t)p->N * 4 : 0);
  L.o_g0 = w.take(L.dc ? (size_t)d * 8 : 0);
  L.o_be = w.take(L.dc ? (size_t)d * 8 : 0);
  L.o_de = w.take(L.dc ? (size_t)d * 4 : 0);
  L.o_gb = w.take(L.dc ? (size_t)d * d * 8 : 0);
  L.o_gst = w.take(L.dc ? 256 : 0);  // status word of the Gram build (it runs beside the 1st stage)
  if (L.host_in) {
    const size_t bx = p->dtype == SLSE_F64 ? 8 : 4;
    L.o_xin = w.take((size_t)p->N * d * bx);
    L.o_yin = w.take((size_t)p->N * bx);
  }
  L.total = w.total;
  return L;
}

struct SketchLayout {
  int64_t Np, ldw;
  SrhtPlan sp;
  size_t o_psd, o_sigma, o_pos, o_big, o_wy, total;
};

SketchLayout sketch_layout(const slse_problem *p, int prec, int64_t m) {
  SketchLayout L{};
  L.Np = padded(p->N);
  L.sp = srht_plan(L.Np);
  L.ldw = (p->d + 7) & ~int64_t(7);
  const size_t eu = elem_bytes_w(prec);
  Layout w;
  L.o_psd = w.take(4 * (size_t)L.Np);
  L.o_sigma = w.take(4 * (size_t)L.Np);
  L.o_pos = w.take(4 * (size_t)L.Np);
  size_t big = draws_ws_bytes(L.Np);
  const size_t wbytes = L.sp.single ? 0 : (size_t)L.Np * L.ldw * eu;
  const size_t wybytes = L.sp.single ? 0 : (size_t)L.Np * eu;
  if (align256(wbytes) + align256(wybytes) > big) big = align256(wbytes) + align256(wybytes);
  // FP8 form at single-pass sizes: BF16 rows first, then quantised
  if (prec == SLSE_PREC_MIXED_FP8 && L.sp.single && (size_t)m * L.ldw * 2 > big) big = (size_t)m * L.ldw * 2;
  L.o_big = w.take(big);
  L.o_wy = L.o_big + align256(wbytes);
  L.total = w.total;
  return L;
}

size_t grad_ws(const slse_problem *p, int nsm) {
  Layout w;
  w.take(kStateBytes);
  w.take((size_t)2 * (nsm > 0 ? nsm : 152) * p->d * 8);
  return w.total;
}

// ------------------------------------------------------------------ helpers
__global__ void k_init_state(DevState *st, int rebase, long long spin_limit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    DevState z = {};
    z.rebase = rebase;
    z.spin_limit = spin_limit;
    *st = z;
  }
}
// Clears the non-positive-pivot flag of the Gram-sweep route before the QR fallback; any
// other status bit (a timeout) is kept for the final report.
__global__ void k_clear_numeric(DevState *st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->status &= ~ST_NUMERIC;
}
__global__ void k_or_status(DevState *st, const unsigned *side_status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->status |= *side_status;
}

__global__ void k_set_stage2(DevState *st, int rebase, int dc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->rebase = rebase;
    st->done = 0;
    st->dc = dc;
    st->bfnext = 0;
    st->dc_fell_back = 0;
    st->step_ref = 0.0;
    st->step_prev = 0.0;
    st->ninner = 0;
  }
}

struct Workspace {
  void *ptr = nullptr;
  bool owned = false;
  cudaStream_t s = nullptr;
  ~Workspace() {
    if (owned && ptr) cudaFreeAsync(ptr, s);
  }
};

slse_status acquire(Workspace &w, void *user, size_t user_bytes, size_t need, cudaStream_t s) {
  w.s = s;
  if (user) {
    if (user_bytes < need) return SLSE_ENOMEM;
    if (reinterpret_cast<uintptr_t>(user) % 256 != 0) return SLSE_EINVAL;
    w.ptr = user;
    return SLSE_OK;
  }
  if (cudaMallocAsync(&w.ptr, need, s) != cudaSuccess) {
    cudaGetLastError();
    w.ptr = nullptr;
    return SLSE_ENOMEM;
  }
  w.owned = true;
  return SLSE_OK;
}

// NVTX range for the phase of slse_fit being enqueued (draws, sketch, Hessian factor, stage 1,
// stage 2); the range in flight is closed on every exit path.
struct NvtxPhase {
  bool open = false;
  void set(const char *name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~NvtxPhase() {
    if (open) nvtxRangePop();
  }
};

struct Events {
  std::vector<cudaEvent_t> ev;
  cudaEvent_t make() {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ev.push_back(e);
    return e;
  }
  ~Events() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

// Pinned host mailbox for the stage-2 stop flag (one per host thread).
struct Mailbox {
  DevState *h = nullptr;
  ~Mailbox() {
    if (h) cudaFreeHost(h);
  }
  DevState *get() {
    if (!h && cudaHostAlloc((void **)&h, 4 * sizeof(DevState), cudaHostAllocDefault) != cudaSuccess) h = nullptr;
    return h;
  }
};
thread_local Mailbox t_mailbox;

float ms_between(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (a && b && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    ms = 0.f;
  }
  return ms;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      if (getenv("SLSE_LOG"))                      \
        fprintf(stderr, "slse: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return SLSE_ECUDA;                           \
    }                                              \
  } while (0)

slse_status status_from_bits(unsigned bits) {
  if (bits & ST_TIMEOUT) return SLSE_ETIMEOUT;
  if (bits & ST_NUMERIC) return SLSE_ENUMERIC;
  if (bits & ST_NOTCONV) return SLSE_ENOTCONV;
  return SLSE_OK;
}

int grad_blocks(int64_t rows, int maxblk) {
  int64_t b = (rows + 31) / 32;
  if (b > maxblk) b = maxblk;
  if (b < 1) b = 1;
  return (int)b;
}

slse_status fit_impl(const slse_problem *pin, const Sched &s, uint64_t seed, double *beta_out, slse_report *rep,
                     slse_trace *tr, void *ws_user, size_t ws_bytes, cudaStream_t st) {
  const int nsm = num_sms();
  if (nsm <= 0) return SLSE_ECUDA;
  const FitLayout L = fit_layout(pin, s, nsm);
  if (is_host_pointer(pin->Y) != L.host_in) return SLSE_EINVAL;  // X and Y in the same kind of memory
  Workspace W;
  slse_status a = acquire(W, ws_user, ws_bytes, L.total, st);
  if (a != SLSE_OK) return a;
  char *base = static_cast<char *>(W.ptr);
  slse_problem prob = *pin;  // device view of the inputs
  const slse_problem *p = &prob;
  DevState *dst = reinterpret_cast<DevState *>(base + L.o_state);
  int32_t *Psd = reinterpret_cast<int32_t *>(base + L.o_psd);
  int32_t *sigma = reinterpret_cast<int32_t *>(base + L.o_sigma);
  int32_t *pos = reinterpret_cast<int32_t *>(base + L.o_pos);
  void *big = base + L.o_big;
  void *WY = base + L.o_wy;
  void *U = base + L.o_u;
  void *V = base + L.o_v;
  double *A = reinterpret_cast<double *>(base + L.o_A);
  double *R = reinterpret_cast<double *>(base + L.o_R);
  double *Hinv = reinterpret_cast<double *>(base + L.o_Hinv);
  void *qrws = base + L.o_qr;
  double *part = reinterpret_cast<double *>(base + L.o_part);
  double *g = reinterpret_cast<double *>(base + L.o_g);
  double *ring = reinterpret_cast<double *>(base + L.o_ring);
  double *b0 = reinterpret_cast<double *>(base + L.o_b0);
  float *d32 = reinterpret_cast<float *>(base + L.o_d32);
  double *outb = reinterpret_cast<double *>(base + L.o_out);
  float *r0 = s.prec != SLSE_PREC_FP64 ? reinterpret_cast<float *>(base + L.o_r0) : nullptr;
  const int d = p->d;
  const bool mixed = s.prec != SLSE_PREC_FP64;     // BF16 or FP8 sketch, FP32 2nd-stage passes
  const bool fp8 = s.prec == SLSE_PREC_MIXED_FP8;
  uint8_t *Us = fp8 ? reinterpret_cast<uint8_t *>(base + L.o_us) : nullptr;
  const int T = s.T;
  int kernels = 0;

  Events E;
  cudaEvent_t e_start = E.make(), e_draws = E.make(), e_mid = E.make(), e_sketch = E.make(), e_qr = E.make(),
              e_s1 = E.make(), e_end = E.make(), e_copied = E.make(), e_sig = E.make();
  if (!e_start || !e_end || !e_mid || !e_copied || !e_sig) return SLSE_ECUDA;
  const int hist_cap = tr ? (tr->cap < T ? tr->cap : T) : 0;
  std::vector<cudaEvent_t> e_it;
  if (tr && tr->ms_hist)
    for (int t = 0; t < hist_cap; ++t) {
      cudaEvent_t e = E.make();
      if (!e) return SLSE_ECUDA;
      e_it.push_back(e);
    }
  auto mark_iter = [&](int t) -> cudaError_t {
    if (t < (int)e_it.size()) return cudaEventRecord(e_it[t], st);
    return cudaSuccess;
  };

  NvtxPhase phase;
  phase.set("slse_fit: draws");
  CK(cudaEventRecord(e_start, st));
  // host inputs: Y (and X, unless pass 1 reads it) is copied into the workspace on a side
  // stream, overlapped with the draws.  Pinned X with contiguous rows on a two-pass SRHT plan
  // is instead read by SRHT pass 1 straight from host memory (every row is gathered exactly
  // once there), and that pass also stores each row segment into the workspace copy: the
  // transfer over the host link and the pass are one step instead of two.
  struct SideStream {
    cudaStream_t h = nullptr;
    ~SideStream() {
      if (h) cudaStreamDestroy(h);
    }
  } side;
  // the stream of the sigma draws; the caller's stream waits for it on every return (pass 2
  // waits for it anyway), so no work of the fit outlives the call's stream order
  struct JoinedStream {
    cudaStream_t h = nullptr, main = nullptr;
    ~JoinedStream() {
      if (!h) return;
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(e, h);
        cudaStreamWaitEvent(main, e, 0);
        cudaEventDestroy(e);
      }
      cudaStreamDestroy(h);
    }
  } sig_side;
  sig_side.main = st;
  const void *x_mapped = nullptr;  // device address of host X read by pass 1 (fused path)
  void *x_copy = nullptr;          // where pass 1 stores it
  if (L.host_in) {
    const size_t bx = p->dtype == SLSE_F64 ? 8 : 4;
    void *xd = base + L.o_xin;
    void *yd = base + L.o_yin;
    if (!L.cs && L.n_samp > 0 && !L.sp.single && pin->ldx == d) {
      cudaPointerAttributes at;
      void *dp = nullptr;
      if (cudaPointerGetAttributes(&at, pin->X) == cudaSuccess && at.type == cudaMemoryTypeHost &&
          cudaHostGetDevicePointer(&dp, const_cast<void *>(pin->X), 0) == cudaSuccess && dp) {
        x_mapped = dp;
        x_copy = xd;
      }
      cudaGetLastError();
    }
    CK(cudaStreamCreateWithFlags(&side.h, cudaStreamNonBlocking));
    CK(cudaStreamWaitEvent(side.h, e_start, 0));
    if (x_mapped) {
      // X arrives through pass 1
    } else if (pin->ldx == d) {  // contiguous rows: one linear copy (a pitched copy splits it per row)
      CK(cudaMemcpyAsync(xd, pin->X, (size_t)p->N * d * bx, cudaMemcpyHostToDevice, side.h));
    } else {
      CK(cudaMemcpy2DAsync(xd, (size_t)d * bx, pin->X, (size_t)pin->ldx * bx, (size_t)d * bx, (size_t)p->N,
                           cudaMemcpyHostToDevice, side.h));
    }
    CK(cudaMemcpyAsync(yd, pin->Y, (size_t)p->N * bx, cudaMemcpyHostToDevice, side.h));
    CK(cudaEventRecord(e_copied, side.h));
    prob.X = xd;
    prob.Y = yd;
    prob.ldx = d;
  }
  k_init_state<<<1, 32, 0, st>>>(dst, 0, debug_spin_limit());
  CK(cudaGetLastError());
  ++kernels;
  const size_t eu = elem_bytes_u(s.prec);
  if (L.cs) {
    // CountSketch family (Sec. 2; SLSE-FRS-CS of Sec. 5): its hashes are drawn inside the
    // one sort-and-gather pass, so the draws phase is empty.
    CK(cudaEventRecord(e_draws, st));
    phase.set("slse_fit: sketch");
    if (L.host_in) CK(cudaStreamWaitEvent(st, e_copied, 0));
    void *lvX[25] = {}, *lvY[25] = {};
    for (size_t i = 0; i < s.m.size(); ++i) {
      int l = 0;
      while ((int64_t(1) << l) < s.m[i]) ++l;
      lvX[l] = static_cast<char *>(U) + (size_t)L.lvl_off[i] * L.ldu * eu;
      lvY[l] = static_cast<char *>(V) + (size_t)L.lvl_off[i] * eu;
    }
    CK(launch_countsketch(L.csp, p->dtype, p->X, p->ldx, p->Y, seed, lvX, lvY, L.ldu,
                          static_cast<char *>(U) + (size_t)L.h0 * L.ldu * eu, static_cast<char *>(V) + (size_t)L.h0 * eu,
                          L.ldu, big, st));
    kernels += 12;
    CK(cudaEventRecord(e_mid, st));
  } else {
    // a1: random draws (none when nothing is sampled: a Gaussian Hessian sketch without subproblems)
    if (L.sig_side) {
      // pass 1 needs only P: sigma and its position map (read from pass 2 on) are drawn after P
      // on a side stream of the lowest priority, beside pass 1 (a latency-bound pass), and pass 2
      // waits for them.  Measured at N' = 2^22: draws 0.57 -> 0.32 ms, pass 1 unchanged (3.49 ms);
      // at the highest priority the sort's CTAs displaced pass 1's clusters (pass 1 4.59 ms)
      CK(launch_draws_perm(L.Np, seed, Psd, big, st));
      CK(cudaEventRecord(e_draws, st));
      int least = 0, greatest = 0;
      CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      CK(cudaStreamCreateWithPriority(&sig_side.h, cudaStreamNonBlocking, least));
      CK(cudaStreamWaitEvent(sig_side.h, e_draws, 0));
      CK(launch_draws_sigma(L.Np, seed, sigma, base + L.o_sigws, sig_side.h));
      CK(launch_pos_map(sigma, L.Np, 0, L.n_samp, L.sp.log2, pos, sig_side.h));
      CK(cudaEventRecord(e_sig, sig_side.h));
      kernels += 10;
    } else {
      if (L.n_samp > 0) {
        CK(launch_draws(L.Np, seed, Psd, nullptr, sigma, nullptr, big, st));
        kernels += 5;  // histogram, scan, scatter, bucket sort (both permutations each), sign fold
        CK(launch_pos_map(sigma, L.Np, 0, L.n_samp, L.sp.single ? L.sp.logN : L.sp.log2, pos, st));
        kernels += 1;
      }
      CK(cudaEventRecord(e_draws, st));
    }
    phase.set("slse_fit: sketch");
    if (L.host_in) CK(cudaStreamWaitEvent(st, e_copied, 0));
    // a2-a4: SRHT into the sampled rows (U = Z[sigma] with Z = H D P X / sqrt(N'); sketch scales applied later)
    __nv_bfloat16 *h16 = fp8 ? reinterpret_cast<__nv_bfloat16 *>(base + L.o_hat16) : nullptr;
    if (L.n_samp == 0) {
      CK(cudaEventRecord(e_mid, st));
    } else if (fp8 && L.sp.single) {  // one-pass sizes: BF16 rows, then the FP8 form (S-hat rows stay BF16)
      CK(launch_srht(L.sp, SLSE_PREC_MIXED_BF16, p->dtype, p->X, p->ldx, p->Y, p->N, d, Psd, pos, nullptr, nullptr,
                     L.ld16, big, V, L.ld16, 1.0 / std::sqrt((double)L.Np), st, nullptr));
      CK(launch_quantize_mx(static_cast<const __nv_bfloat16 *>(big), L.ld16, L.n_samp, d, static_cast<uint8_t *>(U),
                            L.ldu, Us, L.nsb, st));
      CK(cudaMemcpyAsync(h16, static_cast<const __nv_bfloat16 *>(big) + (size_t)L.h0 * L.ld16,
                         (size_t)s.r * L.ld16 * 2, cudaMemcpyDeviceToDevice, st));
      kernels += 2;
    } else {
      // FP8 form: the Hessian-sketch rows (sampling positions >= h0) are written in BF16 to h16
      CK(launch_srht(L.sp, s.prec, p->dtype, x_mapped ? x_mapped : p->X, p->ldx, p->Y, p->N, d, Psd, pos, big, WY,
                     L.ld16, U, V, L.ldu, 1.0 / std::sqrt((double)L.Np), st, L.sp.single ? nullptr : e_mid, Us, L.nsb,
                     h16, L.h0 > 0 ? L.h0 : INT64_MAX, L.ld16, x_copy, &dst->status,
                     L.sig_side ? e_sig : nullptr));
      kernels += L.sp.single ? 1 : 4;  // per pass: the X columns and the Y column
    }
    if (L.gauss) {
      // S-hat X = G X / sqrt(r) (Gaussian sketch, Sec. 2) in place of sampled SRHT rows:
      // BF16 rows for the Gram-sweep route, FP64 rows straight into the QR input
      void *hout = mixed ? static_cast<void *>(base + L.o_hat16) : static_cast<void *>(A);
      const int64_t ldo = mixed ? L.ld16 : d;
      if (mixed) CK(cudaMemsetAsync(hout, 0, (size_t)s.r * L.ld16 * 2, st));
      CK(launch_gaussian(L.gp, p->dtype, p->X, p->ldx, p->Y, seed, hout, ldo, nullptr, 1.0 / std::sqrt((double)s.r),
                         &dst->status, big, st));
      kernels += mixed ? 3 * L.gp.groups : 2;
    }
  }
  CK(cudaEventRecord(e_sketch, st));
  // correction form: the Gram matrix G_b of the BF16 copy of X needs only X and the big region
  // (free once the sketch is formed), so it is formed on a second stream beside the Hessian factor
  // and the 1st stage (memory- and latency-bound work beside a tensor-core product); the 2nd stage
  // waits for it
  struct GramStream {
    cudaStream_t h = nullptr, main = nullptr;
    ~GramStream() {
      if (!h) return;
      // the caller's stream (on which a library-owned workspace is freed) waits for this one,
      // also on an early return between the fork and the join
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(e, h);
        cudaStreamWaitEvent(main, e, 0);
        cudaEventDestroy(e);
      }
      cudaStreamDestroy(h);
    }
  } gram_side;
  gram_side.main = st;
  double *Gb = L.dc ? reinterpret_cast<double *>(base + L.o_gb) : nullptr;
  unsigned *gram_status = L.dc ? reinterpret_cast<unsigned *>(base + L.o_gst) : nullptr;
  cudaEvent_t e_gram0 = nullptr, e_gram1 = nullptr;
  if (L.dc && s.T > 0) {
    e_gram0 = E.make();
    e_gram1 = E.make();
    if (!e_gram0 || !e_gram1) return SLSE_ECUDA;
    CK(cudaStreamCreateWithFlags(&gram_side.h, cudaStreamNonBlocking));
  }
  // The build is forked once the Hessian factor is formed: beside pass 2 (which also reads W) it
  // slowed the pass by half, and beside the Hessian factor's chain of short kernels it tripled the
  // factor's time; beside the 1st stage and the first exact pass it costs least.  (From X, its
  // workspace reuses the sketch's temporaries.)
  auto fork_gram = [&](cudaEvent_t after) -> cudaError_t {
    if (!gram_side.h) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaStreamWaitEvent(gram_side.h, after, 0))) return e;
    if ((e = cudaMemsetAsync(gram_status, 0, sizeof(unsigned), gram_side.h))) return e;
    if ((e = cudaEventRecord(e_gram0, gram_side.h))) return e;
    if (L.gw) {
      const double n2 = (double)(int64_t(1) << L.sp.log2);
      e = launch_gram_w(L.gwp, big, L.ld16, 1.0 / n2, Gb, gram_status,
                        reinterpret_cast<float *>(static_cast<char *>(big) + L.o_gpart), gram_side.h);
      kernels += 3;  // Gram, group sums, final sum
    } else {
      e = launch_gram(L.grp, static_cast<const float *>(p->X), p->ldx, Gb, gram_status, big, gram_side.h);
      kernels += gram_fp32_path(L.grp, static_cast<const float *>(p->X), p->ldx) ? 2 : 3;  // (pack,) Gram, reduce
    }
    if (e) return e;
    return cudaEventRecord(e_gram1, gram_side.h);
  };
  // With the Gram build beside it, the main path (Hessian factor, stages 1 and 2) runs on an
  // internal stream of the highest priority: the build's grid is larger than the GPU, and without
  // priority its pending CTAs were dispatched first, so the short kernels of the Hessian factor
  // waited for most of the build (0.86 ms became 4.3 ms).  The caller's stream joins it after the
  // 2nd stage (and waits for it on every return).
  struct PrioStream {
    cudaStream_t h = nullptr, user = nullptr;
    ~PrioStream() {
      if (!h) return;
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(e, h);
        cudaStreamWaitEvent(user, e, 0);
        cudaEventDestroy(e);
      }
      cudaStreamDestroy(h);
    }
  } prio;
  prio.user = st;
  const cudaStream_t user_st = st;
  if (gram_side.h) {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&prio.h, cudaStreamNonBlocking, greatest));
    CK(cudaStreamWaitEvent(prio.h, e_sketch, 0));
    st = prio.h;
  }
  phase.set("slse_fit: Hessian factor");
  // sketch scales: SRHT S_i X = sqrt(N'/m_i) U[rows], S-hat X = sqrt(N'/r) U[h0 ..]; CountSketch: 1
  auto sq_scale = [&](int64_t m) { return L.cs ? 1.0 : (double)L.Np / (double)m; };
  // a5: H-hat^{-1} = R^{-1} R^{-T} for the R of S-hat X = sqrt(N'/r) U[h0 : h0 + r].  FP64 path:
  // Householder QR, then R^{-1} and H-hat^{-1}.  Mixed path: the same matrix as the inverse of
  // the exactly accumulated Gram matrix R^T R of the BF16 rows, by the blocked sweep operator
  // in FP64, with the Householder QR as fallback on a non-positive pivot.
  bool use_qr = !mixed;
  // the Hessian-sketch rows as BF16 (the FP8 form is widened exactly)
  const void *Uh = U;
  int64_t ldh = L.ldu, h0 = L.h0;
  double hat_scale2 = sq_scale(s.r);
  if (L.gauss) {
    hat_scale2 = 1.0;  // rows already scaled by 1/sqrt(r)
    if (mixed) { Uh = base + L.o_hat16; ldh = L.ld16; h0 = 0; }
  }
  if (fp8) {
    __nv_bfloat16 *h16 = reinterpret_cast<__nv_bfloat16 *>(base + L.o_hat16);
    if (L.h0 == 0 && !L.sp.single) {  // S-hat shares the prefix rows (m_K + r > N'): widen them
      CK(launch_mx_to_bf16(static_cast<const uint8_t *>(U), L.ldu, Us, L.nsb, s.r, d, h16, L.ld16, st));
      ++kernels;
    }
    Uh = h16; ldh = L.ld16; h0 = 0;
  }
  if (mixed) {
    CK(launch_gram_sweep(Uh, ldh, h0, s.r, d, hat_scale2, Hinv, base + L.o_chol, dst, st));
    const int nb = (d + 31) / 32;
    kernels += 3 + 2 * nb;
    DevState *mb = t_mailbox.get();
    if (!mb) return SLSE_ECUDA;
    CK(cudaMemcpyAsync(&mb[3], dst, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (((volatile DevState *)&mb[3])->status & ST_NUMERIC) {
      k_clear_numeric<<<1, 32, 0, st>>>(dst);
      CK(cudaGetLastError());
      ++kernels;
      use_qr = true;
    }
  }
  if (use_qr) {
    if (!(L.gauss && !mixed)) {  // the FP64 Gaussian rows are already in A
      CK(launch_gather_hessian_rows((fp8 || L.gauss) ? SLSE_PREC_MIXED_BF16 : s.prec, Uh, ldh, h0, s.r, d,
                                    std::sqrt(hat_scale2), A, st));
      ++kernels;
    }
    CK(launch_qr(A, s.r, d, d, R, Hinv, qrws, dst, st));
    kernels += 3;
  }
  CK(cudaEventRecord(e_qr, st));
  CK(fork_gram(e_qr));
  phase.set("slse_fit: stage 1");
  if (tr && tr->hinv_out)
    CK(cudaMemcpyAsync(tr->hinv_out, Hinv, (size_t)d * d * 8, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(ring, 0, (size_t)3 * d * 8, st));

  UpdateArgs ua{};
  ua.g = g; ua.Hinv = Hinv; ua.beta_ring = ring; ua.beta0 = b0; ua.delta32 = d32;
  ua.hist = tr ? tr->beta_hist : nullptr; ua.hist_cap = hist_cap; ua.d = d; ua.mu = s.mu; ua.eta = s.eta;
  ua.T = T;

  // a8 stage 1: a_i M-IHS steps on each nested sketch (prefix of the sampled rows)
  int t = 0;
  for (size_t i = 0; i < s.m.size() && t < T; ++i) {
    const int64_t m = s.m[i];
    const int nb = grad_blocks(m, L.nblk);
    // SRHT: the prefix U[0:m_i]; CountSketch: the block of U holding S_i X
    const size_t r0w = L.cs ? (size_t)L.lvl_off[i] : 0;
    const void *Ui = static_cast<const char *>(U) + r0w * L.ldu * eu;
    const void *Vi = static_cast<const char *>(V) + r0w * (fp8 ? 2 : eu);
    for (int j = 0; j < s.a[i] && t < T; ++j) {
      if (fp8)
        CK(launch_grad_mx(static_cast<const uint8_t *>(Ui), L.ldu, Us + r0w * L.nsb, L.nsb,
                          static_cast<const __nv_bfloat16 *>(Vi), m, d, ring, dst, part, nb, st));
      else
        CK(launch_grad(mixed ? GM_STAGE1_BF16 : GM_STAGE1_F64, mixed ? SLSE_BF16 : SLSE_F64, Ui, L.ldu, Vi, m, d,
                       ring, dst, nullptr, nullptr, nullptr, part, nb, 0, st));
      CK(launch_reduce(part, nb, d, sq_scale(m), g, dst, 0, st));
      ua.first = (j == 0 && s.momentum_reset) || t == 0;
      ua.stage2 = 0; ua.thr = 0.0; ua.mixed = 0; ua.check_done = 0;
      CK(launch_update(ua, dst, st));
      kernels += 3;
      CK(mark_iter(t));
      ++t;
    }
  }
  const int t1 = t;
  CK(cudaEventRecord(e_s1, st));
  phase.set("slse_fit: stage 2");
  // a8 stage 2: full-data M-IHS steps until the relative step is small or T is reached.
  // Iteration k+1 is enqueued before the stop flag of iteration k is read back; its
  // kernels return at once when the flag is already set.
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> e_grad;
  // correction form: the Gram matrix G_b of the BF16 copy of X (formed once, here), g(beta_e)
  // beside the gradient, the iterate beta_e of the last exact pass and fl32(beta - beta_e)
  double *g0 = L.dc ? reinterpret_cast<double *>(base + L.o_g0) : nullptr;
  float *de = L.dc ? reinterpret_cast<float *>(base + L.o_de) : nullptr;
  ua.hist_base = t;
  ua.beta_e = L.dc ? reinterpret_cast<double *>(base + L.o_be) : nullptr;
  ua.delta_e = de;
  // a correction step (a d x d product and the update) costs a small fraction of a pass over X
  ua.inner_cost = 0.02;
  // G_b is first read by the 2nd stage's second step (its first pass is exact), so the main stream
  // waits for the side stream only there: the Gram build also overlaps that pass.  The wait is
  // enqueued before the call's last synchronisation in every case.
  bool gram_joined = e_gram1 == nullptr;
  auto join_gram = [&]() -> cudaError_t {
    if (gram_joined) return cudaSuccess;
    gram_joined = true;
    cudaError_t e = cudaStreamWaitEvent(st, e_gram1, 0);
    if (e != cudaSuccess) return e;
    k_or_status<<<1, 32, 0, st>>>(dst, gram_status);  // a timeout of the Gram build
    ++kernels;
    return cudaGetLastError();
  };
  if (t < T) {
    k_set_stage2<<<1, 32, 0, st>>>(dst, mixed ? 1 : 0, L.dc ? 1 : 0);
    CK(cudaGetLastError());
    ++kernels;
    DevState *mb = t_mailbox.get();
    if (!mb) return SLSE_ECUDA;
    const double rho = std::sqrt((double)d / (double)s.r);
    const double thr = s.tol > 0.0 ? s.tol * (1.0 - rho) / rho : 0.0;
    ua.rho = rho;
    const int nb = L.nblk;
    cudaEvent_t e_flag[2] = {E.make(), E.make()};
    if (!e_flag[0] || !e_flag[1]) return SLSE_ECUDA;
    for (int k = 0; t + k < T; ++k) {
      cudaEvent_t g0e = E.make(), g1 = E.make();
      if (!g0e || !g1) return SLSE_ECUDA;
      if (k == 1) CK(join_gram());
      CK(cudaEventRecord(g0e, st));
      // correction form: a pass over X (exact) or a correction step g = g(beta_e) - G_b (beta - beta_e),
      // as the device state selects; the kernels of the other kind return at once
      CK(launch_grad(mixed ? GM_MIXED : GM_F64, p->dtype, p->X, p->ldx, p->Y, p->N, d, ring, dst, d32, r0, b0,
                     part, nb, 1, st));
      if (L.dc) CK(launch_gram_step(Gb, de, g0, g, d, dst, st));
      CK(cudaEventRecord(g1, st));
      e_grad.emplace_back(g0e, g1);
      CK(launch_reduce(part, nb, d, 1.0, g, dst, 1, st, g0));
      ua.first = (k == 0 && s.momentum_reset) || (t + k) == 0;
      ua.stage2 = 1; ua.thr = thr; ua.mixed = mixed ? 1 : 0; ua.check_done = 1;
      CK(launch_update(ua, dst, st));
      kernels += L.dc ? 5 : (mixed ? 4 : 3);
      CK(mark_iter(t + k));
      CK(cudaMemcpyAsync(&mb[k & 1], dst, sizeof(DevState), cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(e_flag[k & 1], st));
      if (k > 0) {
        CK(cudaEventSynchronize(e_flag[(k - 1) & 1]));
        if (((volatile DevState *)&mb[(k - 1) & 1])->done) break;
      }
    }
  }
  CK(join_gram());
  if (prio.h) {  // back to the caller's stream
    cudaEvent_t e_back = E.make();
    if (!e_back) return SLSE_ECUDA;
    CK(cudaEventRecord(e_back, st));
    CK(cudaStreamWaitEvent(user_st, e_back, 0));
    st = user_st;
  }
  CK(launch_copy_beta(ring, dst, d, outb, st));
  ++kernels;
  DevState *mb = t_mailbox.get();
  if (!mb) return SLSE_ECUDA;
  CK(cudaMemcpyAsync(&mb[2], dst, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(e_end, st));
  CK(cudaMemcpyAsync(beta_out, outb, (size_t)d * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const DevState fin = mb[2];
  slse_status status = status_from_bits(fin.status);
  // the report (also formed for the SLSE_LOG trace when the caller passed none)
  slse_report local_rep{};
  const bool log = getenv("SLSE_LOG") != nullptr;
  slse_report *RP = rep ? rep : (log ? &local_rep : nullptr);
  if (RP) {
    RP->ms_copy_in = L.host_in ? ms_between(e_start, e_copied) : 0.0;
    RP->ms_draws = ms_between(e_start, e_draws);
    RP->ms_sketch = ms_between(e_draws, e_sketch);
    RP->ms_srht_pass1 = (L.sp.single || L.cs) ? RP->ms_sketch : ms_between(e_draws, e_mid);
    RP->ms_srht_pass2 = (L.sp.single || L.cs) ? 0.0 : ms_between(e_mid, e_sketch);
    RP->ms_qr = ms_between(e_sketch, e_qr);
    RP->ms_stage1 = ms_between(e_qr, e_s1);
    RP->ms_total = ms_between(e_start, e_end);
    RP->ms_stage2 = RP->ms_total - ms_between(e_start, e_s1);
    // gradient launches that ran a full pass (the speculative one after the stop returns at once),
    // split by pass kind: over X (exact or full form) or over its BF16 copy (correction form)
    const int full = fin.iter - t1;
    double mg = 0.0, mb16 = 0.0;
    int nx = 0, nb16 = 0;
    for (int k = 0; k < full && k < (int)e_grad.size(); ++k) {
      const double ms = ms_between(e_grad[k].first, e_grad[k].second);
      if (k < (int)sizeof(fin.mode_hist) && fin.mode_hist[k] == 1) {
        mb16 += ms;
        ++nb16;
      } else {
        mg += ms;
        ++nx;
      }
    }
    RP->ms_grad2 = mg;
    RP->n_grad2 = nx;
    RP->ms_corr = mb16;
    RP->n_corr = nb16;
    RP->stage2_full = fin.dc_fell_back;
    if (L.dc && e_gram0) {
      RP->ms_gram = ms_between(e_gram0, e_gram1);
      if (L.gw) {
        RP->flops_gram = L.gwp.flops;
        RP->bytes_gram = L.gwp.bytes;
      } else {
        const bool f32 = gram_fp32_path(L.grp, static_cast<const float *>(p->X), p->ldx);
        RP->flops_gram = f32 ? L.grp.flops_f32 : L.grp.flops_packed;
        RP->bytes_gram = f32 ? L.grp.bytes_f32 : L.grp.bytes_packed;
      }
    }
    RP->kernels = kernels;
    RP->iters_stage1 = t1;
    RP->iters_stage2 = fin.iter - t1;
    RP->final_rel_step = fin.rel_step;
    RP->rebases = fin.rebases;
    const double bx = p->dtype == SLSE_F64 ? 8.0 : 4.0, bu = (double)elem_bytes_u(s.prec);
    double bytes = 0.0;
    if (L.cs) bytes += 2.0 * (double)p->N * (d + 1) * bx + (double)L.n_samp * (d + 1) * bu;  // nested and S-hat passes
    else if (L.sp.single) bytes += (double)p->N * (d + 1) * bx + (double)L.n_samp * (d + 1) * bu;
    else bytes += (double)p->N * (d + 1) * bx + 2.0 * (double)L.Np * (d + 1) * bu + (double)L.n_samp * (d + 1) * bu;
    // Gaussian Hessian sketch: one read of X (and, mixed, the packed BF16 copy written and read)
    if (L.gauss) bytes += (double)p->N * d * bx + (mixed ? 2.0 * (double)p->N * L.gp.ncp * 2.0 : 0.0);
    for (size_t i = 0; i < s.m.size(); ++i) bytes += (double)s.a[i] * (double)s.m[i] * (d + 1) * bu;
    // a 2nd-stage pass reads X and one N-vector (Y in FP64 / rebase passes, r0 otherwise)
    RP->bytes_grad2 = (double)p->N * d * bx + (double)p->N * (mixed ? 4.0 : bx);
    bytes += (double)nx * RP->bytes_grad2 + RP->bytes_gram;
    RP->bytes_moved = bytes;
    RP->status = status;
  }
  if (log && RP)
    fprintf(stderr,
            "slse_fit: N=%lld d=%d kind=%d prec=%d status=%d | draws %.3f ms, sketch %.3f ms (pass 1 %.3f, pass 2 "
            "%.3f), Hessian factor %.3f ms, stage 1 %.3f ms (%d its), stage 2 %.3f ms (%d its, %d full passes, "
            "%.3f ms in gradients, %d correction steps), total %.3f ms, %d kernels\n",
            (long long)p->N, d, s.kind, s.prec, (int)status, RP->ms_draws, RP->ms_sketch, RP->ms_srht_pass1,
            RP->ms_srht_pass2, RP->ms_qr, RP->ms_stage1, RP->iters_stage1, RP->ms_stage2, RP->iters_stage2, RP->n_grad2,
            RP->ms_grad2, RP->n_corr, RP->ms_total, RP->kernels);
  if (tr) {
    tr->count = fin.iter < hist_cap ? fin.iter : hist_cap;
    if (tr->ms_hist)
      for (int k = 0; k < tr->count && k < (int)e_it.size(); ++k) tr->ms_hist[k] = ms_between(e_start, e_it[k]);
  }
  return status;
}

}  // namespace

extern "C" {

size_t slse_workspace_size(const slse_problem *prob, const slse_schedule *sched, int32_t op, int64_t arg) {
  const int nsm = num_sms() > 0 ? num_sms() : 152;
  switch (op) {
    case SLSE_OP_FIT: {
      if (!valid_problem(prob)) return 0;
      Sched s;
      if (!make_sched(prob, sched, s)) return 0;
      return fit_layout(prob, s, nsm).total;
    }
    case SLSE_OP_SKETCH: {
      if (!valid_problem(prob)) return 0;
      const int prec = sched ? sched->prec : SLSE_PREC_FP64;
      const int kind = sched ? sched->kind : SLSE_SRHT;
      if (kind == SLSE_COUNTSKETCH) return is_pow2(arg) ? cs_plan(prob->N, prob->d, prec, arg, arg, 0).total : 0;
      if (kind == SLSE_COUNTSKETCH_HAT) return arg >= 1 ? cs_plan(prob->N, prob->d, prec, 0, 0, arg).total : 0;
      if (kind == SLSE_GAUSSIAN) return arg >= 1 ? gauss_plan(prob->N, prob->d, prec, arg, true, nsm).total : 0;
      return sketch_layout(prob, prec, arg).total;
    }
    case SLSE_OP_GRAD:
      if (!valid_problem(prob)) return 0;
      return grad_ws(prob, nsm);
    case SLSE_OP_GRAM: {
      if (!valid_gram_problem(prob)) return 0;
      Layout w;
      w.take(kStateBytes);
      w.take(prob->dtype == SLSE_BF16 ? gram_w_plan(prob->N, prob->d, nsm).part_bytes
                                      : gram_plan(prob->N, prob->d, nsm).total);
      return w.total;
    }
    case SLSE_OP_DRAWS: {
      if (arg < 1 || padded(arg) > kMaxNp) return 0;
      return align256(draws_ws_bytes(padded(arg)));
    }
    case SLSE_OP_QR: {
      if (!prob || prob->d < 1 || prob->d > 512 || arg < prob->d) return 0;
      Layout w;
      w.take(kStateBytes);
      w.take((size_t)arg * prob->d * 8);
      w.take(qr_ws_bytes(arg, prob->d, nsm));
      return w.total;
    }
    default:
      return 0;
  }
}

slse_status slse_fit(const slse_problem *prob, const slse_schedule *sched, uint64_t seed, double *beta_out,
                     slse_report *report, slse_trace *trace, void *workspace, size_t ws_bytes, slse_stream_t stream) {
  if (report) std::memset(report, 0, sizeof(*report));
  if (!valid_problem(prob) || !beta_out) return SLSE_EINVAL;
  if (trace && (trace->cap < 0 || (trace->cap > 0 && !trace->beta_hist && !trace->ms_hist))) return SLSE_EINVAL;
  Sched s;
  if (!make_sched(prob, sched, s)) return SLSE_EINVAL;
  slse_status st = fit_impl(prob, s, seed, beta_out, report, trace, workspace, ws_bytes, (cudaStream_t)stream);
  if (report) report->status = st;
  return st;
}

slse_status slse_sketch(const slse_problem *prob, int32_t kind, int32_t prec, uint64_t seed, int64_t m, void *SX,
                        int64_t ldsx, void *SY, void *workspace, size_t ws_bytes, slse_stream_t stream) {
  if (!valid_problem(prob) || !SX || (!SY && kind != SLSE_GAUSSIAN)) return SLSE_EINVAL;
  if (is_host_pointer(prob->X) || is_host_pointer(prob->Y)) return SLSE_EINVAL;
  if (kind != SLSE_SRHT && kind != SLSE_COUNTSKETCH && kind != SLSE_COUNTSKETCH_HAT && kind != SLSE_GAUSSIAN)
    return SLSE_EINVAL;
  if (prec != SLSE_PREC_FP64 && prec != SLSE_PREC_MIXED_BF16 && prec != SLSE_PREC_MIXED_FP8) return SLSE_EINVAL;
  if (prec != SLSE_PREC_FP64 && prob->dtype != SLSE_F32) return SLSE_EINVAL;
  if (prec == SLSE_PREC_MIXED_FP8 && (kind != SLSE_SRHT || ldsx % 4 != 0 || reinterpret_cast<uintptr_t>(SX) % 4 != 0))
    return SLSE_EINVAL;
  const int64_t Np = padded(prob->N);
  // sampled sketches keep at most N' rows; a Gaussian sketch may have any number (row index 32-bit)
  if (m < 1 || ldsx < prob->d || m > (kind == SLSE_GAUSSIAN ? int64_t(INT32_MAX) : Np)) return SLSE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == SLSE_GAUSSIAN) {
    if (prec == SLSE_PREC_MIXED_FP8) return SLSE_EINVAL;
    const int nsm = num_sms();
    if (nsm <= 0) return SLSE_ECUDA;
    const GaussPlan gp = gauss_plan(prob->N, prob->d, prec, m, SY != nullptr, nsm);
    Workspace W;
    slse_status a = acquire(W, workspace, ws_bytes, gp.total, st);
    if (a != SLSE_OK) return a;
    unsigned *status = reinterpret_cast<unsigned *>(static_cast<char *>(W.ptr) + gp.o_status);
    CK(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
    CK(launch_gaussian(gp, prob->dtype, prob->X, prob->ldx, prob->Y, seed, SX, ldsx, SY, 1.0 / std::sqrt((double)m),
                       status, W.ptr, st));
    return SLSE_OK;
  }
  if (kind != SLSE_SRHT) {
    if (kind == SLSE_COUNTSKETCH && !is_pow2(m)) return SLSE_EINVAL;
    const bool hat = kind == SLSE_COUNTSKETCH_HAT;
    const CsPlan pl = hat ? cs_plan(prob->N, prob->d, prec, 0, 0, m) : cs_plan(prob->N, prob->d, prec, m, m, 0);
    Workspace W;
    slse_status a = acquire(W, workspace, ws_bytes, pl.total, st);
    if (a != SLSE_OK) return a;
    void *lvX[25] = {}, *lvY[25] = {};
    if (!hat) {
      lvX[pl.L] = SX;
      lvY[pl.L] = SY;
    }
    CK(launch_countsketch(pl, prob->dtype, prob->X, prob->ldx, prob->Y, seed, lvX, lvY, ldsx, hat ? SX : nullptr,
                          hat ? SY : nullptr, ldsx, W.ptr, st));
    return SLSE_OK;
  }
  const SketchLayout L = sketch_layout(prob, prec, m);
  Workspace W;
  slse_status a = acquire(W, workspace, ws_bytes, L.total, st);
  if (a != SLSE_OK) return a;
  char *base = static_cast<char *>(W.ptr);
  int32_t *Psd = reinterpret_cast<int32_t *>(base + L.o_psd);
  int32_t *sigma = reinterpret_cast<int32_t *>(base + L.o_sigma);
  int32_t *pos = reinterpret_cast<int32_t *>(base + L.o_pos);
  CK(launch_draws(Np, seed, Psd, nullptr, sigma, nullptr, base + L.o_big, st));
  CK(launch_pos_map(sigma, Np, 0, m, L.sp.single ? L.sp.logN : L.sp.log2, pos, st));
  if (prec == SLSE_PREC_MIXED_FP8) {
    // SX: m x ldsx E4M3 bytes followed by the m x ceil(d/32) block-exponent bytes
    uint8_t *scales = static_cast<uint8_t *>(SX) + (size_t)m * ldsx;
    const int64_t nsb = mx_blocks(prob->d);
    if (L.sp.single) {
      CK(launch_srht(L.sp, SLSE_PREC_MIXED_BF16, prob->dtype, prob->X, prob->ldx, prob->Y, prob->N, prob->d, Psd, pos,
                     nullptr, nullptr, L.ldw, base + L.o_big, SY, L.ldw, 1.0 / std::sqrt((double)m), st, nullptr));
      CK(launch_quantize_mx(reinterpret_cast<const __nv_bfloat16 *>(base + L.o_big), L.ldw, m, prob->d,
                            static_cast<uint8_t *>(SX), ldsx, scales, nsb, st));
    } else {
      CK(launch_srht(L.sp, prec, prob->dtype, prob->X, prob->ldx, prob->Y, prob->N, prob->d, Psd, pos, base + L.o_big,
                     base + L.o_wy, L.ldw, SX, SY, ldsx, 1.0 / std::sqrt((double)m), st, nullptr, scales, nsb));
    }
    return SLSE_OK;
  }
  CK(launch_srht(L.sp, prec, prob->dtype, prob->X, prob->ldx, prob->Y, prob->N, prob->d, Psd, pos, base + L.o_big,
                 base + L.o_wy, L.ldw, SX, SY, ldsx, 1.0 / std::sqrt((double)m), st, nullptr));
  return SLSE_OK;
}

slse_status slse_grad(const slse_problem *prob, const double *beta, double *g_out, int32_t prec, void *workspace,
                      size_t ws_bytes, slse_stream_t stream) {
  if (!valid_problem(prob) || !beta || !g_out) return SLSE_EINVAL;
  if (is_host_pointer(prob->X) || is_host_pointer(prob->Y) || is_host_pointer(beta) || is_host_pointer(g_out))
    return SLSE_EINVAL;
  if (prec != SLSE_PREC_FP64 && prec != SLSE_PREC_MIXED_BF16) return SLSE_EINVAL;
  if (prec == SLSE_PREC_MIXED_BF16 && prob->dtype != SLSE_F32) return SLSE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int nsm = num_sms();
  if (nsm <= 0) return SLSE_ECUDA;
  Workspace W;
  slse_status a = acquire(W, workspace, ws_bytes, grad_ws(prob, nsm), st);
  if (a != SLSE_OK) return a;
  char *base = static_cast<char *>(W.ptr);
  DevState *dst = reinterpret_cast<DevState *>(base);
  double *part = reinterpret_cast<double *>(base + kStateBytes);
  const int nb = grad_blocks(prob->N, 2 * nsm);
  const bool mixed = prec == SLSE_PREC_MIXED_BF16;
  k_init_state<<<1, 32, 0, st>>>(dst, mixed ? 1 : 0, debug_spin_limit());
  CK(cudaGetLastError());
  CK(launch_grad(mixed ? GM_MIXED : GM_F64, prob->dtype, prob->X, prob->ldx, prob->Y, prob->N, prob->d, beta, dst,
                 nullptr, nullptr, nullptr, part, nb, 0, st));
  CK(launch_reduce(part, nb, prob->d, 1.0, g_out, dst, 0, st));
  return SLSE_OK;
}

slse_status slse_gram(const slse_problem *prob, double *G, void *workspace, size_t ws_bytes, slse_stream_t stream) {
  if (!valid_gram_problem(prob) || !G) return SLSE_EINVAL;
  if (is_host_pointer(prob->X) || is_host_pointer(G)) return SLSE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int nsm = num_sms();
  if (nsm <= 0) return SLSE_ECUDA;
  const bool bf16 = prob->dtype == SLSE_BF16;
  const GramPlan gp = bf16 ? GramPlan{} : gram_plan(prob->N, prob->d, nsm);
  const GramWPlan wp = bf16 ? gram_w_plan(prob->N, prob->d, nsm) : GramWPlan{};
  if (bf16 && !gram_w_ok(wp, prob->X, prob->ldx)) return SLSE_EINVAL;
  Layout w;
  const size_t o_state = w.take(kStateBytes);
  const size_t o_gram = w.take(bf16 ? wp.part_bytes : gp.total);
  Workspace W;
  slse_status a = acquire(W, workspace, ws_bytes, w.total, st);
  if (a != SLSE_OK) return a;
  char *base = static_cast<char *>(W.ptr);
  DevState *dst = reinterpret_cast<DevState *>(base + o_state);
  k_init_state<<<1, 32, 0, st>>>(dst, 0, debug_spin_limit());
  CK(cudaGetLastError());
  if (bf16)
    CK(launch_gram_w(wp, prob->X, prob->ldx, 1.0, G, &dst->status, reinterpret_cast<float *>(base + o_gram), st));
  else
    CK(launch_gram(gp, static_cast<const float *>(prob->X), prob->ldx, G, &dst->status, base + o_gram, st));
  return SLSE_OK;
}

slse_status slse_draws(int64_t N, uint64_t seed, int32_t *P, int32_t *sigma, int8_t *D, void *workspace,
                       size_t ws_bytes, slse_stream_t stream) {
  if (N < 1 || padded(N) > kMaxNp || !P || !sigma) return SLSE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t Np = padded(N);
  Workspace W;
  slse_status a = acquire(W, workspace, ws_bytes, align256(draws_ws_bytes(Np)), st);
  if (a != SLSE_OK) return a;
  CK(launch_draws(Np, seed, nullptr, P, sigma, D, W.ptr, st));
  return SLSE_OK;
}

slse_status slse_qr(const double *A, int64_t r, int32_t d, int64_t lda, double *R, double *Hinv, void *workspace,
                    size_t ws_bytes, slse_stream_t stream) {
  if (!A || !R || d < 1 || d > 512 || r < d || lda < d) return SLSE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int nsm = num_sms();
  if (nsm <= 0) return SLSE_ECUDA;
  Layout w;
  const size_t o_state = w.take(kStateBytes);
  const size_t o_a = w.take((size_t)r * d * 8);
  const size_t o_qr = w.take(qr_ws_bytes(r, d, nsm));
  Workspace W;
  slse_status a = acquire(W, workspace, ws_bytes, w.total, st);
  if (a != SLSE_OK) return a;
  char *base = static_cast<char *>(W.ptr);
  DevState *dst = reinterpret_cast<DevState *>(base + o_state);
  double *Ac = reinterpret_cast<double *>(base + o_a);
  k_init_state<<<1, 32, 0, st>>>(dst, 0, debug_spin_limit());
  CK(cudaGetLastError());
  CK(cudaMemcpy2DAsync(Ac, (size_t)d * 8, A, (size_t)lda * 8, (size_t)d * 8, (size_t)r, cudaMemcpyDeviceToDevice, st));
  CK(launch_qr(Ac, r, d, d, R, Hinv, base + o_qr, dst, st));
  return SLSE_OK;
}

int32_t slse_default_schedule(int64_t N, int32_t d, slse_schedule *out, int64_t *m_buf, int32_t *a_buf, int32_t cap) {
  return slse_default_schedule_for(N, d, SLSE_SRHT, out, m_buf, a_buf, cap);
}

int32_t slse_default_schedule_for(int64_t N, int32_t d, int32_t kind, slse_schedule *out, int64_t *m_buf,
                                  int32_t *a_buf, int32_t cap) {
  if (!out || N < 1 || d < 1) return -1;
  if (kind != SLSE_SRHT && kind != SLSE_COUNTSKETCH && kind != SLSE_GAUSSIAN) return -1;
  const int64_t Np = padded(N);
  int32_t K = 0;
  // CountSketch sizes are powers of two: m_1 = 8d rounded up
  const int64_t m1 = kind == SLSE_COUNTSKETCH ? padded(8 * (int64_t)d) : 8 * (int64_t)d;
  for (int64_t m = m1; m <= Np / 2; m *= 2) {
    if (K < cap && m_buf && a_buf) {
      m_buf[K] = m;
      a_buf[K] = 2;
    }
    ++K;
  }
  std::memset(out, 0, sizeof(*out));
  out->K = K < cap ? K : cap;
  out->m = m_buf;
  out->a = a_buf;
  out->r = 6 * (int64_t)d;
  out->eta = (double)d / (double)out->r;
  out->mu = (1.0 - out->eta) * (1.0 - out->eta);
  out->T = 100;
  out->tol = 0.0;
  out->kind = kind;
  out->prec = SLSE_PREC_FP64;
  out->momentum_reset = 0;  // Algorithm 2: one global counter t, momentum carries
  out->stage2 = SLSE_STAGE2_CORRECTION;
  return K;
}

int32_t slse_tuning_schedule(int64_t N, int32_t d, int32_t kind, slse_schedule *out, int64_t *m_buf, int32_t *a_buf,
                             int32_t cap) {
  if (slse_default_schedule_for(N, d, kind, out, nullptr, nullptr, 0) < 0) return -1;
  const int64_t Np = padded(N);
  std::vector<int64_t> m;
  for (int j = 0; j <= 6; ++j) m.push_back(16 * (int64_t)d << j);
  m.push_back(8192 * (int64_t)d);
  std::vector<int64_t> keep;
  for (int64_t v : m) {
    if (kind == SLSE_COUNTSKETCH) v = padded(v);
    if (v <= Np / 2 && (keep.empty() || v > keep.back())) keep.push_back(v);
  }
  const int32_t K = (int32_t)keep.size();
  for (int32_t i = 0; i < K && i < cap && m_buf && a_buf; ++i) {
    m_buf[i] = keep[i];
    a_buf[i] = 3;
  }
  out->K = K < cap ? K : cap;
  out->m = m_buf;
  out->a = a_buf;
  return K;
}

double slse_ai_bound(double omega, int64_t m_prev, int64_t m_i, int32_t d) {
  if (!(omega > 0.0) || m_prev <= d || m_i <= d) return NAN;
  const double r = std::sqrt((double)(m_i - d) / (double)(m_prev - d));
  return std::log(((1.0 + omega) * r + 1.0) / omega) / std::log(3.0);
}

const char *slse_status_string(int32_t s) {
  switch (s) {
    case SLSE_OK: return "ok";
    case SLSE_EINVAL: return "invalid argument";
    case SLSE_ENOMEM: return "workspace too small or allocation failed";
    case SLSE_ECUDA: return "CUDA runtime error";
    case SLSE_ENOTCONV: return "iteration cap reached before the tolerance";
    case SLSE_ENUMERIC: return "non-finite iterate or zero pivot";
    case SLSE_ETIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
  }
}

int32_t slse_version(void) { return 100; }

int64_t slse_debug_spin_limit(int64_t polls) {
  return (int64_t)g_spin_limit.exchange(polls > 0 ? (long long)polls : 0, std::memory_order_relaxed);
}

}  // extern "C"
