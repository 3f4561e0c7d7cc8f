// Residual-gradient pass for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc (or any allocator) at the
// point where they need a gradient: plugins whose host application owns every
// device allocation and hands out only fixed buffers, or real-time loops that forbid
// allocation after start-up.  slse_grad needs a small scratch area (a status word and one partial
// gradient per CTA) and gets it from the caller's workspace or from
// cudaMallocAsync.  slse_grad_noalloc runs the same gradient kernels but takes
// its scratch from the fixed array below, which lives in the library image: every
// GPU that loads the library holds these bytes until the process exits.
//
// Host code may not use the array's name as a device address (in host code it
// names a host-side stand-in).  The device address is obtained once per device
// with cudaGetSymbolAddress, with that device current, and cached; the same set-up
// loads the code of every kernel the entry point can launch, so that no later call
// loads a module (module loading allocates device memory).  A cudaDeviceReset
// destroys the array with its context: the cached address is then stale, so this
// entry point must not be called again in that process after a reset.
#include <mutex>

#include "slse_internal.cuh"

namespace {

constexpr size_t kNoAllocStateBytes = 4096;              // DevState (cleared by every call)
constexpr size_t kNoAllocPartialBytes = size_t(1) << 20; // per-CTA partial gradients (FP64)
constexpr size_t kNoAllocBytes = kNoAllocStateBytes + kNoAllocPartialBytes;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void k_clear_state(slse::DevState *st, int rebase) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    slse::DevState z = {};
    z.rebase = rebase;
    *st = z;
  }
}

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set up on first use).
slse_status scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SLSE_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return SLSE_ECUDA;
    }
    cudaFuncAttributes fa;
    if (slse::preload_grad_kernels() != cudaSuccess || cudaFuncGetAttributes(&fa, (const void *)k_clear_state) != cudaSuccess) {
      cudaGetLastError();
      return SLSE_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SLSE_OK;
}

}  // namespace

extern "C" slse_status slse_grad_noalloc(const slse_problem *prob, const double *beta, double *g_out,
                                         int32_t prec, slse_stream_t stream) {
  using namespace slse;
  if (!valid_problem(prob) || !beta || !g_out) return SLSE_EINVAL;
  if (prec != SLSE_PREC_FP64 && prec != SLSE_PREC_MIXED_BF16) return SLSE_EINVAL;
  if (prec == SLSE_PREC_MIXED_BF16 && prob->dtype != SLSE_F32) return SLSE_EINVAL;
  if (is_host_pointer(prob->X) || is_host_pointer(prob->Y) || is_host_pointer(beta) || is_host_pointer(g_out))
    return SLSE_EINVAL;
  // the partials of at least one CTA must fit: d <= kNoAllocPartialBytes / 8 (always true for d <= 512)
  const int64_t max_blocks = (int64_t)(kNoAllocPartialBytes / (8 * (size_t)prob->d));
  if (max_blocks < 1) return SLSE_ENOMEM;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
    cudaGetLastError();
    return SLSE_ECUDA;
  }
  int64_t nblk = (prob->N + 31) / 32;
  if (nblk > 2 * (int64_t)nsm) nblk = 2 * (int64_t)nsm;
  if (nblk > max_blocks) nblk = max_blocks;
  if (nblk < 1) nblk = 1;
  void *base = nullptr;
  const slse_status st = scratch_address(&base);
  if (st != SLSE_OK) return st;
  DevState *ds = static_cast<DevState *>(base);
  double *part = reinterpret_cast<double *>(static_cast<char *>(base) + kNoAllocStateBytes);
  const cudaStream_t s = (cudaStream_t)stream;
  const bool mixed = prec == SLSE_PREC_MIXED_BF16;
  k_clear_state<<<1, 32, 0, s>>>(ds, mixed ? 1 : 0);
  if (cudaGetLastError() != cudaSuccess) return SLSE_ECUDA;
  if (launch_grad(mixed ? GM_MIXED : GM_F64, prob->dtype, prob->X, prob->ldx, prob->Y, prob->N, prob->d, beta, ds,
                  nullptr, nullptr, nullptr, part, (int)nblk, 0, s) != cudaSuccess)
    return SLSE_ECUDA;
  if (launch_reduce(part, (int)nblk, prob->d, 1.0, g_out, ds, 0, s) != cudaSuccess) return SLSE_ECUDA;
  return SLSE_OK;
}
