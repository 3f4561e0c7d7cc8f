// Gram matrix G_b = Xb^T Xb of the BF16 rounding Xb of X on the tensor cores, for the Hessian term
// of the mixed 2nd stage's correction form: between exact passes the gradient is
// g(beta) = g(beta_e) - Xb^T Xb (beta - beta_e), and with G_b formed once each of those steps is a
// d x d product instead of a pass over X.  Xb^T Xb is a dense (d x N)(N x d) contraction, so it
// runs on tcgen05 (BF16 operands, FP32 accumulation in tensor memory).
//
// Both operands of the MMA are the same rows of X in the K-major core-matrix layout (element
// (n, k) of a 32-row chunk at byte (n div 8) 512 + (k div 8) 128 + (n mod 8) 16 + (k mod 8) 2, n the
// column of X and k the row in the chunk), so column c of a chunk starts at byte 64 c.  A tile is
// 128 rows of G_b (MMA M = 128, A = 128 columns of the chunk) times up to 256 columns (B).  Each CTA
// keeps its tiles in tensor memory for a range of at most 8192 rows and writes them as an FP32
// partial; the reduction adds the ranges' partials in a fixed order in FP64 (deterministic) from
// the upper triangle and mirrors it, so G_b is exactly symmetric.
//
// Three ways in:
//  - k_gram_w (BF16 input: the SRHT intermediate W inside the fit, BF16 X through slse_gram): the
//    MMAs read the row-major tiles as MN-major operands straight from TMA boxes.
//  - k_gram_f32 (X FP32 with 16-byte aligned rows and d a multiple of 4): 1-3 CTAs per range of
//    rows; each copies the columns its tiles read, 32 rows at a time, into shared memory (2-D TMA
//    boxes of 32 rows x 128 columns; zeros past the edges), eight converter warps round them to
//    BF16 into the chunk layout (one column of 8 rows per thread and step: 8 conflict-free 4-byte
//    reads, one 16-byte write) and warp 1 issues the MMAs of the CTA's tiles.  The CTAs of a range
//    sit next to each other in the grid and share X's rows through L2; the tiles cover the upper
//    triangle with equal MMA work per CTA (roles below).
//  - k_gram_tc (any other X): X is first packed to BF16 chunks by the Gaussian sketch's packer,
//    then streamed by bulk copies; the CTA of column block i0 forms rows i0 .. i0 + 127 times all
//    columns (the CTAs of a range then run at one rate and share the chunks through L2).
// Every mbarrier wait gives up after 2 s (ST_TIMEOUT, NaN output); copies in flight are awaited
// and tensor memory is freed on that path too.  Shared memory is sized so that one CTA runs per SM
// (its tensor-memory allocation then always succeeds at once).
#include "tc_common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cuda_bf16.h>

#include <initializer_list>

namespace slse {
namespace {

constexpr int kGM = 128;                 // rows of G_b per CTA (MMA M)
constexpr int kGK = 32;                  // rows of X per chunk
constexpr int kGSBO = kGK * 16;          // bytes between 8-column groups of a chunk
constexpr int kGThreads = 128;           // warp 0: copies, warp 1: MMAs, warps 0-3: epilogue
constexpr int kGMaxStages = 6;
constexpr int64_t kGMaxRangeChunks = 256;
// k_gram_f32: every CTA reads and rounds the columns its tiles read (own segments, no copies
// between CTAs) rather than one segment each with the hub receiving the others': measured faster
// at N = 2^22 (d = 512: 3.5 against 4.2 ms; d = 384: 2.7 against 3.1 ms), the CTAs of a range
// sharing X through L2; the hub form is kept as the other form of the roles
constexpr bool kFOwn = true;
constexpr int kFConv = 8;                        // converter warps of k_gram_f32
constexpr int kFThreads = 64 + 32 * kFConv;      // + copy warp + MMA warp

// MMAs of one 32-row chunk at shared address xb: A = columns i0 .. i0 + 127, B = columns
// 0 .. W - 1 (W a multiple of 128) in pieces of <= 256 columns; accumulate unless this is the
// range's first chunk.
__device__ __forceinline__ void gram_chunk_mma(uint32_t tmem, uint32_t xb, int i0, int W, bool first) {
  const uint32_t ab = xb + (uint32_t)i0 * 64u;
#pragma unroll
  for (int ks = 0; ks < kGK / 16; ++ks) {
    // K step ks covers core-matrix columns 2 ks, 2 ks + 1 (128 bytes apart)
    const uint64_t ad = umma_desc(ab + ks * 256, 128, kGSBO);
    const uint32_t acc = (!first || ks > 0) ? 1u : 0u;
    for (int c = 0; c < W; c += 256) {
      const int n = W - c < 256 ? W - c : 256;
      umma_bf16(tmem + (uint32_t)c, ad, umma_desc(xb + (uint32_t)c * 64u + ks * 256, 128, kGSBO),
                umma_idesc_bf16(kGM, n), acc);
    }
  }
}

// the accumulator of rows i0 + 32 q + lane (q = warp mod 4), columns c (relative to i0) of
// c0, c0 + cstep, ... in 32-column pieces, to the range's partial
__device__ __forceinline__ void gram_store(uint32_t tmem, float *part_row, int W, int q, int c0, int cstep) {
  for (int c = c0; c < W; c += cstep) {
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
#pragma unroll
    for (int j = 0; j < 32; j += 4)
      *reinterpret_cast<uint4 *>(part_row + c + j) = make_uint4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  }
}

struct GramArgs {
  const uint8_t *xt;   // nchunk packed chunks of ncp * 64 bytes
  float *part;         // [splits][ncp][ncp]
  unsigned *status;
  int64_t nchunk, cps; // chunks, chunks per range
  int ncp;             // packed columns: a multiple of 128, <= 512
  int tmem_cols;       // power of two >= ncp
  int stages;
};

__global__ void __launch_bounds__(kGThreads, 1) k_gram_tc(const GramArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = a.stages;
  const uint32_t bC = (uint32_t)a.ncp * (kGK * 2);  // bytes of one chunk
  uint8_t *sX = sm;
  uint64_t *full = reinterpret_cast<uint64_t *>(sX + (size_t)S * bC);
  uint64_t *empty = full + S;
  uint64_t *accum = empty + S;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(accum + 1);
  volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort_f = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
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
  const int i0 = (int)blockIdx.x * kGM;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0, s = 0;
      uint32_t ph = 0;
      for (int k = 0; k < nk; ++k) {
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_f, a.status)) break;
        mbar_arrive_expect_tx(&full[s], bC);
        bulk_g2s(sX + (size_t)s * bC, a.xt + (size_t)(c0 + k) * bC, bC, &full[s]);
        issued = k + 1;
        if (++s == S) { s = 0; ph ^= 1u; }
      }
      // copies in flight land before the CTA exits (on the normal path the MMA thread has
      // already seen every one of them)
      const int first = issued > S ? issued - S : 0;
      for (int k = first; k < issued; ++k) {
        volatile int never = 0;
        mbar_wait(&full[k % S], (uint32_t)(k / S) & 1u, &never, a.status);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      for (int k = 0; k < nk; ++k) {
        if (!mbar_wait(&full[s], ph, abort_f, a.status)) break;
        tc_fence_after();
        gram_chunk_mma(tmem, smem_u32(sX + (size_t)s * bC), i0, a.ncp, k == 0);
        umma_commit(&empty[s]);
        if (++s == S) { s = 0; ph ^= 1u; }
      }
      umma_commit(accum);  // arrives once every MMA issued above has completed
    }
  }
  // epilogue: TMEM lanes 32 warp .. 32 warp + 31 hold rows i0 + 32 warp + lane of G_b
  {
    const bool ok = mbar_wait(accum, 0u, abort_f, a.status);
    tc_fence_after();
    if (__all_sync(0xFFFFFFFFu, ok && !*abort_f) && nk > 0)
      gram_store(tmem, a.part + ((int64_t)blockIdx.y * a.ncp + i0 + 32 * warp + lane) * a.ncp, a.ncp, warp, 0, 32);
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// Roles of the CTAs of one cluster of k_gram_f32 (Q = 1, 2 or 3 CTAs, one range of rows).  CTA r
// reads and rounds the columns lo .. hi - 1 of X (its segment; empty for the hub of d > 384) and
// forms its tiles: tile t is rows 128 a_blk .. 128 a_blk + 127 of G_b times columns b_lo .. b_lo +
// n - 1 (n <= 256, one MMA per K step) in tensor-memory columns toff ...  Rank 0 (the hub) receives
// every other CTA's rounded segment into its own chunk buffer (a bulk copy between the CTAs' shared
// memories) and forms the tiles that need columns of several segments.  The tiles of all ranks
// cover the upper triangle of G_b (i <= j) once, with equal MMA work per CTA:
//   ncp 128: r0 [0,128)   : (0, 0, 128)
//   ncp 256: r0 [0,256)   : (0, 0, 256) (1, 128, 128)
//   ncp 384: r0 [0,128)   : (0, 0, 256) (0, 256, 128)          r1 [128,384): (1, 128, 256) (2, 256, 128)
//   ncp 512: r0 (none)    : (0, 256, 256) (1, 256, 256)
//            r1 [0,256)   : (0, 0, 256) (1, 0, 256)            r2 [256,512): (2, 256, 256) (3, 256, 256)
// so each column of X is read from DRAM and rounded once, and no CTA waits on a wider one.
struct GramRole {
  int lo, hi;  // segment
  int ntile;
  int a_blk[2], b_lo[2], n[2], toff[2];
};

struct GramF32Args {
  CUtensorMap tmap;     // X as (d, N) FP32, boxes of 128 columns x 32 rows
  int64_t N;
  int d;
  float *part;          // [splits][ncp][ncp], upper triangle
  unsigned *status;
  int64_t nstage, cps;  // 32-row stages of X, stages per range
  int ncp, tmem_cols, Q;
  int in_bytes;         // bytes the hub receives per stage
  int own;              // every CTA reads and rounds the columns its tiles read (segment = that
                        // range; no copies between CTAs, a cluster of one)
  int s3, nb;           // FP32 stages, chunk buffers (the hub's of the full width, a peer's of its segment)
  int o_bar;            // byte offset of the barriers (the same in every CTA of the cluster)
  int o16[3];           // byte offset of each role's chunk buffers
  GramRole role[3];
};

constexpr int kFMaxB = 8;   // most stages or buffers of any kind

__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cl_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_addr) : "memory");
}
// shared -> peer shared bulk copy completing on the peer's mbarrier (16-byte aligned, size a
// multiple of 16)
__device__ __forceinline__ void bulk_s2c(uint32_t cl_dst, const void *src, uint32_t bytes, uint32_t cl_bar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   cl_dst),
               "r"(smem_u32(src)), "r"(bytes), "r"(cl_bar)
               : "memory");
}

// 2-D tiled TMA load of the box at (x, y) of the tensor map into shared memory, completing on an
// mbarrier (x a multiple of 4 for FP32; boxes past the edge of X read zeros)
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared memory of a CTA: s3 FP32 stages of its segment (32 rows x sw columns, in row-major panels
// of 128 columns), then its nb chunk buffers (the hub's of the full width, columns at their own
// offsets; a peer's of its segment, columns relative to lo), then the barriers at o_bar.
// Per stage k the hub's buffer k mod nb is released (its incoming bytes expected, hubfree signalled
// to the peers) once the hub's MMAs of stage k - nb have completed; a peer rounds stage k into its
// buffer k mod nb once its own MMAs of stage k - nb have completed and the hub has released stage k
// (which implies that the peer's copy of stage k - nb, out of the same buffer, has landed), then
// copies the segment into the hub's buffer and issues its own tiles.  (A separate signal of each
// landed copy, so that the hub could hold more buffers than the peers, measured slower.)
__global__ void __launch_bounds__(kFThreads, 1) k_gram_f32(const __grid_constant__ GramF32Args a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int rank = (int)blockIdx.x;  // cluster (Q, 1, 1) over grid (Q, ranges)
  const bool hub = rank == 0 && !a.own;
  // the role, selected with static indices so that it stays in registers (a dynamic index into
  // the parameter array would copy it to local memory, on the MMA issue path)
  const GramRole ro = rank == 0 ? a.role[0] : (rank == 1 ? a.role[1] : a.role[2]);
  const int sw = ro.hi - ro.lo;                      // segment width: 0, 128 or 256
  const int ncol = sw > 0 ? (ro.hi < a.d ? ro.hi : a.d) - ro.lo : 0;  // columns of X inside the segment
  const int cbase = hub ? 0 : ro.lo;                 // column at byte 0 of this CTA's chunk buffers
  const int nb = a.nb;
  const uint32_t b32 = (uint32_t)sw * (kGK * 4u);    // one FP32 stage
  const uint32_t b16 = (uint32_t)(hub ? a.ncp : sw) * (kGK * 2u);  // one chunk buffer
  float *s32 = reinterpret_cast<float *>(sm);
  uint8_t *s16 = sm + a.o16[rank];
  uint64_t *full32 = reinterpret_cast<uint64_t *>(sm + a.o_bar);
  uint64_t *empty32 = full32 + kFMaxB;
  uint64_t *fullb = empty32 + kFMaxB;
  uint64_t *emptyb = fullb + kFMaxB;
  uint64_t *hubfree = emptyb + kFMaxB;  // peers: the hub released its buffer for a stage
  uint64_t *accum = hubfree + kFMaxB;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(accum + 1);
  volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.s3; ++s) {
      mbar_init(&full32[s], 1);
      mbar_init(&empty32[s], kFConv);
    }
    for (int b = 0; b < nb; ++b) {
      mbar_init(&fullb[b], hub ? 1 + (sw > 0 ? kFConv : 0) : kFConv);
      mbar_init(&emptyb[b], 1);
      mbar_init(&hubfree[b], 1);
    }
    mbar_init(accum, 1);
    *abort_f = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  // the peers' barriers are initialised before any remote arrive or copy reaches them
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int64_t st0 = (int64_t)blockIdx.y * a.cps;
  const int64_t st1 = st0 + a.cps < a.nstage ? st0 + a.cps : a.nstage;
  const int nk = (int)(st1 - st0);
  const int64_t row0 = st0 * kGK;
  auto rows_of = [&](int k) -> int {
    const int64_t r = a.N - (row0 + (int64_t)k * kGK);
    return r < kGK ? (int)r : kGK;
  };
  // operand offsets and instruction descriptors of the (at most 2) tiles, once
  uint32_t a_off[2], b_off[2], idesc[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    a_off[t] = (uint32_t)(kGM * ro.a_blk[t] - cbase) * 64u;
    b_off[t] = (uint32_t)(ro.b_lo[t] - cbase) * 64u;
    idesc[t] = umma_idesc_bf16(kGM, t < ro.ntile ? ro.n[t] : 128);
  }
  auto tiles_mma = [&](uint32_t xb, bool first) {
#pragma unroll
    for (int ks = 0; ks < kGK / 16; ++ks) {
      const uint32_t acc = (!first || ks > 0) ? 1u : 0u;
#pragma unroll
      for (int t = 0; t < 2; ++t)
        if (t < ro.ntile)
          umma_bf16(tmem + (uint32_t)ro.toff[t], umma_desc(xb + a_off[t] + ks * 256, 128, kGSBO),
                    umma_desc(xb + b_off[t] + ks * 256, 128, kGSBO), idesc[t], acc);
    }
  };

  if (warp == 0) {
    // copies of the segment: one TMA box (32 rows x 128 columns, 16 KB) per 128 columns and stage
    if (lane == 0 && ncol > 0) {
      const int npan = sw / 128;
      int issued = 0;
      for (int k = 0; k < nk; ++k) {
        const int s = k % a.s3;
        if (!mbar_wait(&empty32[s], ((uint32_t)(k / a.s3) & 1u) ^ 1u, abort_f, a.status)) break;
        mbar_arrive_expect_tx(&full32[s], b32);
        for (int pn = 0; pn < npan; ++pn)
          tma_load_2d(s32 + (size_t)s * (b32 / 4) + pn * (kGK * 128), &a.tmap, ro.lo + 128 * pn,
                      (int)(row0 + (int64_t)k * kGK), &full32[s]);
        issued = k + 1;
      }
      // copies in flight land before the CTA exits
      const int first = issued > a.s3 ? issued - a.s3 : 0;
      for (int k = first; k < issued; ++k) {
        volatile int never = 0;
        mbar_wait(&full32[k % a.s3], (uint32_t)(k / a.s3) & 1u, &never, a.status);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (hub) {
        auto release = [&](int j) {
          const int b = j % nb;
          mbar_arrive_expect_tx(&fullb[b], (uint32_t)a.in_bytes);
          for (int r = 1; r < a.Q; ++r) mbar_arrive_remote(cluster_addr(smem_u32(&hubfree[b]), r));
        };
        int released = nk < nb ? nk : nb, consumed = 0;
        for (int j = 0; j < released; ++j) release(j);
        for (int k = 0; k < nk; ++k) {
          const int b = k % nb;
          if (!mbar_wait(&fullb[b], (uint32_t)(k / nb) & 1u, abort_f, a.status)) break;
          consumed = k + 1;
          tc_fence_after();
          tiles_mma(smem_u32(s16 + (size_t)b * b16), k == 0);
          umma_commit(&emptyb[b]);
          const int j = k - 1 + nb;  // the stage that reuses stage k - 1's buffer
          if (k >= 1 && j < nk) {
            if (!mbar_wait(&emptyb[(k - 1) % nb], (uint32_t)((k - 1) / nb) & 1u, abort_f, a.status)) break;
            release(j);
            released = j + 1;
          }
        }
        umma_commit(accum);  // arrives once every MMA issued above has completed
        // every copy into this CTA has landed before it exits: after a failure, the stages released
        // but not consumed (the latest phase of their buffers) are awaited, each wait bounded
        for (int j = consumed; j < released; ++j) {
          volatile int never = 0;
          mbar_wait(&fullb[j % nb], (uint32_t)(j / nb) & 1u, &never, a.status);
        }
      } else {
        for (int k = 0; k < nk; ++k) {
          const int b = k % nb;
          if (!mbar_wait(&fullb[b], (uint32_t)(k / nb) & 1u, abort_f, a.status)) break;
          tc_fence_after();
          // the rounded segment to the hub's buffer b (released for this stage: the converters
          // waited for that), then this CTA's own tiles
          uint8_t *seg = s16 + (size_t)b * b16;
          uint8_t *hub_seg = sm + a.o16[0] + (size_t)b * ((size_t)a.ncp * kGK * 2) + (size_t)ro.lo * 64;
          if (!a.own) bulk_s2c(cluster_addr(smem_u32(hub_seg), 0), seg, b16, cluster_addr(smem_u32(&fullb[b]), 0));
          tiles_mma(smem_u32(seg), k == 0);
          umma_commit(&emptyb[b]);
        }
        umma_commit(accum);
      }
    }
  } else if (sw > 0) {
    // converters: item (n, k8) = column lo + n, rows 8 k8 .. 8 k8 + 7 of the stage; consecutive
    // threads take consecutive columns
    const int ct = threadIdx.x - 64;
    const int lsw = sw == 512 ? 9 : (sw == 256 ? 8 : (sw == 128 ? 7 : -1));  // -1: divide
    for (int k = 0; k < nk; ++k) {
      const int s = k % a.s3, b = k % nb;
      const uint32_t pb = (uint32_t)(k / nb) & 1u;
      bool ok = mbar_wait(&full32[s], (uint32_t)(k / a.s3) & 1u, abort_f, a.status);
      ok = ok && mbar_wait(&emptyb[b], pb ^ 1u, abort_f, a.status);
      if (!hub && !a.own) ok = ok && mbar_wait(&hubfree[b], pb, abort_f, a.status);
      if (!__all_sync(0xFFFFFFFFu, ok)) break;
      const int nr = rows_of(k);
      const float *src = s32 + (size_t)s * (b32 / 4);
      uint8_t *dst = s16 + (size_t)b * b16 + (size_t)(ro.lo - cbase) * 64;
      for (int it = ct; it < sw * (kGK / 8); it += 32 * kFConv) {
        const int n = lsw >= 0 ? (it & (sw - 1)) : it % sw, k8 = lsw >= 0 ? (it >> lsw) : it / sw;
        const int pan = (n >> 7) * (kGK * 128) + (n & 127);  // panel of 128 columns, row-major
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = 8 * k8 + 2 * q;
          const float f0 = (n < ncol && r < nr) ? src[pan + r * 128] : 0.f;
          const float f1 = (n < ncol && r + 1 < nr) ? src[pan + (r + 1) * 128] : 0.f;
          const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);  // row r in the low half
          w[q] = *reinterpret_cast<const uint32_t *>(&h);
        }
        *reinterpret_cast<uint4 *>(dst + (n >> 3) * kGSBO + k8 * 128 + (n & 7) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
      }
      fence_proxy_async_smem();  // the MMAs and the copy to the hub (async proxy) read these writes
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&fullb[b]);
        mbar_arrive(&empty32[s]);
      }
    }
  }
  // epilogue (converter warps): TMEM lanes 32 q .. 32 q + 31, q = warp mod 4, hold rows
  // 128 a_blk + 32 q + lane of tile t; the two warps of a lane quarter take alternate 32-column
  // pieces
  if (warp >= 2) {
    const bool ok = mbar_wait(accum, 0u, abort_f, a.status);
    tc_fence_after();
    const int q = warp & 3;
    if (__all_sync(0xFFFFFFFFu, ok && !*abort_f) && nk > 0) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t >= ro.ntile) break;
        float *row = a.part + ((int64_t)blockIdx.y * a.ncp + kGM * ro.a_blk[t] + 32 * q + lane) * a.ncp + ro.b_lo[t];
        gram_store(tmem + (uint32_t)ro.toff[t], row, ro.n[t], q, 32 * ((warp - 2) >> 2), 64);
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
  // no CTA leaves while a peer may still signal it or copy into it
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The partials are summed in two streaming steps, each in a fixed order (deterministic): groups of
// kRG ranges into FP64 group sums (consecutive threads read consecutive entries of one range's
// partial: every partial is read in contiguous rows), then the groups, scaled and mirrored.  (One
// thread per entry walking all ranges, 1 MB apart, took 0.49 ms at 512 ranges: latency and TLB
// bound.)  Only the upper triangle (j >= i) is read; NaN after a timeout.
constexpr int kRG = 16;

// grp[g][i][j] = sum of part[r][i][j] over ranges r of group g, j >= i; grid (ncp rows x ncp / 128
// column blocks, groups), 128 threads
__global__ void __launch_bounds__(128) k_gram_reduce_grp(const float *__restrict__ part, int splits, int ncp,
                                                         double *__restrict__ grp) {
  const int i = blockIdx.x / (ncp / 128), j = (blockIdx.x % (ncp / 128)) * 128 + threadIdx.x;
  if (j < i) return;
  const int g = blockIdx.y;
  const int r1 = (g + 1) * kRG < splits ? (g + 1) * kRG : splits;
  const int64_t e = (int64_t)i * ncp + j, step = (int64_t)ncp * ncp;
  double acc = 0.0;
  for (int r = g * kRG; r < r1; ++r) acc += (double)__ldg(part + r * step + e);
  grp[g * step + e] = acc;
}

// G[i, j] = G[j, i] = scale x the sum of the group sums, i <= j < d
__global__ void k_gram_reduce(const double *__restrict__ grp, int ngroups, int ncp, int d, double scale,
                              const unsigned *status, double *G) {
  const bool bad = (*(volatile const unsigned *)status & ST_TIMEOUT) != 0;
  const int i = blockIdx.y;
  const int j = i + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= d) return;
  const int64_t e = (int64_t)i * ncp + j, step = (int64_t)ncp * ncp;
  double v = 0.0;
  for (int g = 0; g < ngroups; ++g) v += grp[g * step + e];
  v *= scale;
  if (bad) v = __longlong_as_double(0x7FF8000000000000ll);
  G[(int64_t)i * d + j] = v;
  G[(int64_t)j * d + i] = v;
}

// both reduction steps; grp holds ceil(splits / kRG) ncp^2 doubles
cudaError_t launch_gram_reduce(const float *part, int splits, int ncp, int d, double scale, double *grp,
                               const unsigned *status, double *G, cudaStream_t s) {
  const int ng = (splits + kRG - 1) / kRG;
  k_gram_reduce_grp<<<dim3((unsigned)(ncp / 128) * (unsigned)ncp, (unsigned)ng), 128, 0, s>>>(part, splits, ncp, grp);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  k_gram_reduce<<<dim3((unsigned)((d + 255) / 256), (unsigned)d), 256, 0, s>>>(grp, ng, ncp, d, scale, status, G);
  return cudaGetLastError();
}
size_t gram_grp_bytes(int splits, int ncp) { return (size_t)((splits + kRG - 1) / kRG) * ncp * ncp * 8; }

int64_t gcdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t gal256(size_t x) { return (x + 255) & ~(size_t)255; }

// ranges of at most max_units units (8192 rows): the FP32 sum of a range in tensor memory then
// stays within ~2e-5 of sum |x_i x_j| (measured 9e-6 at 3400 rows); at least one range per SM and
// column block (or cluster)
void gram_split(int64_t nunit, int mt, int nsm, int64_t &cps, int &splits, int64_t max_units = kGMaxRangeChunks) {
  int64_t sp = (nsm > 0 ? nsm : 152) / mt;
  if (sp < gcdiv(nunit, max_units)) sp = gcdiv(nunit, max_units);
  if (sp < 1) sp = 1;
  if (sp > nunit) sp = nunit;
  cps = gcdiv(nunit, sp);
  splits = (int)gcdiv(nunit, cps);
}

// the roles of the cluster's CTAs for ncp columns (the table above k_gram_f32); returns Q
int gram_roles(int ncp, GramRole *ro, int *in_bytes) {
  auto set = [](GramRole &r, int lo, int hi, std::initializer_list<int> t) {
    r = GramRole{};
    r.lo = lo;
    r.hi = hi;
    const int *v = t.begin();
    r.ntile = (int)t.size() / 3;
    int off = 0;
    for (int k = 0; k < r.ntile; ++k) {
      r.a_blk[k] = v[3 * k];
      r.b_lo[k] = v[3 * k + 1];
      r.n[k] = v[3 * k + 2];
      r.toff[k] = off;
      off += r.n[k];
    }
  };
  int Q = 1;
  if (ncp == 128) {
    set(ro[0], 0, 128, {0, 0, 128});
  } else if (ncp == 256) {
    set(ro[0], 0, 256, {0, 0, 256, 1, 128, 128});
  } else if (ncp == 384) {
    Q = 2;
    set(ro[0], 0, 128, {0, 0, 256, 0, 256, 128});
    set(ro[1], 128, 384, {1, 128, 256, 2, 256, 128});
  } else {
    Q = 3;
    set(ro[0], 0, 0, {0, 256, 256, 1, 256, 256});
    set(ro[1], 0, 256, {0, 0, 256, 1, 0, 256});
    set(ro[2], 256, 512, {2, 256, 256, 3, 256, 256});
  }
  int in = 0;
  for (int r = 1; r < Q; ++r) in += (ro[r].hi - ro[r].lo) * 64;
  if (in_bytes) *in_bytes = in;
  return Q;
}

// own segments: each CTA's segment becomes the range of columns its tiles read
void gram_own_segments(int Q, GramRole *ro) {
  for (int r = 0; r < Q; ++r) {
    int lo = 1 << 30, hi = 0;
    for (int t = 0; t < ro[r].ntile; ++t) {
      const int c[4] = {kGM * ro[r].a_blk[t], kGM * (ro[r].a_blk[t] + 1), ro[r].b_lo[t], ro[r].b_lo[t] + ro[r].n[t]};
      lo = c[0] < lo ? c[0] : lo;
      lo = c[2] < lo ? c[2] : lo;
      hi = c[1] > hi ? c[1] : hi;
      hi = c[3] > hi ? c[3] : hi;
    }
    ro[r].lo = lo;
    ro[r].hi = hi;
  }
}

// shared-memory layout of k_gram_f32 (see there): 3 FP32 stages and 3 chunk buffers (measured
// fastest: 4 stages and up to 6 hub buffers were slower); the barriers at one offset for all
// roles; one CTA per SM
void gram_f32_layout(int ncp, const GramRole *ro, int Q, GramF32Args &a, size_t &smem) {
  int wmax = 0;
  for (int r = 0; r < Q; ++r) wmax = ro[r].hi - ro[r].lo > wmax ? ro[r].hi - ro[r].lo : wmax;
  a.s3 = wmax > 256 ? 2 : 3;  // own segments up to 512 columns: 2 + 2 buffers fit
  a.nb = wmax > 256 ? 2 : 3;
  int top = 0;
  for (int r = 0; r < Q; ++r) {
    const int sw = ro[r].hi - ro[r].lo;
    a.o16[r] = a.s3 * sw * kGK * 4;
    const int end = a.o16[r] + (r == 0 && !a.own ? ncp : sw) * a.nb * kGK * 2;
    if (end > top) top = end;
  }
  a.o_bar = (top + 7) & ~7;
  smem = (size_t)a.o_bar + (5 * kFMaxB + 1) * 8 + 8 + 1024;
  if (smem < 233472 / 2 + 1) smem = 233472 / 2 + 1;
}

// ---------------------------------------------------------------------------------------------
// Gram matrix of a BF16 matrix B (k_gram_w): of the SRHT intermediate W inside the mixed fit, and
// of BF16 X through slse_gram.  Pass 1 of the two-pass SRHT writes W = (I (x) H_n2) P D X in BF16
// (H_n2 unnormalised, P a row permutation with zero padding rows, D signs): W^T W = n2 X^T X
// exactly, so G_b = W_b^T W_b / n2 serves the correction form like the Gram of the BF16 rounding of
// X (the same relative rounding, 2^-9 per element), at half the bytes and with no rounding work:
// the MMA reads W's row-major tiles as MN-major operands straight from the TMA boxes (64 columns x
// 64 rows, 128-byte swizzle).
// Roles as in k_gram_f32 (the same tiles); each 64-column box of a stage is loaded once by one CTA
// and multicast to the CTAs whose tiles read it, the loads spread over the cluster:
//   ncp 512: boxes 0-3 -> {r0, r1}: r1 loads 0, 1, 2, r0 loads 3; boxes 4-7 -> {r0, r2}: r2 loads
//            4, 5, 6, r0 loads 7
//   ncp 384: boxes 0-1 -> {r0}: r0 loads; boxes 2-5 -> {r0, r1}: r1 loads 2, 3, 4, r0 loads 5
//   ncp <= 256: one CTA loads every box
// A CTA releases a stage's buffer (its incoming bytes expected, the loaders of its boxes told) once
// its MMAs of the stage that used the buffer before have completed; a loader issues a stage's
// boxes once every destination has released the buffer.
// rows of B per stage: KR = 64 (4 K steps; 32-row stages, twice as many in flight, measured 1.7x
// slower at d = 512); a box is 64 columns x KR rows (KR 128 bytes)
// boxes multicast within a cluster (each loaded once) or loaded by every CTA that reads them: the
// latter measured 1.8x faster at d = 512 (1.83 against 3.28 ms at N = 2^22; the cluster's
// buffer hand-offs serialised the stages), so multicast is kept only as the other form of the roles
constexpr bool kWMulticast = false;
constexpr int kWThreads = 224;           // warp 0: loads, warp 1: MMAs, warp 2: releases, warps 3-6: epilogue

struct GramWRole {
  int ntile;
  int a_blk[2], b_lo[2], n[2], toff[2];
  uint32_t issue;      // bit j: this CTA loads box j
  uint32_t feeds;      // bit q: CTA q loads boxes this CTA reads (it is told of releases)
  int nfree;           // number of CTAs a release of this CTA's loads waits for
  int recv_bytes;      // bytes this CTA receives per stage
};

struct GramWArgs {
  CUtensorMap tmap;    // B as (d, rows) BF16, boxes of 64 columns x 64 rows, 128-byte swizzle
  float *part;         // [splits][ncp][ncp], upper triangle
  unsigned *status;
  int64_t nstage, cps;
  int ncp, nbox, tmem_cols, Q, S;
  int o_bar;
  uint16_t dest[8];    // CTA mask receiving box j (multicast)
  int mc;              // boxes multicast within the cluster (else every CTA loads its own)
  GramWRole role[3];
};

// shared-memory descriptor of a tcgen05 operand in the 128-byte-swizzled layout (MN-major here:
// lbo = bytes between 64-element groups along M/N, sbo = bytes between 8-row groups along K)
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}
// 2-D TMA load multicast to the CTAs of mask (the same shared offset and mbarrier in each)
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, "
      "{%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

template <int KR>
__global__ void __launch_bounds__(kWThreads, 1) k_gram_w(const __grid_constant__ GramWArgs a) {
  constexpr uint32_t kBox = KR * 128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int rank = (int)blockIdx.x;  // cluster (Q, 1, 1) over grid (Q, ranges)
  const GramWRole ro = rank == 0 ? a.role[0] : (rank == 1 ? a.role[1] : a.role[2]);
  const int S = a.S;
  const uint32_t bstage = (uint32_t)a.nbox * kBox;
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + a.o_bar);
  uint64_t *empty = full + kFMaxB;
  uint64_t *slotfree = empty + kFMaxB;  // the destinations of this CTA's loads released a buffer
  uint64_t *accum = slotfree + kFMaxB;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(accum + 1);
  volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
  volatile int *s_released = reinterpret_cast<volatile int *>(tslot + 2);
  volatile int *s_consumed = reinterpret_cast<volatile int *>(tslot + 3);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&slotfree[s], ro.nfree > 0 ? ro.nfree : 1);
    }
    mbar_init(accum, 1);
    *abort_f = 0;
    *s_released = 0;
    *s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int64_t st0 = (int64_t)blockIdx.y * a.cps;
  const int64_t st1 = st0 + a.cps < a.nstage ? st0 + a.cps : a.nstage;
  const int nk = (int)(st1 - st0);

  if (warp == 0) {
    if (lane == 0 && ro.issue != 0u) {
      for (int k = 0; k < nk; ++k) {
        const int s = k % S;
        if (!mbar_wait(&slotfree[s], (uint32_t)(k / S) & 1u, abort_f, a.status)) break;
        const int y = (int)((st0 + k) * KR);
        for (int j = 0; j < a.nbox; ++j) {
          if (!(ro.issue >> j & 1u)) continue;
          uint8_t *dst = sm + (size_t)s * bstage + (size_t)j * kBox;
          if (!a.mc) tma_load_2d(dst, &a.tmap, 64 * j, y, &full[s]);
          else tma_load_2d_mc(dst, &a.tmap, 64 * j, y, &full[s], a.dest[j]);
        }
      }
    }
  } else if (warp == 1) {
    // MMAs only: stage k as soon as its boxes have landed (no other wait on this path)
    if (lane == 0) {
      uint32_t idesc[2];
#pragma unroll
      for (int t = 0; t < 2; ++t)
        idesc[t] = umma_idesc_bf16(kGM, t < ro.ntile ? ro.n[t] : 128) | (1u << 15) | (1u << 16);  // A, B MN-major
      int consumed = 0;
      for (int k = 0; k < nk; ++k) {
        const int s = k % S;
        if (!mbar_wait(&full[s], (uint32_t)(k / S) & 1u, abort_f, a.status)) break;
        consumed = k + 1;
        tc_fence_after();
        const uint32_t xb = smem_u32(sm + (size_t)s * bstage);
#pragma unroll
        for (int ks = 0; ks < KR / 16; ++ks) {
          const uint32_t acc = (k > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
          for (int t = 0; t < 2; ++t)
            if (t < ro.ntile)
              umma_bf16(tmem + (uint32_t)ro.toff[t],
                        umma_desc_sw128(xb + (uint32_t)(2 * ro.a_blk[t]) * kBox + ks * 2048u, kBox, 1024),
                        umma_desc_sw128(xb + (uint32_t)(ro.b_lo[t] / 64) * kBox + ks * 2048u, kBox, 1024),
                        idesc[t], acc);
        }
        umma_commit(&empty[s]);
      }
      umma_commit(accum);
      *s_consumed = consumed;
    }
  } else if (warp == 2) {
    // releases: buffer s for stage j (its incoming bytes expected, its loaders told) once the MMAs
    // of stage j - S have completed
    if (lane == 0) {
      int released = 0;
      for (int j = 0; j < nk; ++j) {
        const int s = j % S;
        if (j >= S && !mbar_wait(&empty[s], (uint32_t)((j - S) / S) & 1u, abort_f, a.status)) break;
        mbar_arrive_expect_tx(&full[s], (uint32_t)ro.recv_bytes);
        for (int q = 0; q < a.Q; ++q) {
          if (!(ro.feeds >> q & 1u)) continue;
          if (q == rank) mbar_arrive(&slotfree[s]);
          else mbar_arrive_remote(cluster_addr(smem_u32(&slotfree[s]), q));
        }
        released = j + 1;
      }
      *s_released = released;
    }
  } else {
    // epilogue: TMEM lanes 32 q .. 32 q + 31, q = warp mod 4, hold rows 128 a_blk + 32 q + lane
    const bool ok = mbar_wait(accum, 0u, abort_f, a.status);
    tc_fence_after();
    const int q = warp & 3;
    if (__all_sync(0xFFFFFFFFu, ok && !*abort_f) && nk > 0) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t >= ro.ntile) break;
        float *row = a.part + ((int64_t)blockIdx.y * a.ncp + kGM * ro.a_blk[t] + 32 * q + lane) * a.ncp + ro.b_lo[t];
        gram_store(tmem + (uint32_t)ro.toff[t], row, ro.n[t], q, 0, 32);
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  // every copy into this CTA has landed before it exits: after a failure, the stages released but
  // not consumed (the latest phase of their buffers) are awaited, each wait bounded
  if (threadIdx.x == 0) {
    for (int j = *s_consumed; j < *s_released; ++j) {
      volatile int never = 0;
      mbar_wait(&full[j % S], (uint32_t)(j / S) & 1u, &never, a.status);
    }
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// roles of k_gram_w for ncp columns (the table above it); returns Q
int gram_w_roles(int ncp, int box_bytes, GramWArgs &a, bool multicast) {
  GramRole cr[3];
  const int Q = gram_roles(ncp, cr, nullptr);
  a.Q = Q;
  a.nbox = ncp / 64;
  for (int r = 0; r < 3; ++r) {
    GramWRole &w = a.role[r];
    w = GramWRole{};
    if (r >= Q) continue;
    w.ntile = cr[r].ntile;
    for (int t = 0; t < 2; ++t) {
      w.a_blk[t] = cr[r].a_blk[t];
      w.b_lo[t] = cr[r].b_lo[t];
      w.n[t] = cr[r].n[t];
      w.toff[t] = cr[r].toff[t];
    }
  }
  a.mc = multicast && Q > 1 ? 1 : 0;
  for (int j = 0; j < 8; ++j) a.dest[j] = 0;
  if (!a.mc) {
    // every CTA loads the boxes its tiles read (the CTAs of a range run side by side, so the
    // second reader of a box mostly finds it in L2)
    for (int r = 0; r < Q; ++r) {
      GramWRole &w = a.role[r];
      for (int t = 0; t < w.ntile; ++t) {
        for (int c = kGM * w.a_blk[t]; c < kGM * (w.a_blk[t] + 1); c += 64) w.issue |= 1u << (c / 64);
        for (int c = w.b_lo[t]; c < w.b_lo[t] + w.n[t]; c += 64) w.issue |= 1u << (c / 64);
      }
      w.feeds = 1u << r;
      w.nfree = 1;
      w.recv_bytes = __builtin_popcount(w.issue) * box_bytes;
    }
    return Q;
  }
  uint32_t issuer[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (Q == 1) {
    for (int j = 0; j < a.nbox; ++j) { a.dest[j] = 1; issuer[j] = 0; }
  } else if (Q == 2) {
    const int iss[6] = {0, 0, 1, 1, 1, 0};
    for (int j = 0; j < 6; ++j) { a.dest[j] = j < 2 ? 0x1 : 0x3; issuer[j] = (uint32_t)iss[j]; }
  } else {
    const int iss[8] = {1, 1, 1, 0, 2, 2, 2, 0};
    for (int j = 0; j < 8; ++j) { a.dest[j] = j < 4 ? 0x3 : 0x5; issuer[j] = (uint32_t)iss[j]; }
  }
  for (int r = 0; r < Q; ++r) {
    GramWRole &w = a.role[r];
    uint32_t dests = 0;
    for (int j = 0; j < a.nbox; ++j) {
      if ((int)issuer[j] == r) { w.issue |= 1u << j; dests |= a.dest[j]; }
      if (a.dest[j] >> r & 1u) { w.recv_bytes += box_bytes; w.feeds |= 1u << issuer[j]; }
    }
    w.nfree = __builtin_popcount(dests);
  }
  return Q;
}

// shared memory of k_gram_w: S stages of all boxes (the same offsets in every CTA), the barriers
void gram_w_layout(int ncp, int kr, GramWArgs &a, size_t &smem) {
  const int bstage = ncp / 64 * kr * 128;
  int S = 200 * 1024 / bstage;
  if (S > kFMaxB) S = kFMaxB;
  if (S < 2) S = 2;
  a.S = S;
  a.o_bar = S * bstage;
  smem = (size_t)a.o_bar + (3 * kFMaxB + 1) * 8 + 16 + 1024;
  if (smem < 233472 / 2 + 1) smem = 233472 / 2 + 1;
}

}  // namespace

GramPlan gram_plan(int64_t N, int d, int nsm) {
  GramPlan p{};
  p.N = N;
  p.d = d;
  p.ncp = (int)gcdiv(d, kGM) * kGM;
  int tc = 32;
  while (tc < p.ncp) tc <<= 1;
  p.tmem_cols = tc;
  const int mt = p.ncp / kGM;
  // packed path
  const size_t bC = (size_t)p.ncp * kGK * 2;
  int S = (int)((232448 - 2048) / bC);
  if (S > kGMaxStages) S = kGMaxStages;
  p.stages = S;
  size_t smem = (size_t)S * bC + (2 * S + 1) * 8 + 8 + 1024;
  if (smem < 233472 / 2 + 1) smem = 233472 / 2 + 1;  // one CTA per SM
  p.smem = smem;
  p.nchunk = gcdiv(N, 2 * kGK) * 2;  // the packer writes chunks in pairs (zero rows past N)
  gram_split(p.nchunk, mt, nsm, p.cps, p.splits);
  // FP32 path: one cluster of Q CTAs per range
  GramRole ro[3];
  p.q_f = gram_roles(p.ncp, ro, nullptr);
  p.nstage = gcdiv(N, kGK);
  gram_split(p.nstage, p.q_f, nsm, p.cps_f, p.splits_f);
  GramF32Args lay{};
  lay.own = kFOwn ? 1 : 0;
  if (lay.own) gram_own_segments(p.q_f, ro);
  gram_f32_layout(p.ncp, ro, p.q_f, lay, p.smem_f);
  double ent_f = 0.0;  // accumulator entries of one range
  for (int r = 0; r < p.q_f; ++r)
    for (int t = 0; t < ro[r].ntile; ++t) ent_f += (double)kGM * ro[r].n[t];
  const double ent_p = (double)p.ncp * p.ncp;
  p.flops_f32 = 2.0 * (double)p.nstage * kGK * ent_f;
  p.flops_packed = 2.0 * (double)p.nchunk * kGK * ent_p;
  p.bytes_f32 = (double)N * d * 4.0 + 2.0 * (double)p.splits_f * ent_f * 4.0;
  p.bytes_packed = (double)N * d * 4.0 + 2.0 * (double)p.nchunk * kGK * p.ncp * 2.0 + 2.0 * (double)p.splits * ent_p * 4.0;
  const int sp = p.splits > p.splits_f ? p.splits : p.splits_f;
  p.o_xt = 0;
  p.o_part = gal256((size_t)p.nchunk * bC);
  p.o_grp = p.o_part + gal256((size_t)sp * p.ncp * p.ncp * 4);
  p.total = p.o_grp + gal256(gram_grp_bytes(sp, p.ncp));
  return p;
}

namespace {
// X as a 2-D tensor (d columns, N rows, row stride ldx floats) with 128 x 32 boxes; false when the
// driver's encoder is unavailable or refuses
bool gram_tensor_map(CUtensorMap *m, const float *X, int64_t ldx, int64_t N, int d) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    cudaGetLastError();
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)ldx * 4u};
  const cuuint32_t box[2] = {128u, (cuuint32_t)kGK};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

bool gram_fp32_path(const GramPlan &p, const float *X, int64_t ldx) {
  return p.d % 4 == 0 && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
}

cudaError_t launch_gram(const GramPlan &p, const float *X, int64_t ldx, double *G, unsigned *status, void *ws,
                        cudaStream_t s) {
  uint8_t *base = static_cast<uint8_t *>(ws);
  float *part = reinterpret_cast<float *>(base + p.o_part);
  const int mt = p.ncp / kGM;
  cudaError_t e;
  int splits;
  GramF32Args a{};
  if (gram_fp32_path(p, X, ldx) && gram_tensor_map(&a.tmap, X, ldx, p.N, p.d)) {
    if ((e = cudaFuncSetAttribute(k_gram_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem_f))) return e;
    a.N = p.N; a.d = p.d; a.part = part; a.status = status;
    a.nstage = p.nstage; a.cps = p.cps_f; a.ncp = p.ncp; a.tmem_cols = p.tmem_cols;
    a.Q = gram_roles(p.ncp, a.role, &a.in_bytes);
    a.own = kFOwn ? 1 : 0;
    if (a.own) gram_own_segments(a.Q, a.role);
    size_t smem_f = 0;
    gram_f32_layout(p.ncp, a.role, a.Q, a, smem_f);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.Q, (unsigned)p.splits_f);
    cfg.blockDim = dim3(kFThreads);
    cfg.dynamicSmemBytes = p.smem_f;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.own ? 1u : (unsigned)a.Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((e = cudaLaunchKernelEx(&cfg, k_gram_f32, a))) return e;
    splits = p.splits_f;
  } else {
    uint8_t *xt = base + p.o_xt;
    if ((e = launch_pack_bf16(X, ldx, p.N, p.d, p.ncp, xt, s))) return e;
    if ((e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem))) return e;
    GramArgs b{};
    b.xt = xt; b.part = part; b.status = status; b.nchunk = p.nchunk; b.cps = p.cps; b.ncp = p.ncp;
    b.tmem_cols = p.tmem_cols; b.stages = p.stages;
    k_gram_tc<<<dim3((unsigned)mt, (unsigned)p.splits), kGThreads, p.smem, s>>>(b);
    splits = p.splits;
  }
  if ((e = cudaGetLastError())) return e;
  return launch_gram_reduce(part, splits, p.ncp, p.d, 1.0, reinterpret_cast<double *>(base + p.o_grp), status, G, s);
}

GramWPlan gram_w_plan(int64_t rows, int d, int nsm) {
  GramWPlan p{};
  p.rows = rows;
  p.d = d;
  p.ncp = (int)gcdiv(d, kGM) * kGM;
  int tc = 32;
  while (tc < p.ncp) tc <<= 1;
  p.tmem_cols = tc;
  GramWArgs a{};
  p.kr = 64;
  const int Q = gram_w_roles(p.ncp, p.kr * 128, a, kWMulticast);
  p.q = Q;
  p.nstage = gcdiv(rows, p.kr);
  gram_split(p.nstage, Q, nsm, p.cps, p.splits, 8192 / p.kr);
  gram_w_layout(p.ncp, p.kr, a, p.smem);
  double ent = 0.0;
  for (int r = 0; r < Q; ++r)
    for (int t = 0; t < a.role[r].ntile; ++t) ent += (double)kGM * a.role[r].n[t];
  p.o_grp = gal256((size_t)p.splits * p.ncp * p.ncp * 4);
  p.part_bytes = p.o_grp + gal256(gram_grp_bytes(p.splits, p.ncp));
  p.flops = 2.0 * (double)p.nstage * p.kr * ent;
  p.bytes = (double)rows * d * 2.0 + 2.0 * (double)p.splits * ent * 4.0;
  return p;
}

bool gram_w_ok(const GramWPlan &p, const void *B, int64_t ldb) {
  return ldb % 8 == 0 && (reinterpret_cast<uintptr_t>(B) & 15u) == 0 && p.d >= 1 && p.d <= 512;
}

cudaError_t launch_gram_w(const GramWPlan &p, const void *B, int64_t ldb, double scale, double *G, unsigned *status,
                          float *part, cudaStream_t s) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    cudaGetLastError();
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!enc || !gram_w_ok(p, B, ldb)) return cudaErrorInvalidValue;
  GramWArgs a{};
  const cuuint64_t dims[2] = {(cuuint64_t)p.d, (cuuint64_t)p.rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ldb * 2u};
  const cuuint32_t box[2] = {64u, (cuuint32_t)p.kr};
  const cuuint32_t estr[2] = {1u, 1u};
  if (enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(B), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  a.part = part;
  a.status = status;
  a.nstage = p.nstage;
  a.cps = p.cps;
  a.ncp = p.ncp;
  a.tmem_cols = p.tmem_cols;
  gram_w_roles(p.ncp, p.kr * 128, a, kWMulticast);
  size_t smem = 0;
  gram_w_layout(p.ncp, p.kr, a, smem);
  cudaError_t e;
  auto kern = p.kr == 32 ? k_gram_w<32> : k_gram_w<64>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)a.Q, (unsigned)p.splits);
  cfg.blockDim = dim3(kWThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.mc ? (unsigned)a.Q : 1u;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if ((e = cudaLaunchKernelEx(&cfg, kern, a))) return e;
  return launch_gram_reduce(part, p.splits, p.ncp, p.d, scale,
                            reinterpret_cast<double *>(reinterpret_cast<char *>(part) + p.o_grp), status, G, s);
}

}  // namespace slse
