// CountSketch family (paper Sec. 2: the sparse projection whose columns hold one random
// sign in a uniformly random row; Sec. 5 runs SLSE-FRS with it in place of the SRHT).
//
// Definitions (the same as the CPU oracle's, from the paper's description):
//   row k of [X | Y] goes, with sign s(k), to bucket h(k) mod m of the m-row sketch
//   (m a power of two); h(k) = w0 and s(k) = -1 iff bit 0 of w1, with (w0, w1) the
//   Philox4x32-10 words of counter (k, stream 3).  Nested sizes share h, so the smaller
//   sketches are folds of the larger ones.  The Hessian sketch S-hat (r rows) uses an
//   independent hash floor(w0 r / 2^32) and sign from stream 4.  No scale factor.
//
// GB300 design: the data is read once, in whole rows, in bucket order.
//   1. Argsort of the row indices (sort.cuh) by (bit-reversed low L bits of h, index):
//      every bucket of every nested size 2^l <= 2^L is then a contiguous run of the
//      sorted list, with its rows in index order (a fixed summation order).  The
//      Hessian sketch's list is sorted in the same launch.
//   2. Run starts of each group of buckets (k_group_starts).
//   3. Top levels: one warp per (group of 2^F level-L buckets, 256-column chunk)
//      (k_cs_nested).  The warp streams the group's rows through a cp.async ring in
//      shared memory (several rows in flight per warp), forms the level-L bucket sums in
//      FP32 (FP64 on the FP64 path) and folds them pairwise in registers down to level
//      L - F, writing each level's rows; the level L - F sums also go to a scratch
//      buffer at working precision when smaller sizes remain.
//      When the level-L buckets are large (N / 2^L >= 64 rows), one CTA per bucket
//      (k_cs_bucket) instead: its warps sum contiguous slices of the bucket and the
//      partial rows are added in a fixed order.
//   4. Lower levels: level l from level l + 1 by adding rows b and b + 2^l
//      (k_cs_fold), from the working-precision scratch.
//   5. S-hat: k_cs_bucket over the r buckets of the second list.
// Outputs are in natural bucket order (row b of the m-row sketch is bucket b).
#include "sort.cuh"

namespace slse {
namespace {

using sortk::RowKey;

constexpr int kCsStreamNested = 3, kCsStreamHat = 4;

struct CsArgs {
  const void *X;
  int64_t ldx;
  const void *Y;
  int d;
  uint32_t k0, k1;
  int stream;            // sign stream (3 nested, 4 Hessian sketch)
  const int32_t *rows;   // sorted row list
  const int64_t *starts; // group g = rows[starts[g] .. starts[g+1])
  int64_t ngroups;
  int L;                 // nested: bits of the top level
  int F;                 // nested: levels folded in registers below L
  int nested;            // 1: group index is a bit-reversed bucket prefix; 0: Hessian-sketch bucket
  void *outX[25];        // nested: output of level l (rows 2^l, natural order); may be null
  void *outY[25];
  int64_t ldo;
  void *scrX;            // working-precision rows of level L - F (null: not needed)
  void *scrY;
  int64_t lds;
  int vec_in, vec_out;
  int ncw;               // column chunks of kChunkCols per row (1 or 2)
};

__device__ __forceinline__ uint32_t brev_low(uint32_t x, int L) { return L > 0 ? (__brev(x) >> (32 - L)) : 0u; }

template <class Tin, class Tacc, int VEC, int MAXQ>
__device__ __forceinline__ void load_row(const Tin *row, int d, int lane, bool vec, Tacc (&v)[MAXQ][VEC]) {
#pragma unroll
  for (int q = 0; q < MAXQ; ++q) {
    const int e0 = (lane + 32 * q) * VEC;
    if constexpr (VEC == 4 && sizeof(Tin) == 4) {
      if (vec && e0 < d) {
        const float4 t = __ldcs(reinterpret_cast<const float4 *>(row + e0));
        v[q][0] = (Tacc)t.x; v[q][1] = (Tacc)t.y; v[q][2] = (Tacc)t.z; v[q][3] = (Tacc)t.w;
        continue;
      }
    } else if constexpr (VEC == 2 && sizeof(Tin) == 8) {
      if (vec && e0 < d) {
        const double2 t = __ldcs(reinterpret_cast<const double2 *>(row + e0));
        v[q][0] = (Tacc)t.x; v[q][1] = (Tacc)t.y;
        continue;
      }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) v[q][e] = (e0 + e < d) ? (Tacc)row[e0 + e] : Tacc(0);
  }
}

template <class Tout, class Tacc> __device__ __forceinline__ void put(Tout *p, Tacc v) {
  if constexpr (sizeof(Tout) == 2) *p = __float2bfloat16_rn((float)v);
  else *p = (Tout)v;
}

template <class Tout, class Tacc, int VEC, int MAXQ>
__device__ __forceinline__ void store_row(Tout *row, int d, int lane, bool vec, const Tacc (&v)[MAXQ][VEC]) {
#pragma unroll
  for (int q = 0; q < MAXQ; ++q) {
    const int e0 = (lane + 32 * q) * VEC;
    if (e0 >= d) continue;
    if constexpr (sizeof(Tout) == 2 && VEC == 4) {
      if (vec) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn((float)v[q][0], (float)v[q][1]);
        const __nv_bfloat162 hi = __floats2bfloat162_rn((float)v[q][2], (float)v[q][3]);
        uint2 t;
        t.x = *reinterpret_cast<const uint32_t *>(&lo);
        t.y = *reinterpret_cast<const uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(row + e0) = t;
        continue;
      }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e)
      if (e0 + e < d) put(row + e0 + e, v[q][e]);
  }
}

template <class Tacc, int VEC, int MAXQ>
__device__ __forceinline__ void zero(Tacc (&v)[MAXQ][VEC]) {
#pragma unroll
  for (int q = 0; q < MAXQ; ++q)
#pragma unroll
    for (int e = 0; e < VEC; ++e) v[q][e] = Tacc(0);
}

template <class T> __device__ __forceinline__ T *row_ptr(void *base, int64_t ld, int64_t row) {
  return static_cast<T *>(base) + row * ld;
}

// Per-row metadata: (row index, member of its group, sign).
__device__ __forceinline__ void row_meta(const CsArgs &a, int64_t k, int &member, float &sign) {
  const U4 w = philox4x32_10((uint32_t)k, (uint32_t)(k >> 32), (uint32_t)a.stream, 0u, a.k0, a.k1);
  sign = (w.y & 1u) ? -1.f : 1.f;
  member = a.nested ? (int)(brev_low(w.x, a.L) & ((1u << a.F) - 1u)) : 0;
}

// ---------------------------------------------------------------------------------
// Row streaming.  A warp owns a column chunk of kChunkCols columns (rows of d <= 512
// are split in two chunks handled by two warps, which read the two halves of the same
// rows at about the same time).  On the vector path every lane copies its 16-byte pieces
// of a row into its own slots of a per-warp shared-memory ring with cp.async, kRing - 1
// rows ahead of the row being summed, so a warp keeps several rows in flight without
// holding them in registers.  Row indices, signs, members and y values come 32 rows at a
// time (one per lane) and are broadcast by shuffles.
constexpr int kRing = 4;
constexpr int kChunkCols = 256;
constexpr int kWarps = 8;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <class Tin> constexpr int vec_of() { return 16 / (int)sizeof(Tin); }

// Calls on_row(member, sign, y, v) for the rows rows[lo..hi) in order; v holds this lane's
// columns c0 + (lane + 32 q) VEC + e of the row (zero past d).
template <class Tin, class Tacc, class OnRow>
__device__ __forceinline__ void stream_rows(const CsArgs &a, int64_t lo, int64_t hi, int c0, int lane, uint4 *ring,
                                            OnRow &&on_row) {
  constexpr int VEC = vec_of<Tin>();
  constexpr int MAXQ = kChunkCols / (32 * VEC);
  const unsigned FULL = 0xffffffffu;
  const int d = a.d;
  const Tin *X = static_cast<const Tin *>(a.X);
  const Tin *Y = static_cast<const Tin *>(a.Y);
  int64_t kA = 0, kB = 0;
  int mA = 0, mB = 0;
  float sA = 0.f, sB = 0.f;
  Tacc yA = Tacc(0), yB = Tacc(0);
  auto meta = [&](int64_t b, int64_t &k, int &mj, float &sg, Tacc &yv) {
    const int64_t p = b + lane;
    k = 0; mj = 1 << 30; sg = 0.f; yv = Tacc(0);
    if (p < hi) {
      k = a.rows[p];
      row_meta(a, k, mj, sg);
      yv = (Tacc)Y[k];
    }
  };
  int64_t base = lo;
  meta(base, kA, mA, sA, yA);
  meta(base + 32, kB, mB, sB, yB);
  auto row_at = [&](int64_t p) -> int64_t {
    const int off = (int)(p - base);
    return __shfl_sync(FULL, off < 32 ? kA : kB, off & 31);
  };
  const bool vec = a.vec_in != 0;
  auto issue = [&](int64_t p) {
    const int64_t k = row_at(p);
    const int slot = (int)(p % kRing);
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int e0 = c0 + (lane + 32 * q) * VEC;
      if (e0 < d) cp_async16(&ring[(slot * MAXQ + q) * 32 + lane], X + k * a.ldx + e0);
    }
    cp_async_commit();
  };
  if (vec)
    for (int i = 0; i < kRing - 1; ++i) {
      if (lo + i < hi) issue(lo + i);
      else cp_async_commit();
    }
  for (int64_t p = lo; p < hi; ++p) {
    Tacc v[MAXQ][VEC];
    if (vec) {
      if (p + kRing - 1 < hi) issue(p + kRing - 1);
      else cp_async_commit();
      cp_async_wait<kRing - 1>();
      const int slot = (int)(p % kRing);
#pragma unroll
      for (int q = 0; q < MAXQ; ++q) {
        const int e0 = c0 + (lane + 32 * q) * VEC;
        const uint4 t = ring[(slot * MAXQ + q) * 32 + lane];
        if constexpr (sizeof(Tin) == 4) {
          const float f[4] = {__uint_as_float(t.x), __uint_as_float(t.y), __uint_as_float(t.z), __uint_as_float(t.w)};
#pragma unroll
          for (int e = 0; e < VEC; ++e) v[q][e] = e0 < d ? (Tacc)f[e] : Tacc(0);
        } else {
          const double f[2] = {__hiloint2double((int)t.y, (int)t.x), __hiloint2double((int)t.w, (int)t.z)};
#pragma unroll
          for (int e = 0; e < VEC; ++e) v[q][e] = e0 < d ? (Tacc)f[e] : Tacc(0);
        }
      }
    } else {
      const int64_t k = row_at(p);
#pragma unroll
      for (int q = 0; q < MAXQ; ++q) {
        const int e0 = c0 + (lane + 32 * q) * VEC;
#pragma unroll
        for (int e = 0; e < VEC; ++e) v[q][e] = (e0 + e < d) ? (Tacc)X[k * a.ldx + e0 + e] : Tacc(0);
      }
    }
    const int off = (int)(p - base);
    const int mj = __shfl_sync(FULL, off < 32 ? mA : mB, off & 31);
    const float sg = __shfl_sync(FULL, off < 32 ? sA : sB, off & 31);
    const Tacc yv = __shfl_sync(FULL, off < 32 ? yA : yB, off & 31);
    on_row(mj, (Tacc)sg, yv, v);
    if (off == 31) {  // slide the metadata window
      kA = kB; mA = mB; sA = sB; yA = yB;
      base += 32;
      meta(base + 32, kB, mB, sB, yB);
    }
  }
  if (vec) cp_async_wait<0>();
}

template <class Tout, class Tacc, int VEC, int MAXQ>
__device__ __forceinline__ void store_chunk(Tout *row, int d, int c0, int lane, bool vec, const Tacc (&v)[MAXQ][VEC]) {
#pragma unroll
  for (int q = 0; q < MAXQ; ++q) {
    const int e0 = c0 + (lane + 32 * q) * VEC;
    if (e0 >= d) continue;
    if constexpr (sizeof(Tout) == 2 && VEC == 4) {
      if (vec) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn((float)v[q][0], (float)v[q][1]);
        const __nv_bfloat162 hi = __floats2bfloat162_rn((float)v[q][2], (float)v[q][3]);
        uint2 t;
        t.x = *reinterpret_cast<const uint32_t *>(&lo);
        t.y = *reinterpret_cast<const uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(row + e0) = t;
        continue;
      }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e)
      if (e0 + e < d) put(row + e0 + e, v[q][e]);
  }
}

// One warp per (group of 2^F level-L buckets, column chunk); 8 warps per CTA.
template <class Tin, class Tacc, class Tout, int F>
__global__ void __launch_bounds__(256, 2) k_cs_nested(const CsArgs a) {
  constexpr int VEC = vec_of<Tin>();
  constexpr int MAXQ = kChunkCols / (32 * VEC);
  constexpr int NS = F > 0 ? F : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint4 *ring = reinterpret_cast<uint4 *>(smem_raw) + wib * (kRing * MAXQ * 32);
  const int64_t unit = (int64_t)blockIdx.x * kWarps + wib;
  const int64_t g = unit / a.ncw;
  const int chunk = (int)(unit % a.ncw);
  if (g >= a.ngroups) return;
  const int c0 = chunk * kChunkCols;
  const int d = a.d;
  const bool vout = a.vec_out != 0, ylane = chunk == 0 && lane == 0;

  Tacc acc[MAXQ][VEC], stk[NS][MAXQ][VEC];
  Tacc accy = Tacc(0), stky[NS];
  zero(acc);
  int member = 0;  // next level-L bucket of the group to be emitted

  // Emit the level-L bucket `j` of the group (its sum is in acc) and fold it into the
  // pairwise tree: bucket pairs (2t, 2t+1) form level L-1, and so on down to level L-F.
  auto emit = [&](int j) {
    {
      const int64_t b = brev_low((uint32_t)((g << F) | j), a.L);
      if (a.outX[a.L]) {
        store_chunk<Tout, Tacc, VEC, MAXQ>(row_ptr<Tout>(a.outX[a.L], a.ldo, b), d, c0, lane, vout, acc);
        if (ylane) put(static_cast<Tout *>(a.outY[a.L]) + b, accy);
      }
      if (F == 0 && a.scrX) {
        store_chunk<Tacc, Tacc, VEC, MAXQ>(row_ptr<Tacc>(a.scrX, a.lds, b), d, c0, lane, true, acc);
        if (ylane) static_cast<Tacc *>(a.scrY)[b] = accy;
      }
    }
    bool carry = true;
#pragma unroll
    for (int lev = 1; lev <= F; ++lev) {
      if (!carry) break;
      if (((j >> (lev - 1)) & 1) == 0) {
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
#pragma unroll
          for (int e = 0; e < VEC; ++e) stk[lev - 1][q][e] = acc[q][e];
        stky[lev - 1] = accy;
        carry = false;
      } else {
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[q][e] = stk[lev - 1][q][e] + acc[q][e];
        accy = stky[lev - 1] + accy;
        const int l = a.L - lev;
        const int64_t b = brev_low((uint32_t)((g << (F - lev)) | (j >> lev)), l);
        if (a.outX[l]) {
          store_chunk<Tout, Tacc, VEC, MAXQ>(row_ptr<Tout>(a.outX[l], a.ldo, b), d, c0, lane, vout, acc);
          if (ylane) put(static_cast<Tout *>(a.outY[l]) + b, accy);
        }
        if (lev == F && a.scrX) {
          store_chunk<Tacc, Tacc, VEC, MAXQ>(row_ptr<Tacc>(a.scrX, a.lds, b), d, c0, lane, true, acc);
          if (ylane) static_cast<Tacc *>(a.scrY)[b] = accy;
        }
      }
    }
    zero(acc);
    accy = Tacc(0);
  };

  stream_rows<Tin, Tacc>(a, a.starts[g], a.starts[g + 1], c0, lane, ring,
                         [&](int mj, Tacc sg, Tacc yv, const Tacc (&v)[MAXQ][VEC]) {
                           while (member < mj) emit(member++);
#pragma unroll
                           for (int q = 0; q < MAXQ; ++q)
#pragma unroll
                             for (int e = 0; e < VEC; ++e) acc[q][e] += sg * v[q][e];
                           accy += sg * yv;
                         });
  while (member < (1 << F)) emit(member++);
}

// One CTA per bucket: the 8 warps cover (column chunk, row slice) pairs; each sums its
// slice of the bucket's rows in index order, and the slices' partial rows are added in
// slice order.
template <class Tin, class Tacc, class Tout>
__global__ void __launch_bounds__(256) k_cs_bucket(const CsArgs a) {
  constexpr int VEC = vec_of<Tin>();
  constexpr int MAXQ = kChunkCols / (32 * VEC);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint4 *ring = reinterpret_cast<uint4 *>(smem_raw) + w * (kRing * MAXQ * 32);
  Tacc *part = reinterpret_cast<Tacc *>(reinterpret_cast<uint4 *>(smem_raw) + kWarps * kRing * MAXQ * 32);  // [slices][513]
  const int ncw = a.ncw, nsl = kWarps / a.ncw;
  const int chunk = w % ncw, slice = w / ncw;
  const int c0 = chunk * kChunkCols;
  const int64_t g = blockIdx.x;
  const int d = a.d;
  const int64_t lo = a.starts[g], hi = a.starts[g + 1];
  const int64_t len = (hi - lo + nsl - 1) / nsl;
  const int64_t s0 = lo + slice * len < hi ? lo + slice * len : hi;
  const int64_t s1 = s0 + len < hi ? s0 + len : hi;

  Tacc acc[MAXQ][VEC];
  Tacc accy = Tacc(0);
  zero(acc);
  stream_rows<Tin, Tacc>(a, s0, s1, c0, lane, ring, [&](int, Tacc sg, Tacc yv, const Tacc (&v)[MAXQ][VEC]) {
#pragma unroll
    for (int q = 0; q < MAXQ; ++q)
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[q][e] += sg * v[q][e];
    accy += sg * yv;
  });
#pragma unroll
  for (int q = 0; q < MAXQ; ++q)
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int c = c0 + (lane + 32 * q) * VEC + e;
      if (c < d) part[slice * 513 + c] = acc[q][e];
    }
  if (chunk == 0 && lane == 0) part[slice * 513 + 512] = accy;
  __syncthreads();
  const int64_t b = a.nested ? (int64_t)brev_low((uint32_t)g, a.L) : g;
  for (int c = threadIdx.x; c <= 512; c += blockDim.x) {
    if (c < d || c == 512) {
      Tacc sum = Tacc(0);
      for (int u = 0; u < nsl; ++u) sum += part[u * 513 + c];
      if (c < d) {
        void *o = a.nested ? a.outX[a.L] : a.outX[0];
        if (o) put(row_ptr<Tout>(o, a.ldo, b) + c, sum);
        if (a.scrX) row_ptr<Tacc>(a.scrX, a.lds, b)[c] = sum;
      } else {
        void *o = a.nested ? a.outY[a.L] : a.outY[0];
        if (o) put(static_cast<Tout *>(o) + b, sum);
        if (a.scrY) static_cast<Tacc *>(a.scrY)[b] = sum;
      }
    }
  }
}

// Level with m rows from the level with 2m rows: out[b] = in[b] + in[b + m].
template <class Tacc, class Tout>
__global__ void k_cs_fold(const Tacc *in, const Tacc *in_y, int64_t lds, int64_t m, int d, Tacc *nx, Tacc *ny,
                          Tout *ox, Tout *oy, int64_t ldo) {
  const int64_t n = m * (int64_t)(d + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / (d + 1);
    const int c = (int)(i - b * (d + 1));
    if (c < d) {
      const Tacc s = in[b * lds + c] + in[(b + m) * lds + c];
      if (nx) nx[b * lds + c] = s;
      if (ox) put(ox + b * ldo + c, s);
    } else {
      const Tacc s = in_y[b] + in_y[b + m];
      if (ny) ny[b] = s;
      if (oy) put(oy + b, s);
    }
  }
}

// Group starts of a sorted list: group of position p = top `gbits` bits of its key
// (nested) or its Hessian-sketch bucket.  starts[g] = first position of group g;
// starts[ngroups] = n.  Every entry is written exactly once.
__global__ void k_group_starts(RowKey key, const int32_t *rows, int64_t n, int gbits, int hat, int64_t ngroups,
                               int64_t *starts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > n) return;
  auto gid = [&](int64_t q) -> int64_t {
    const unsigned long long k = sortk::row_key(key, rows[q]);
    if (hat) return key.rb > 0 ? (int64_t)(k >> (64 - key.rb)) : 0;
    return gbits > 0 ? (int64_t)(k >> (64 - gbits)) : 0;
  };
  const int64_t cur = p < n ? gid(p) : ngroups;
  const int64_t prev = p > 0 ? gid(p - 1) : -1;
  for (int64_t s = prev + 1; s <= cur; ++s) starts[s] = p;
}

inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct CsWs {
  sortk::SortArrays w;
  int32_t *rows[2];
  int64_t *starts[2];
  void *scr[2];     // working-precision level scratch (double buffer)
  void *scr_y[2];
};

}  // namespace

CsPlan cs_plan(int64_t N, int d, int prec, int64_t m_min, int64_t m_max, int64_t r) {
  CsPlan p{};
  p.N = N;
  p.d = d;
  p.prec = prec;
  p.r = r;
  p.L = m_max > 0 ? sortk::bits_for(m_max) : -1;
  p.l1 = m_min > 0 ? sortk::bits_for(m_min) : -1;
  p.big = p.L >= 0 && N >= (int64_t(64) << p.L);
  p.F = 0;
  if (p.L >= 0 && !p.big) {  // levels folded in registers: 4 (FP32 sums), 1 (FP64 sums)
    const int fmax = prec == SLSE_PREC_FP64 ? 1 : 4;
    p.F = p.L - p.l1 < fmax ? p.L - p.l1 : fmax;
    if (p.F < 0) p.F = 0;
  }
  p.ib = sortk::bits_for(N);
  p.Bn = p.L >= 0 ? (sortk::bits_for(N) > 10 ? sortk::bits_for(N) - 10 : 0) : 0;
  p.rb = r > 0 ? sortk::bits_for(r) : 0;
  p.Bh = 0;
  if (r > 0) {  // expected rows of a non-empty bucket <= 1024
    while (p.Bh < 24) {
      const double used = p.Bh <= p.rb ? (double)r / (double)(int64_t(1) << (p.rb - p.Bh))
                                       : (double)r * (double)(int64_t(1) << (p.Bh - p.rb));
      if ((double)N / (used < 1.0 ? 1.0 : used) <= 1024.0) break;
      ++p.Bh;
    }
  }
  const size_t acc = prec == SLSE_PREC_FP64 ? 8 : 4;
  p.lds = (d + 7) & ~int64_t(7);
  const int64_t scr_rows = (p.L >= 0 && p.L - p.F > p.l1) ? (int64_t(1) << (p.L - p.F)) : 0;
  p.o_sort0 = 0;
  p.o_sort1 = p.o_sort0 + al(sortk::sort_ws_bytes(N, p.Bn));
  p.o_rows0 = p.o_sort1 + al(sortk::sort_ws_bytes(r > 0 ? N : 1, p.Bh));
  p.o_rows1 = p.o_rows0 + al(4 * (size_t)N);
  const int64_t ng0 = p.L >= 0 ? (int64_t(1) << (p.L - p.F)) : 1;
  p.o_st0 = p.o_rows1 + al(4 * (size_t)N);
  p.o_st1 = p.o_st0 + al(8 * (size_t)(ng0 + 1));
  p.o_scr0 = p.o_st1 + al(8 * (size_t)(r + 2));
  p.o_scr1 = p.o_scr0 + al((size_t)scr_rows * (p.lds + 1) * acc);
  p.total = p.o_scr1 + al((size_t)(scr_rows / 2) * (p.lds + 1) * acc);
  return p;
}

namespace {

template <class Tin, class Tacc, class Tout, int F>
cudaError_t launch_nested(const CsArgs &a, int64_t nunits, cudaStream_t s) {
  constexpr int MAXQ = kChunkCols / (32 * vec_of<Tin>());
  const size_t smem = (size_t)kWarps * kRing * MAXQ * 32 * sizeof(uint4);
  auto kern = k_cs_nested<Tin, Tacc, Tout, F>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)((nunits + kWarps - 1) / kWarps), 32 * kWarps, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Tin, class Tacc, class Tout>
cudaError_t launch_bucket(const CsArgs &a, int64_t nbuckets, cudaStream_t s) {
  constexpr int MAXQ = kChunkCols / (32 * vec_of<Tin>());
  const size_t smem = (size_t)kWarps * kRing * MAXQ * 32 * sizeof(uint4) + (size_t)kWarps * 513 * sizeof(Tacc);
  auto kern = k_cs_bucket<Tin, Tacc, Tout>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)nbuckets, 32 * kWarps, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Tin, class Tacc, class Tout, int VEC>
cudaError_t run_cs(const CsPlan &pl, const void *X, int64_t ldx, const void *Y, uint64_t seed,
                   void *const *lvX, void *const *lvY, int64_t ldo, void *hatX, void *hatY, int64_t ldh,
                   void *ws, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  const int64_t N = pl.N;
  const int d = pl.d;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  int32_t *rows0 = reinterpret_cast<int32_t *>(base + pl.o_rows0);
  int32_t *rows1 = reinterpret_cast<int32_t *>(base + pl.o_rows1);
  int64_t *st0 = reinterpret_cast<int64_t *>(base + pl.o_st0);
  int64_t *st1 = reinterpret_cast<int64_t *>(base + pl.o_st1);
  const bool nested = pl.L >= 0;
  const bool hat = pl.r > 0;

  // 1. both sorted lists
  sortk::SortArrays w{};
  RowKey kn{sortk::KEY_CS_NESTED, kCsStreamNested, k0, k1, nested ? pl.L : 0, 0u, 0, pl.ib};
  RowKey kh{sortk::KEY_CS_HAT, kCsStreamHat, k0, k1, 0, (uint32_t)(hat ? pl.r : 1), pl.rb, pl.ib};
  w.key[0] = kn;
  w.key[1] = kh;
  sortk::carve_sort(w, 0, base + pl.o_sort0, nested ? N : 0, pl.Bn);
  sortk::carve_sort(w, 1, base + pl.o_sort1, hat ? N : 0, pl.Bh);
  w.out[0] = rows0;
  w.out[1] = rows1;
  cudaError_t e = sortk::launch_sort_pair(w, s);
  if (e != cudaSuccess) return e;

  const int T = 256;
  CsArgs a{};
  a.X = X; a.ldx = ldx; a.Y = Y; a.d = d; a.k0 = k0; a.k1 = k1;
  a.ldo = ldo; a.lds = pl.lds;
  auto vec_ok = [](const void *p, int64_t ld, size_t eb, int v) {
    return reinterpret_cast<uintptr_t>(p) % (v * eb) == 0 && ld % v == 0;
  };
  a.vec_in = (d % VEC == 0 && vec_ok(X, ldx, sizeof(Tin), VEC)) ? 1 : 0;
  a.ncw = (d + kChunkCols - 1) / kChunkCols;

  if (nested) {
    // 2. group starts, 3. top levels
    const int gbits = pl.L - pl.F;
    const int64_t ng = int64_t(1) << gbits;
    k_group_starts<<<(unsigned)((N + 1 + T - 1) / T), T, 0, s>>>(kn, rows0, N, gbits, 0, ng, st0);
    a.stream = kCsStreamNested;
    a.rows = rows0; a.starts = st0; a.ngroups = ng; a.L = pl.L; a.F = pl.F; a.nested = 1;
    bool vout = true;
    for (int l = 0; l <= 24; ++l) {
      a.outX[l] = lvX ? lvX[l] : nullptr;
      a.outY[l] = lvY ? lvY[l] : nullptr;
      if (a.outX[l] && !vec_ok(a.outX[l], ldo, sizeof(Tout), VEC)) vout = false;
    }
    a.vec_out = (vout && d % VEC == 0) ? 1 : 0;
    const bool folds = pl.L - pl.F > pl.l1;
    a.scrX = folds ? base + pl.o_scr0 : nullptr;
    a.scrY = folds ? static_cast<void *>(static_cast<Tacc *>(a.scrX) + (int64_t(1) << (pl.L - pl.F)) * pl.lds) : nullptr;
    if (pl.big) {
      e = launch_bucket<Tin, Tacc, Tout>(a, ng, s);
    } else {
      const int64_t nunits = ng * a.ncw;
      if constexpr (sizeof(Tacc) == 8) {
        if (pl.F == 0) e = launch_nested<Tin, Tacc, Tout, 0>(a, nunits, s);
        else e = launch_nested<Tin, Tacc, Tout, 1>(a, nunits, s);
      } else {
        switch (pl.F) {
          case 0: e = launch_nested<Tin, Tacc, Tout, 0>(a, nunits, s); break;
          case 1: e = launch_nested<Tin, Tacc, Tout, 1>(a, nunits, s); break;
          case 2: e = launch_nested<Tin, Tacc, Tout, 2>(a, nunits, s); break;
          case 3: e = launch_nested<Tin, Tacc, Tout, 3>(a, nunits, s); break;
          default: e = launch_nested<Tin, Tacc, Tout, 4>(a, nunits, s); break;
        }
      }
    }
    if (e != cudaSuccess) return e;
    // 4. lower levels by folding the scratch
    if (folds) {
      Tacc *cx = static_cast<Tacc *>(a.scrX), *cy = static_cast<Tacc *>(a.scrY);
      Tacc *bufx[2] = {cx, reinterpret_cast<Tacc *>(base + pl.o_scr1)};
      for (int l = pl.L - pl.F - 1, bsel = 1; l >= pl.l1; --l, bsel ^= 1) {
        const int64_t m = int64_t(1) << l;
        Tacc *nx = (l > pl.l1) ? bufx[bsel] : nullptr;
        Tacc *ny = nx ? nx + m * pl.lds : nullptr;
        const int64_t n = m * (d + 1);
        unsigned grid = (unsigned)((n + T - 1) / T);
        if (grid > 65535u * 8u) grid = 65535u * 8u;
        k_cs_fold<Tacc, Tout><<<grid, T, 0, s>>>(cx, cy, pl.lds, m, d, nx, ny,
                                                 lvX ? static_cast<Tout *>(lvX[l]) : nullptr,
                                                 lvY ? static_cast<Tout *>(lvY[l]) : nullptr, ldo);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cx = nx;
        cy = ny;
      }
    }
  }
  if (hat) {
    k_group_starts<<<(unsigned)((N + 1 + T - 1) / T), T, 0, s>>>(kh, rows1, N, 0, 1, pl.r, st1);
    CsArgs h = a;
    h.stream = kCsStreamHat;
    h.rows = rows1; h.starts = st1; h.ngroups = pl.r; h.L = 0; h.F = 0; h.nested = 0;
    for (int l = 0; l <= 24; ++l) { h.outX[l] = nullptr; h.outY[l] = nullptr; }
    h.outX[0] = hatX; h.outY[0] = hatY; h.ldo = ldh;
    h.scrX = nullptr; h.scrY = nullptr;
    h.vec_out = 0;
    if ((e = launch_bucket<Tin, Tacc, Tout>(h, pl.r, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_countsketch(const CsPlan &pl, int xdtype, const void *X, int64_t ldx, const void *Y, uint64_t seed,
                               void *const *lvX, void *const *lvY, int64_t ldo, void *hatX, void *hatY, int64_t ldh,
                               void *ws, cudaStream_t s) {
  using bf16 = __nv_bfloat16;
  if (pl.d < 1 || pl.d > 512) return cudaErrorInvalidValue;
  if (pl.prec == SLSE_PREC_FP64) {
    if (xdtype == SLSE_F64)
      return run_cs<double, double, double, 2>(pl, X, ldx, Y, seed, lvX, lvY, ldo, hatX, hatY, ldh, ws, s);
    return run_cs<float, double, double, 4>(pl, X, ldx, Y, seed, lvX, lvY, ldo, hatX, hatY, ldh, ws, s);
  }
  if (pl.prec == SLSE_PREC_MIXED_BF16 && xdtype == SLSE_F32)
    return run_cs<float, float, bf16, 4>(pl, X, ldx, Y, seed, lvX, lvY, ldo, hatX, hatY, ldh, ws, s);
  return cudaErrorInvalidValue;
}

}  // namespace slse
