// Per-segment median/MAD normalisation and power (paper §2.2.3, Eq. 8).
//
// One CTA of 256 threads per segment (normalisation block).  The block's
// complex bins are staged into shared memory by one TMA bulk copy (or read
// from global memory when the block is too large for shared memory).  The
// real and imaginary parts are normalised separately, as Eq. 8 prescribes,
// with EXACT order statistics found by a value-bucket select that serves both
// components at once:
//   * bucket b(x) = floor((x - lo) * scale) over the block's [lo, hi] is
//     non-decreasing in x (each step is a monotone rounding), so the rank-r
//     element lies in the bucket where the cumulative count passes r;
//   * one histogram pass (2048 buckets per component), one block-wide scan,
//     one gather pass of the target bucket(s) -- a handful of values for
//     noise -- and one warp per component ranks them;
//   * if a target bucket is crowded (a block dominated by a strong tone) the
//     select refines it level by level: the bucket's [min, max] becomes the
//     next range and only its elements are bucketed again; a range with
//     min == max means every remaining candidate is equal.
// An even count takes the mean of ranks n/2-1 and n/2.  The MAD is the same
// select on |x - median|, whose range [0, max deviation] follows from the
// median pass.  Then a = (x - med) / (kappa MAD), kappa = 1/Phi^{-1}(3/4),
// and P = (a^2 + b^2)/2, written coalesced.  The DC bin of a series is taken
// as 0 + 0i.  A segment whose MAD is 0 gets P = 0.  On request the kernel
// also records the selected order statistics (the two middle values of each
// component and of its deviations), which the adjoint needs.
//
// The paper's GPU version estimates the median by median-of-medians (§2.5);
// this kernel keeps the exact median of the CPU version, which the FP32 and
// FP64 results can then agree on to rounding.
#include <algorithm>

#include "common.cuh"
#include "ptx.cuh"

namespace ps {

namespace {

constexpr double kKappa = 1.482602218505602;  // 1 / Phi^{-1}(3/4)
constexpr int kMaxSmemBins = 16384 + 4096;     // float2 elements staged in shared memory
constexpr int kStoreBins = 8192;               // blocks up to this size keep their bucket indices
constexpr int kBuckets = kHistBins;            // value buckets per level
constexpr int kPerThread = kBuckets / (kNormThreads / 2);   // buckets per scanning thread
constexpr int kCap = 256;                      // values ranked directly
constexpr int kMaxLevels = 8;
constexpr int kWarpsN = kNormThreads / 32;

template <int NT>
struct SelSharedT {
  uint32_t hist[2][kBuckets];
  uint32_t wsum[2][NT / 64];
  float red[NT / 32][4];
  float lo[kMaxLevels][2], scale[kMaxLevels][2];
  uint32_t b1[kMaxLevels][2], b2[kMaxLevels][2];
  uint32_t rank[2], below[2], cnt[2], list_n[2];
  float list[2][kCap];
  float res[2][2];
  float mm[4];     // block min0, min1, max0, max1
  int done[2];
  uint32_t flag;
};
using SelShared = SelSharedT<kNormThreads>;

__device__ __forceinline__ uint32_t bucket_of(float x, float lo, float scale) {
  const float t = (x - lo) * scale;
  return min(static_cast<uint32_t>(fmaxf(t, 0.0f)), static_cast<uint32_t>(kBuckets - 1));
}

__device__ __forceinline__ float bucket_scale(float lo, float hi) {
  // shrink a hair so that hi stays in the last bucket
  return (hi > lo) ? static_cast<float>(kBuckets) / (hi - lo) * (1.0f - 1.0f / 4096.0f) : 0.0f;
}

// Block min/max of both components over the values cand(e, v0, c0, v1, c1)
// flags as candidates; result in sh.mm.
template <int NT, class Cand>
__device__ __forceinline__ void block_minmax(SelSharedT<NT> &sh, Cand cand, int n) {
  float a0 = INFINITY, a1 = INFINITY, z0 = -INFINITY, z1 = -INFINITY;
  for (int e = threadIdx.x; e < n; e += NT) {
    float v0, v1;
    bool c0, c1;
    cand(e, v0, c0, v1, c1);
    if (c0) { a0 = fminf(a0, v0); z0 = fmaxf(z0, v0); }
    if (c1) { a1 = fminf(a1, v1); z1 = fmaxf(z1, v1); }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 = fminf(a0, __shfl_xor_sync(0xffffffffu, a0, o));
    a1 = fminf(a1, __shfl_xor_sync(0xffffffffu, a1, o));
    z0 = fmaxf(z0, __shfl_xor_sync(0xffffffffu, z0, o));
    z1 = fmaxf(z1, __shfl_xor_sync(0xffffffffu, z1, o));
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh.red[wid][0] = a0;
    sh.red[wid][1] = a1;
    sh.red[wid][2] = z0;
    sh.red[wid][3] = z1;
  }
  __syncthreads();
  if (wid == 0 && lane < 4) {
    // lane k reduces column k over the warps
    float r = (lane < 2) ? INFINITY : -INFINITY;
    for (int w = 0; w < NT / 32; ++w) r = (lane < 2) ? fminf(r, sh.red[w][lane]) : fmaxf(r, sh.red[w][lane]);
    sh.mm[lane] = r;
  }
  __syncthreads();
}

// Block-wide scan of both histograms: threads [0, 128) scan component 0,
// [128, 256) component 1, kPerThread consecutive buckets each (summed in a
// skewed order to spread banks).  Writes the buckets holding ranks r and
// r + pair, the count below the first and the cumulative count through the
// second.
template <int NT>
__device__ __forceinline__ void scan_find(SelSharedT<NT> &sh, int level, bool pair) {
  constexpr int kPer = kBuckets / (NT / 2);   // buckets per scanning thread
  const int c = threadIdx.x / (NT / 2);
  const int t = threadIdx.x % (NT / 2);
  const uint32_t *h = sh.hist[c] + kPer * t;
  uint32_t local = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) local += h[(j + t) & (kPer - 1)];
  const int lane = t & 31, wid = t >> 5;
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) sh.wsum[c][wid] = incl;
  __syncthreads();
  uint32_t base = 0;
  for (int j = 0; j < wid; ++j) base += sh.wsum[c][j];
  const uint32_t excl = base + incl - local;
  const uint32_t r1 = sh.rank[c];
  const uint32_t r2 = r1 + (pair ? 1u : 0u);
  if (!sh.done[c] && ((r1 >= excl && r1 < excl + local) || (r2 >= excl && r2 < excl + local))) {
    uint32_t acc = excl;
    for (int j = 0; j < kPer; ++j) {
      const uint32_t nxt = acc + h[j];
      if (r1 >= acc && r1 < nxt) {
        sh.b1[level][c] = kPer * t + j;
        sh.below[c] = acc;
      }
      if (r2 >= acc && r2 < nxt) {
        sh.b2[level][c] = kPer * t + j;
        sh.cnt[c] = nxt;
      }
      acc = nxt;
    }
  }
  __syncthreads();
}

// One warp per component ranks its gathered list (ties by list position)
// and stores the values of ranks `want` and `want + 1`.
template <class Sh>
__device__ __forceinline__ void rank_lists(Sh &sh, const bool (&active)[2], bool pair) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 2 && active[warp]) {
    const int c = warp;
    const uint32_t m = sh.list_n[c];
    const uint32_t want = sh.rank[c] - sh.below[c];
    for (uint32_t i = lane; i < m; i += 32) {
      const float v = sh.list[c][i];
      uint32_t rk = 0;
      for (uint32_t f = 0; f < m; ++f) {
        const float u = sh.list[c][f];
        rk += (u < v || (u == v && f < i)) ? 1u : 0u;
      }
      if (rk == want) sh.res[c][0] = v;
      if (pair && rk == want + 1) sh.res[c][1] = v;
    }
  }
  __syncthreads();
}

// Ranks r and r + 1 in different buckets b1 < b2 (every bucket between them
// empty): rank r is the largest value of bucket b1 and rank r + 1 the
// smallest of bucket b2.  Block reduction of those two per component from
// each thread's contributions; results to res[c][0..1] where split[c].
template <int NW, class Sh>
__device__ __forceinline__ void split_pair(Sh &sh, const bool (&split)[2], float x0, float x1, float n0, float n1) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x0 = fmaxf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    n0 = fminf(n0, __shfl_xor_sync(0xffffffffu, n0, o));
    n1 = fminf(n1, __shfl_xor_sync(0xffffffffu, n1, o));
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh.red[wid][0] = x0;
    sh.red[wid][1] = x1;
    sh.red[wid][2] = n0;
    sh.red[wid][3] = n1;
  }
  __syncthreads();
  if (threadIdx.x < 2 && split[threadIdx.x]) {
    const int c = threadIdx.x;
    float hi = -INFINITY, lo = INFINITY;
    for (int w = 0; w < NW; ++w) {
      hi = fmaxf(hi, sh.red[w][c]);
      lo = fminf(lo, sh.red[w][2 + c]);
    }
    sh.res[c][0] = hi;
    sh.res[c][1] = lo;
  }
  __syncthreads();
}

// Multi-level select (the general path): get(e, v0, v1) gives element e's
// two component values; level 0 starts from the whole block.
template <int NT, class Get>
__device__ void select_levels(SelSharedT<NT> &sh, Get get, int n, uint32_t rank, bool pair,
                                           float (&out_lo)[2], float (&out_hi)[2]) {
  if (threadIdx.x < 2) {
    sh.rank[threadIdx.x] = rank;
    sh.done[threadIdx.x] = 0;
  }
  __syncthreads();
  auto cand = [&](int e, float &v0, bool &c0, float &v1, bool &c1, int levels) {
    get(e, v0, v1);
    c0 = !sh.done[0];
    c1 = !sh.done[1];
    for (int L = 0; L < levels; ++L) {
      if (c0) {
        const uint32_t b = bucket_of(v0, sh.lo[L][0], sh.scale[L][0]);
        c0 = b >= sh.b1[L][0] && b <= sh.b2[L][0];
      }
      if (c1) {
        const uint32_t b = bucket_of(v1, sh.lo[L][1], sh.scale[L][1]);
        c1 = b >= sh.b1[L][1] && b <= sh.b2[L][1];
      }
    }
  };
  for (int level = 0; level < kMaxLevels; ++level) {
    block_minmax(sh, [&](int e, float &v0, bool &c0, float &v1, bool &c1) { cand(e, v0, c0, v1, c1, level); }, n);
    if (threadIdx.x < 2) {
      const int c = threadIdx.x;
      sh.list_n[c] = 0u;
      if (!sh.done[c]) {
        const float mn = sh.mm[c], mx = sh.mm[2 + c];
        if (!(mx > mn)) {
          sh.res[c][0] = mn;   // every remaining candidate has this value
          sh.res[c][1] = mn;
          sh.done[c] = 1;
        } else {
          sh.lo[level][c] = mn;
          sh.scale[level][c] = bucket_scale(mn, mx);
        }
      }
    }
    for (int j = threadIdx.x; j < 2 * kBuckets; j += NT) (&sh.hist[0][0])[j] = 0u;
    __syncthreads();
    if (sh.done[0] && sh.done[1]) break;
    for (int e = threadIdx.x; e < n; e += NT) {
      float v0, v1;
      bool c0, c1;
      cand(e, v0, c0, v1, c1, level);
      if (c0) atomicAdd(&sh.hist[0][bucket_of(v0, sh.lo[level][0], sh.scale[level][0])], 1u);
      if (c1) atomicAdd(&sh.hist[1][bucket_of(v1, sh.lo[level][1], sh.scale[level][1])], 1u);
    }
    __syncthreads();
    scan_find<NT>(sh, level, pair);
    bool split[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) split[c] = !sh.done[c] && pair && sh.b1[level][c] != sh.b2[level][c];
    if (split[0] || split[1]) {
      float x0 = -INFINITY, x1 = -INFINITY, n0 = INFINITY, n1 = INFINITY;
      for (int e = threadIdx.x; e < n; e += NT) {
        float v0, v1;
        bool c0, c1;
        cand(e, v0, c0, v1, c1, level);
        if (c0 && split[0]) {
          const uint32_t b = bucket_of(v0, sh.lo[level][0], sh.scale[level][0]);
          if (b == sh.b1[level][0]) x0 = fmaxf(x0, v0);
          if (b == sh.b2[level][0]) n0 = fminf(n0, v0);
        }
        if (c1 && split[1]) {
          const uint32_t b = bucket_of(v1, sh.lo[level][1], sh.scale[level][1]);
          if (b == sh.b1[level][1]) x1 = fmaxf(x1, v1);
          if (b == sh.b2[level][1]) n1 = fminf(n1, v1);
        }
      }
      split_pair<NT / 32>(sh, split, x0, x1, n0, n1);
      if (threadIdx.x < 2 && split[threadIdx.x]) sh.done[threadIdx.x] = 1;
      __syncthreads();
      if (sh.done[0] && sh.done[1]) break;
    }
    bool gather[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) gather[c] = !sh.done[c] && (sh.cnt[c] - sh.below[c] <= static_cast<uint32_t>(kCap));
    if (gather[0] || gather[1]) {
      for (int e = threadIdx.x; e < n; e += NT) {
        float v0, v1;
        bool c0, c1;
        cand(e, v0, c0, v1, c1, level + 1);   // includes this level's [b1, b2]
        if (c0 && gather[0]) sh.list[0][atomicAdd(&sh.list_n[0], 1u)] = v0;
        if (c1 && gather[1]) sh.list[1][atomicAdd(&sh.list_n[1], 1u)] = v1;
      }
      __syncthreads();
      rank_lists(sh, gather, pair);
    }
    if (threadIdx.x < 2) {
      const int c = threadIdx.x;
      if (gather[c]) sh.done[c] = 1;
      else if (!sh.done[c]) sh.rank[c] -= sh.below[c];   // the next level refines [b1, b2]
    }
    __syncthreads();
    if (sh.done[0] && sh.done[1]) break;
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    out_lo[c] = sh.res[c][0];
    out_hi[c] = pair ? sh.res[c][1] : sh.res[c][0];
  }
  __syncthreads();
}

// Level-0 select for both components over the known range [lo, hi]:
// histogram (keeping each element's packed bucket indices in `bkt` when it is
// given), scan, gather, rank.  Returns false, having decided nothing, when a
// target bucket holds more than kCap values.
template <class Get>
__device__ __forceinline__ bool select_fast(SelShared &sh, Get get, uint32_t *bkt, int n, uint32_t rank, bool pair,
                                            float lo0, float lo1, float hi0, float hi1, float (&out_lo)[2],
                                            float (&out_hi)[2]) {
  const float s0 = bucket_scale(lo0, hi0), s1 = bucket_scale(lo1, hi1);
  const bool flat0 = !(hi0 > lo0), flat1 = !(hi1 > lo1);
  for (int j = threadIdx.x; j < 2 * kBuckets; j += kNormThreads) (&sh.hist[0][0])[j] = 0u;
  if (threadIdx.x < 2) {
    sh.rank[threadIdx.x] = rank;
    sh.done[threadIdx.x] = 0;
    sh.list_n[threadIdx.x] = 0u;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += kNormThreads) {
    float v0, v1;
    get(e, v0, v1);
    const uint32_t q0 = bucket_of(v0, lo0, s0), q1 = bucket_of(v1, lo1, s1);
    atomicAdd(&sh.hist[0][q0], 1u);
    atomicAdd(&sh.hist[1][q1], 1u);
    if (bkt) bkt[e] = q0 | (q1 << 16);
  }
  __syncthreads();
  scan_find<kNormThreads>(sh, 0, pair);
  if ((!flat0 && sh.cnt[0] - sh.below[0] > static_cast<uint32_t>(kCap)) ||
      (!flat1 && sh.cnt[1] - sh.below[1] > static_cast<uint32_t>(kCap))) {
    __syncthreads();
    return false;
  }
  // a flat component (all values equal) gathers nothing: its answer is lo
  const uint32_t l0 = flat0 ? 1u : sh.b1[0][0], h0 = flat0 ? 0u : sh.b2[0][0];
  const uint32_t l1 = flat1 ? 1u : sh.b1[0][1], h1 = flat1 ? 0u : sh.b2[0][1];
  for (int e = threadIdx.x; e < n; e += kNormThreads) {
    float v0, v1;
    uint32_t q0, q1;
    if (bkt) {
      const uint32_t q = bkt[e];
      q0 = q & 0xffffu;
      q1 = q >> 16;
    } else {
      get(e, v0, v1);
      q0 = bucket_of(v0, lo0, s0);
      q1 = bucket_of(v1, lo1, s1);
    }
    const bool g0 = q0 >= l0 && q0 <= h0, g1 = q1 >= l1 && q1 <= h1;
    if (g0 || g1) {
      get(e, v0, v1);
      if (g0) sh.list[0][atomicAdd(&sh.list_n[0], 1u)] = v0;
      if (g1) sh.list[1][atomicAdd(&sh.list_n[1], 1u)] = v1;
    }
  }
  __syncthreads();
  const bool active[2] = {!flat0, !flat1};
  rank_lists(sh, active, pair);
  out_lo[0] = flat0 ? lo0 : sh.res[0][0];
  out_lo[1] = flat1 ? lo1 : sh.res[1][0];
  out_hi[0] = flat0 ? lo0 : (pair ? sh.res[0][1] : sh.res[0][0]);
  out_hi[1] = flat1 ? lo1 : (pair ? sh.res[1][1] : sh.res[1][0]);
  __syncthreads();
  return true;
}

__device__ __forceinline__ float mean_of(float a, float b) {
  return static_cast<float>(0.5 * (static_cast<double>(a) + static_cast<double>(b)));
}

// The block's statistic from its selected order statistics (the mean of the
// two middle values for an even count), worked out in FP64 by one thread and
// broadcast through bc: FP64 runs at a small fraction of the FP32 rate, so
// the whole block must not repeat it.  The next write to bc comes after
// further barriers, so one barrier suffices.
__device__ __forceinline__ void bcast_mid(float *bc, const float (&lo)[2], const float (&hi)[2], bool even,
                                          float &a, float &b) {
  if (threadIdx.x == 0) {
    bc[0] = even ? mean_of(lo[0], hi[0]) : lo[0];
    bc[1] = even ? mean_of(lo[1], hi[1]) : lo[1];
  }
  __syncthreads();
  a = bc[0];
  b = bc[1];
}

// 1 / (kappa MAD) of both components (0 for a degenerate block), one thread in FP64.
__device__ __forceinline__ void bcast_inv(float *bc, float mad_re, float mad_im, float &inv_re, float &inv_im) {
  if (threadIdx.x == 0) {
    const bool degenerate = !(mad_re > 0.0f) || !(mad_im > 0.0f);
    bc[2] = degenerate ? 0.0f : static_cast<float>(1.0 / (kKappa * static_cast<double>(mad_re)));
    bc[3] = degenerate ? 0.0f : static_cast<float>(1.0 / (kKappa * static_cast<double>(mad_im)));
  }
  __syncthreads();
  inv_re = bc[2];
  inv_im = bc[3];
}

__global__ void __launch_bounds__(kNormThreads) normalise_kernel(
    const float2 *__restrict__ spec, float *__restrict__ power, float4 *__restrict__ stats,
    const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off, int n_series, int seg_len,
    uint32_t *__restrict__ counters, int smem_bins, float *__restrict__ sel) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  SelShared &sh = *reinterpret_cast<SelShared *>(smem_raw + 128);
  unsigned char *tail = smem_raw + 128 + ((sizeof(SelShared) + 127) & ~size_t(127));
  float2 *data = reinterpret_cast<float2 *>(tail);
  uint32_t *bkt_store = reinterpret_cast<uint32_t *>(tail + 8 * static_cast<size_t>(smem_bins));

  const int64_t g = blockIdx.x;
  int lo = 0, hi = n_series - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const SeriesDev S = series[lo];
  const int64_t sl = g - S.seg_off;
  const int64_t b0 = sl * seg_len;
  const int64_t b1 = (sl == S.n_seg - 1) ? S.m : b0 + seg_len;
  const int n = static_cast<int>(b1 - b0);
  const float2 *src = spec + S.spec_off + b0;
  const bool in_smem = n <= smem_bins;
  // bucket indices are kept only where the launch reserved room for them
  uint32_t *bkt = (in_smem && smem_bins <= kStoreBins) ? bkt_store : nullptr;

  if (in_smem) {
    // float2 pairs: a 16-byte multiple from a 16-byte aligned source
    const int n_tma = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0u) ? (n & ~1) : 0;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && n_tma > 0) {
      mbar_arrive_expect_tx(bar, static_cast<uint32_t>(n_tma) * 8u);
      tma_load_1d(data, src, static_cast<uint32_t>(n_tma) * 8u, bar);
    }
    for (int e = n_tma + threadIdx.x; e < n; e += kNormThreads) data[e] = src[e];
    // one thread waits on the copy (bounded); the others sleep in the barrier
    if (threadIdx.x == 0) sh.flag = (n_tma == 0 || mbar_wait_bounded(bar, 0, 2000000000ull)) ? 1u : 0u;
    __syncthreads();
    if (sh.flag == 0u) {
      if (threadIdx.x == 0) atomicOr(counters + 2, kErrTimeout);
      return;
    }
    if (b0 == 0 && threadIdx.x == 0) data[0] = make_float2(0.0f, 0.0f);   // DC := 0
    __syncthreads();
  }
  const bool dc_here = (b0 == 0);
  auto val = [&](int e) -> float2 {
    if (in_smem) return data[e];
    if (dc_here && e == 0) return make_float2(0.0f, 0.0f);
    return src[e];
  };

  const bool even = (n % 2) == 0;
  const uint32_t rank = even ? static_cast<uint32_t>(n / 2 - 1) : static_cast<uint32_t>(n / 2);

  // range of both components
  block_minmax(sh,
               [&](int e, float &v0, bool &c0, float &v1, bool &c1) {
                 const float2 v = val(e);
                 v0 = v.x;
                 v1 = v.y;
                 c0 = c1 = true;
               },
               n);
  const float mn0 = sh.mm[0], mn1 = sh.mm[1], mx0 = sh.mm[2], mx1 = sh.mm[3];
  __syncthreads();

  // medians
  auto raw = [&](int e, float &v0, float &v1) {
    const float2 v = val(e);
    v0 = v.x;
    v1 = v.y;
  };
  float lo_v[2], hi_v[2];
  if (!select_fast(sh, raw, bkt, n, rank, even, mn0, mn1, mx0, mx1, lo_v, hi_v))
    select_levels(sh, raw, n, rank, even, lo_v, hi_v);
  float med_re, med_im;
  bcast_mid(sh.mm, lo_v, hi_v, even, med_re, med_im);
  if (sel != nullptr && threadIdx.x == 0) {
    // the selected order statistics, for the adjoint of the median
    sel[8 * g + 0] = lo_v[0];
    sel[8 * g + 1] = hi_v[0];
    sel[8 * g + 4] = lo_v[1];
    sel[8 * g + 5] = hi_v[1];
  }

  // MADs: the same selection on |x - med|, over [0, max deviation]
  auto dev = [&](int e, float &v0, float &v1) {
    const float2 v = val(e);
    v0 = fabsf(v.x - med_re);
    v1 = fabsf(v.y - med_im);
  };
  const float dh0 = fmaxf(fabsf(mx0 - med_re), fabsf(med_re - mn0));
  const float dh1 = fmaxf(fabsf(mx1 - med_im), fabsf(med_im - mn1));
  if (!select_fast(sh, dev, bkt, n, rank, even, 0.0f, 0.0f, dh0, dh1, lo_v, hi_v))
    select_levels(sh, dev, n, rank, even, lo_v, hi_v);
  float mad_re, mad_im;
  bcast_mid(sh.mm, lo_v, hi_v, even, mad_re, mad_im);
  if (sel != nullptr && threadIdx.x == 0) {
    // the selected deviations, for the adjoint of the MAD
    sel[8 * g + 2] = lo_v[0];
    sel[8 * g + 3] = hi_v[0];
    sel[8 * g + 6] = lo_v[1];
    sel[8 * g + 7] = hi_v[1];
  }

  float inv_re, inv_im;
  bcast_inv(sh.mm, mad_re, mad_im, inv_re, inv_im);
  float *out = power + S.p_off + b0;
  for (int e = threadIdx.x; e < n; e += kNormThreads) {
    const float2 v = val(e);
    const float a = (v.x - med_re) * inv_re;
    const float b = (v.y - med_im) * inv_im;
    out[e] = 0.5f * (a * a + b * b);
  }
  if (threadIdx.x == 0 && stats != nullptr) stats[g] = make_float4(med_re, mad_re, med_im, mad_im);
}

// ---------------------------------------------------------------------------
// Lean register kernel: one CTA of NT threads per block of up to NT K + 1
// bins.  Thread t holds bins t, t + NT, ..., t + (K - 1) NT in registers,
// and thread 0 also bin NT K when the block has that one more bin (the last
// block of a power-of-two series ends with the Nyquist bin).  A block with
// fewer bins fills its missing slots with pads: the block maximum for the
// median and the largest deviation for the MAD, which leaves every order
// statistic of rank below n where it is.  Both selects of a block run the
// same exact value-bucket select over both components at once:
//   (1) a histogram over 1024 value buckets: the bucket of x is the low bits
//       of fma(x, s, magic - lo s) with magic = 1.5 2^23 (whose ulp is 1), so
//       one multiply-add of those bits forms the shared-memory address of a
//       fire-and-forget red.shared.add;
//   (2) a block-wide scan finds the bucket(s) holding ranks r and r + 1;
//   (3) every thread appends its values in those buckets to a short list;
//   (4) one warp per component ranks its list and forms the statistic (the
//       FP64 mean of the two middle values for an even count; for the MAD
//       also 1 / (kappa MAD)).
// The MAD's values are the deviations x - med, formed once in place (the
// histogram and the gather take their absolute value as an operand
// modifier); the power is formed from the same registers.  The bucket map is
// monotone (one rounding of an exact x s + off) and lands in [0, 1022] while
// the offset magic - lo s is a float of integer resolution (|.| < 2^24) and s
// is finite; a block outside that (a tight cluster far from zero, an
// infinity or NaN) or with more than kLeanCap values in its target buckets (a
// block dominated by a strong tone) takes the multi-level select, which
// re-reads the block from global memory.  Nine block barriers per block.
constexpr int kLeanBuckets = 1024;
constexpr int kLeanGuard = 8;                     // unused buckets on each side of the map's range
constexpr int kLeanRow = kLeanBuckets + 2 * kLeanGuard;
constexpr int kLeanCap = 128;                     // gathered values ranked directly, per component
constexpr float kBucketMagic = 12582912.0f;       // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;      // its bit pattern

template <int NT>
struct LeanShared {
  uint32_t hist[2][2][kLeanRow];   // [median, MAD][component]
  float4 red[NT / 32];             // per-warp min0, min1, max0, max1
  float list[2][kLeanCap];
  uint32_t list_n[2];
  uint32_t b1[2], b2[2], below[2], through[2];
  uint32_t wsum[2][NT / 64];       // the bucket scan's per-warp totals
  float res[2][2];                 // selected order statistics (rank r, rank r + 1)
  float stat[2];                   // median or MAD per component
  float inv[2];                    // 1 / (kappa MAD), 0 if MAD = 0
};

struct LeanScale {
  float s, off;
};

__device__ __forceinline__ LeanScale lean_scale(float lo, float hi) {
  const float s = (hi > lo) ? 1022.0f / (hi - lo) : 0.0f;
  return LeanScale{s, fmaf(-lo, s, kBucketMagic)};
}

// The map x -> fma(x, s, off) is exact to one rounding at integer
// resolution, so monotone with values in [magic, magic + 1022] for x in
// [lo, hi]; false (NaN included) where that does not hold.
__device__ __forceinline__ bool lean_exact(const LeanScale &sc) {
  return sc.s < INFINITY && fabsf(sc.off) < 16777216.0f;
}

__device__ __forceinline__ void red_inc_shared(uint32_t addr) {
  asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
}

// NaN-propagating minimum / maximum (a NaN anywhere in a block sends it to
// the multi-level select).
__device__ __forceinline__ float nmin(float a, float b) {
  float r;
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float nmax(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float warp_nmin(float v) {
  float r;
  asm volatile("redux.sync.min.NaN.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float warp_nmax(float v) {
  float r;
  asm volatile("redux.sync.max.NaN.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}

// One exact select of ranks `rank` (and rank + 1 when `pair`) of both
// components over [lo, hi] from this thread's K register values (their
// absolute values with kAbs) and the extra value fx when has_x.
// hist[sel] must be zero and visible.  On return (after a barrier) every
// thread holds the order statistics in olo / ohi, and sh.stat the statistic
// (with sh.inv for the MAD, sel = 1); false (decided by the whole block,
// no statistic written) when the fast path does not apply.
template <int NT, int K, bool kAbs>
__device__ __forceinline__ bool lean_select(LeanShared<NT> &sh, int sel, const float2 (&v)[K], bool has_x, float2 fx,
                                            uint32_t rank, bool pair, const float (&lo)[2], const float (&hi)[2],
                                            float (&olo)[2], float (&ohi)[2]) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const LeanScale s0 = lean_scale(lo[0], hi[0]), s1 = lean_scale(lo[1], hi[1]);
  const bool flat0 = !(hi[0] > lo[0]), flat1 = !(hi[1] > lo[1]);
  // (a non-flat range needs s > 0: with s = 0 an infinite value would map to NaN)
  if (!lean_exact(s0) || !lean_exact(s1) || (!flat0 && !(s0.s > 0.0f)) || (!flat1 && !(s1.s > 0.0f))) return false;
  auto val = [&](int j) -> float2 { return kAbs ? make_float2(fabsf(v[j].x), fabsf(v[j].y)) : v[j]; };
  if (kAbs) fx = make_float2(fabsf(fx.x), fabsf(fx.y));
  if (t < 2) {   // this select's gather state (the previous select is done with it)
    sh.list_n[t] = 0u;
    sh.b1[t] = 0xffffffffu;
    sh.b2[t] = 0xffffffffu;
  }
  const uint32_t hb0 = smem_addr(&sh.hist[sel][0][kLeanGuard]) - 4u * kMagicBits;
  const uint32_t hb1 = smem_addr(&sh.hist[sel][1][kLeanGuard]) - 4u * kMagicBits;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float2 f = val(j);
    red_inc_shared(hb0 + 4u * __float_as_uint(fmaf(f.x, s0.s, s0.off)));
    red_inc_shared(hb1 + 4u * __float_as_uint(fmaf(f.y, s1.s, s1.off)));
  }
  if (has_x) {
    red_inc_shared(hb0 + 4u * __float_as_uint(fmaf(fx.x, s0.s, s0.off)));
    red_inc_shared(hb1 + 4u * __float_as_uint(fmaf(fx.y, s1.s, s1.off)));
  }
  __syncthreads();
  {
    // block-wide scan: thread t sums kPer consecutive buckets of component
    // t / (NT / 2); a warp scan and the per-warp totals give each thread its
    // range of ranks, and the threads holding ranks r and r + 1 record their
    // buckets
    constexpr int kPer = 2 * kLeanBuckets / NT;
    const int c = t / (NT / 2), tt = t % (NT / 2);
    const int sl = tt & 31, sw = tt >> 5;
    const uint32_t *h = &sh.hist[sel][c][kLeanGuard + kPer * tt];
    uint32_t hv[kPer], local = 0;
    if constexpr (kPer % 4 == 0) {
#pragma unroll
      for (int q = 0; q < kPer; q += 4) {
        const uint4 u = *reinterpret_cast<const uint4 *>(h + q);
        hv[q] = u.x;
        hv[q + 1] = u.y;
        hv[q + 2] = u.z;
        hv[q + 3] = u.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < kPer; ++q) hv[q] = h[q];
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) local += hv[q];
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (sl >= o) incl += u;
    }
    if (sl == 31) sh.wsum[c][sw] = incl;
    __syncthreads();
    uint32_t acc = incl - local;
    for (int w = 0; w < sw; ++w) acc += sh.wsum[c][w];
    const uint32_t r1 = rank, r2 = rank + (pair ? 1u : 0u);
    if ((r1 - acc < local) || (r2 - acc < local)) {
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const uint32_t nxt = acc + hv[q];
        if (r1 >= acc && r1 < nxt) {
          sh.b1[c] = kPer * tt + q;
          sh.below[c] = acc;
        }
        if (r2 >= acc && r2 < nxt) {
          sh.b2[c] = kPer * tt + q;
          sh.through[c] = nxt;
        }
        acc = nxt;
      }
    }
  }
  __syncthreads();
  // every thread classifies both components: a flat range (all values
  // equal: nothing to gather), few enough values to gather, or the slow path
  uint32_t base0 = 0u, span0 = 0u, base1 = 0u, span1 = 0u;
  bool fast = true;
  if (!flat0) {
    const uint32_t b1 = sh.b1[0], b2 = sh.b2[0];
    fast = fast && b2 != 0xffffffffu && sh.through[0] - sh.below[0] <= static_cast<uint32_t>(kLeanCap);
    base0 = kMagicBits + b1;
    span0 = b2 - b1;
  }
  if (!flat1) {
    const uint32_t b1 = sh.b1[1], b2 = sh.b2[1];
    fast = fast && b2 != 0xffffffffu && sh.through[1] - sh.below[1] <= static_cast<uint32_t>(kLeanCap);
    base1 = kMagicBits + b1;
    span1 = b2 - b1;
  }
  if (!fast) return false;
  auto append = [&](int c, float x) {
    const uint32_t i = atomicAdd(&sh.list_n[c], 1u);
    if (i < static_cast<uint32_t>(kLeanCap)) sh.list[c][i] = x;
  };
  // a flat component's map is the constant magic: never within [base, base + span] = [0, 0]
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float2 f = val(j);
    if (__float_as_uint(fmaf(f.x, s0.s, s0.off)) - base0 <= span0) append(0, f.x);
    if (__float_as_uint(fmaf(f.y, s1.s, s1.off)) - base1 <= span1) append(1, f.y);
  }
  if (has_x) {
    if (__float_as_uint(fmaf(fx.x, s0.s, s0.off)) - base0 <= span0) append(0, fx.x);
    if (__float_as_uint(fmaf(fx.y, s1.s, s1.off)) - base1 <= span1) append(1, fx.y);
  }
  __syncthreads();
  if (warp < 2) {
    const int c = warp;
    if (c ? !flat1 : !flat0) {
      const uint32_t m = min(sh.list_n[c], static_cast<uint32_t>(kLeanCap));
      const uint32_t want = rank - sh.below[c];
      for (uint32_t i = lane; i < m; i += 32) {
        const float x = sh.list[c][i];
        uint32_t rk = 0;
        for (uint32_t f = 0; f < m; ++f) {
          const float u = sh.list[c][f];
          rk += (u < x || (u == x && f < i)) ? 1u : 0u;
        }
        if (rk == want) sh.res[c][0] = x;
        if (pair && rk == want + 1) sh.res[c][1] = x;
      }
    } else if (lane == 0) {
      sh.res[c][0] = lo[c];
      sh.res[c][1] = lo[c];
    }
    __syncwarp();
    if (lane == 0) {
      const float a = sh.res[c][0], b = pair ? sh.res[c][1] : a;
      const float st = pair ? mean_of(a, b) : a;
      sh.stat[c] = st;
      if (sel == 1) sh.inv[c] = (st > 0.0f) ? static_cast<float>(1.0 / (kKappa * static_cast<double>(st))) : 0.0f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    olo[c] = sh.res[c][0];
    ohi[c] = pair ? sh.res[c][1] : sh.res[c][0];
  }
  return true;
}

// The multi-level select over the block in global memory: the raw values
// (dev = false) or their deviations |x - c| (dev = true): the rare path.
// Inlined: an out-of-line call measured slower (2^23 series 48 against 36 us),
// its register saves around the call included.
template <int NT>
__device__ __forceinline__ void lean_fallback(SelSharedT<NT> &sh, const float2 *src, bool dc_here, int n, uint32_t rank,
                                           bool pair, bool dev, float c0, float c1, float *out) {
  float lo_v[2], hi_v[2];
  __syncthreads();
  select_levels<NT>(sh, [&](int e, float &v0, float &v1) {
    const float2 f = (dc_here && e == 0) ? make_float2(0.0f, 0.0f) : src[e];
    v0 = dev ? fabsf(f.x - c0) : f.x;
    v1 = dev ? fabsf(f.y - c1) : f.y;
  }, n, rank, pair, lo_v, hi_v);
  out[0] = lo_v[0];
  out[1] = lo_v[1];
  out[2] = hi_v[0];
  out[3] = hi_v[1];
}

template <int NT, int K>
constexpr int lean_min_blocks() {
  return NT == 1024 ? 1 : (K <= 8 ? 5 : 4);
}

template <int NT, int K>
__global__ void __launch_bounds__(NT, lean_min_blocks<NT, K>()) normalise_lean_kernel(
    const float2 *__restrict__ spec, float *__restrict__ power, float4 *__restrict__ stats,
    const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off, int n_series, int seg_len,
    float *__restrict__ sel, int64_t seg_base, float4 *__restrict__ norm) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  LeanShared<NT> &sh = *reinterpret_cast<LeanShared<NT> *>(smem_raw);
  SelSharedT<NT> &legacy = *reinterpret_cast<SelSharedT<NT> *>(smem_raw);   // the fallback's (same memory)
  const int64_t g = seg_base + blockIdx.x;
  int lo_s = 0, hi_s = n_series - 1;
  while (lo_s < hi_s) {
    const int mid = (lo_s + hi_s + 1) >> 1;
    if (seg_off[mid] <= g) lo_s = mid; else hi_s = mid - 1;
  }
  const SeriesDev S = series[lo_s];
  const int64_t sl = g - S.seg_off;
  const int64_t b0 = sl * seg_len;
  const int n = static_cast<int>(((sl == S.n_seg - 1) ? S.m : b0 + seg_len) - b0);   // <= NT K + 1
  const float2 *src = spec + S.spec_off + b0;
  const int t = threadIdx.x;
  constexpr int kFull = NT * K;
  const bool dc_here = (b0 == 0);
  const bool full = n >= kFull;
  const int nv = full ? K : ((t < n) ? (n - 1 - t) / NT + 1 : 0);
  // the block's first value stands in for missing slots in the range pass
  const float2 first = dc_here ? make_float2(0.0f, 0.0f) : __ldg(src);
  float2 v[K];
  if (full) {
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = __ldg(src + j * NT + t);
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = (j < nv) ? __ldg(src + j * NT + t) : first;
  }
  if (dc_here && t == 0) v[0] = make_float2(0.0f, 0.0f);   // DC := 0
  const bool has_x = (t == 0) && (n > kFull);
  float2 vx = has_x ? __ldg(src + kFull) : first;

  // both selects' histograms zeroed while the loads are in flight
  {
    uint4 *hz = reinterpret_cast<uint4 *>(&sh.hist[0][0][0]);
    constexpr int kWords16 = static_cast<int>(sizeof(sh.hist) / 16);
    for (int i = t; i < kWords16; i += NT) hz[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  // range of both components (a NaN propagates)
  float a0 = nmin(v[0].x, vx.x), a1 = nmin(v[0].y, vx.y), z0 = nmax(v[0].x, vx.x), z1 = nmax(v[0].y, vx.y);
#pragma unroll
  for (int j = 1; j < K; ++j) {
    a0 = nmin(a0, v[j].x);
    a1 = nmin(a1, v[j].y);
    z0 = nmax(z0, v[j].x);
    z1 = nmax(z1, v[j].y);
  }
  a0 = warp_nmin(a0);
  a1 = warp_nmin(a1);
  z0 = warp_nmax(z0);
  z1 = warp_nmax(z1);
  if ((t & 31) == 0) sh.red[t >> 5] = make_float4(a0, a1, z0, z1);
  __syncthreads();
  float mn[2], mx[2];
  {
    float4 r = sh.red[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
      const float4 q = sh.red[w];
      r = make_float4(nmin(r.x, q.x), nmin(r.y, q.y), nmax(r.z, q.z), nmax(r.w, q.w));
    }
    mn[0] = r.x;
    mn[1] = r.y;
    mx[0] = r.z;
    mx[1] = r.w;
  }
  const bool even = (n % 2) == 0;
  const uint32_t rank = even ? static_cast<uint32_t>(n / 2 - 1) : static_cast<uint32_t>(n / 2);
  if (!full) {
    // pads at the block maximum: no order statistic of rank < n moves
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j >= nv) v[j] = make_float2(mx[0], mx[1]);
  }
  float lo_v[2], hi_v[2];
  float med[2], mad[2], inv[2];
  float fb[4];
  bool fell_back = false;
  if (lean_select<NT, K, false>(sh, 0, v, has_x, vx, rank, even, mn, mx, lo_v, hi_v)) {
    med[0] = sh.stat[0];
    med[1] = sh.stat[1];
  } else {
    lean_fallback<NT>(legacy, src, dc_here, n, rank, even, false, 0.0f, 0.0f, fb);
    lo_v[0] = fb[0];
    lo_v[1] = fb[1];
    hi_v[0] = fb[2];
    hi_v[1] = fb[3];
    med[0] = even ? mean_of(lo_v[0], hi_v[0]) : lo_v[0];
    med[1] = even ? mean_of(lo_v[1], hi_v[1]) : lo_v[1];
    fell_back = true;
  }
  if (sel != nullptr && t == 0) {
    sel[8 * g + 0] = lo_v[0];
    sel[8 * g + 1] = hi_v[0];
    sel[8 * g + 4] = lo_v[1];
    sel[8 * g + 5] = hi_v[1];
  }
  if (fell_back) {
    // the fallback used the shared memory: zero the MAD histogram again
    __syncthreads();
    uint32_t *hz = &sh.hist[1][0][0];
    for (int j = t; j < 2 * kLeanRow; j += NT) hz[j] = 0u;
    __syncthreads();
  }
  // deviations x - med in place; pads at the largest deviation
#pragma unroll
  for (int j = 0; j < K; ++j) {
    v[j].x -= med[0];
    v[j].y -= med[1];
  }
  vx.x -= med[0];
  vx.y -= med[1];
  const float dlo[2] = {0.0f, 0.0f};
  const float dhi[2] = {fmaxf(fabsf(mx[0] - med[0]), fabsf(mn[0] - med[0])),
                        fmaxf(fabsf(mx[1] - med[1]), fabsf(mn[1] - med[1]))};
  if (!full) {
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j >= nv) v[j] = make_float2(dhi[0], dhi[1]);
  }
  if (lean_select<NT, K, true>(sh, 1, v, has_x, vx, rank, even, dlo, dhi, lo_v, hi_v)) {
    mad[0] = sh.stat[0];
    mad[1] = sh.stat[1];
    inv[0] = sh.inv[0];
    inv[1] = sh.inv[1];
  } else {
    lean_fallback<NT>(legacy, src, dc_here, n, rank, even, true, med[0], med[1], fb);
    lo_v[0] = fb[0];
    lo_v[1] = fb[1];
    hi_v[0] = fb[2];
    hi_v[1] = fb[3];
    mad[0] = even ? mean_of(lo_v[0], hi_v[0]) : lo_v[0];
    mad[1] = even ? mean_of(lo_v[1], hi_v[1]) : lo_v[1];
    inv[0] = mad[0] > 0.0f ? static_cast<float>(1.0 / (kKappa * static_cast<double>(mad[0]))) : 0.0f;
    inv[1] = mad[1] > 0.0f ? static_cast<float>(1.0 / (kKappa * static_cast<double>(mad[1]))) : 0.0f;
  }
  if (sel != nullptr && t == 0) {
    sel[8 * g + 2] = lo_v[0];
    sel[8 * g + 3] = hi_v[0];
    sel[8 * g + 6] = lo_v[1];
    sel[8 * g + 7] = hi_v[1];
  }
  // a block with either MAD zero is degenerate: P = 0
  if (!(inv[0] > 0.0f) || !(inv[1] > 0.0f)) {
    inv[0] = 0.0f;
    inv[1] = 0.0f;
  }
  // the power (unless only the statistics are wanted: power == nullptr)
  if (power != nullptr) {
    float *out = power + S.p_off + b0;
    if (full) {
#pragma unroll
      for (int j = 0; j < K; ++j) out[j * NT + t] = power_of_dev(v[j].x, v[j].y, inv[0], inv[1]);
    } else {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < nv) out[j * NT + t] = power_of_dev(v[j].x, v[j].y, inv[0], inv[1]);
    }
    if (has_x) out[kFull] = power_of_dev(vx.x, vx.y, inv[0], inv[1]);
  }
  if (t == 0 && stats != nullptr) stats[g] = make_float4(med[0], mad[0], med[1], mad[1]);
  if (t == 0 && norm != nullptr) norm[g] = make_float4(med[0], inv[0], med[1], inv[1]);
}

// Kernel shapes (threads, bins per thread) of the lean register kernel, by
// block size: a shape takes blocks of up to NT K + 1 bins.  (128-thread CTAs
// with twice the bins per thread measured slower: the batch of 2048-bin
// blocks 7.6 against 6.8 ms.)
struct LeanShape {
  int nt, k;
};
constexpr LeanShape kLeanShapes[] = {{256, 1}, {256, 2}, {256, 4}, {256, 6}, {256, 8},
                                     {256, 12}, {256, 16}, {1024, 8}, {1024, 12}, {1024, 16}};

int64_t largest_block(pulscan_plan p) {
  int64_t max_n = 0;
  for (int64_t i = 0; i < p->n_base; ++i) {
    const auto &se = p->series[i];
    max_n = std::max<int64_t>(max_n, se.m - (se.n_seg - 1) * p->seg_len);
  }
  return max_n;
}

// (threads, bins per thread) of the lean kernel for the plan's largest
// block, or (0, 0) for the staged kernel.
void lean_shape(pulscan_plan p, int *nt, int *k) {
  const int64_t max_n = largest_block(p);
  *nt = 0;
  *k = 0;
  for (const LeanShape &s : kLeanShapes) {
    if (max_n <= static_cast<int64_t>(s.nt) * s.k + 1) {
      *nt = s.nt;
      *k = s.k;
      return;
    }
  }
}

template <int NT>
constexpr int lean_smem() {
  return static_cast<int>(sizeof(LeanShared<NT>) > sizeof(SelSharedT<NT>) ? sizeof(LeanShared<NT>)
                                                                          : sizeof(SelSharedT<NT>));
}

// Segments [seg_lo, seg_lo + n_seg) of the series (all of them by default).
template <int NT, int K>
void launch_lean(pulscan_plan p, const float *d_spec, float *d_power, float4 *st4, float *d_sel, cudaStream_t s,
                 int64_t seg_lo = 0, int64_t n_seg = -1, float4 *norm = nullptr) {
  if (n_seg < 0) n_seg = p->base_seg;
  normalise_lean_kernel<NT, K><<<static_cast<unsigned>(n_seg), NT, lean_smem<NT>(), s>>>(
      reinterpret_cast<const float2 *>(d_spec), d_power, st4, p->d_series, p->d_seg_off,
      static_cast<int>(p->n_base), p->seg_len, d_sel, seg_lo, norm);
}

int normalise_smem(pulscan_plan p, int *bins_out) {
  int64_t max_n = 0;
  for (int64_t i = 0; i < p->n_base; ++i) {
    const auto &se = p->series[i];
    const int64_t last = se.m - (se.n_seg - 1) * p->seg_len;
    max_n = std::max<int64_t>(max_n, last);
  }
  const int bins = static_cast<int>(std::min<int64_t>(max_n, kMaxSmemBins));
  const int store = (bins <= kStoreBins) ? bins : 0;
  if (bins_out) *bins_out = bins;
  return 128 + static_cast<int>((sizeof(SelShared) + 127) & ~size_t(127)) + 8 * bins + 4 * store;
}

static int dispatch_lean(pulscan_plan p, int nt, int k, const float *d_spec, float *d_power, float4 *st4,
                         float *d_sel, cudaStream_t s, int64_t seg_lo, int64_t n_seg, float4 *norm = nullptr) {
  switch (nt * 100 + k) {
  case 25601: launch_lean<256, 1>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 25602: launch_lean<256, 2>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 25604: launch_lean<256, 4>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 25606: launch_lean<256, 6>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 25608: launch_lean<256, 8>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 25612: launch_lean<256, 12>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 25616: launch_lean<256, 16>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 102408: launch_lean<1024, 8>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 102412: launch_lean<1024, 12>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  case 102416: launch_lean<1024, 16>(p, d_spec, d_power, st4, d_sel, s, seg_lo, n_seg, norm); break;
  default: return 0;
  }
  return nt;
}

}  // namespace

SmemLimit g_lim_norm;

int prepare_normalise(pulscan_plan p) { return ensure_smem(normalise_kernel, normalise_smem(p, nullptr), g_lim_norm); }

bool normalise_range_ok(pulscan_plan p) {
  int nt = 0, k = 0;
  lean_shape(p, &nt, &k);
  return nt > 0 && p->fidelity != PULSCAN_FIDELITY_PAPER_GPU;
}

// Segments [seg_lo, seg_lo + n_seg) only, with the lean kernel (a part of a
// pipelined batch); PULSCAN_ERR_UNSUPPORTED where the plan's blocks need the
// staged kernel or another mode.
int launch_normalise_range(pulscan_plan p, const float *d_spec, float *d_power, int64_t seg_lo, int64_t n_seg,
                           cudaStream_t s) {
  if (p->fidelity == PULSCAN_FIDELITY_PAPER_GPU || n_seg > 0x7fffffffLL)
    return fail(PULSCAN_ERR_UNSUPPORTED, "no range launch in this mode");
  if (n_seg <= 0) return PULSCAN_OK;
  int nt = 0, k = 0;
  lean_shape(p, &nt, &k);
  if (nt == 0 || dispatch_lean(p, nt, k, d_spec, d_power, reinterpret_cast<float4 *>(p->d_stats), nullptr, s, seg_lo,
                               n_seg) == 0)
    return fail(PULSCAN_ERR_UNSUPPORTED, "blocks too large for the register kernel");
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

// The block statistics alone, as (med_re, 1 / (kappa MAD_re), med_im,
// 1 / (kappa MAD_im)) per segment into p->d_norm (both inverses 0 for a
// degenerate block), for the fused search; the median / MAD pairs into
// p->d_stats as usual.  Register kernel only.
int launch_normalise_stats(pulscan_plan p, const float *d_spec, cudaStream_t s) {
  if (!normalise_range_ok(p) || p->base_seg > 0x7fffffffLL)
    return fail(PULSCAN_ERR_UNSUPPORTED, "blocks too large for the register kernel");
  int nt = 0, k = 0;
  lean_shape(p, &nt, &k);
  if (dispatch_lean(p, nt, k, d_spec, nullptr, reinterpret_cast<float4 *>(p->d_stats), nullptr, s, 0, p->base_seg,
                    reinterpret_cast<float4 *>(p->d_norm)) == 0)
    return fail(PULSCAN_ERR_UNSUPPORTED, "blocks too large for the register kernel");
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

int launch_normalise(pulscan_plan p, const float *d_spec, float *d_power, float *d_stats, cudaStream_t s) {
  return launch_normalise_sel(p, d_spec, d_power, d_stats, nullptr, s);
}

int launch_normalise_sel(pulscan_plan p, const float *d_spec, float *d_power, float *d_stats, float *d_sel,
                         cudaStream_t s) {
  if (p->fidelity == PULSCAN_FIDELITY_PAPER_GPU) {
    if (d_sel != nullptr) return fail(PULSCAN_ERR_UNSUPPORTED, "no adjoint for the median-of-medians statistics");
    return launch_normalise_mom(p, d_spec, d_power, d_stats, s);
  }
  if (p->base_seg > 0x7fffffffLL) return fail(PULSCAN_ERR_UNSUPPORTED, "too many segments");
  float4 *st4 = d_stats ? reinterpret_cast<float4 *>(d_stats) : reinterpret_cast<float4 *>(p->d_stats);
  int nt = 0, k = 0;
  lean_shape(p, &nt, &k);
  nt = dispatch_lean(p, nt, k, d_spec, d_power, st4, d_sel, s, 0, -1);
  if (nt > 0) {
    PS_CUDA(cudaGetLastError());
    return PULSCAN_OK;
  }
  int bins = 0;
  const int smem = normalise_smem(p, &bins);
  if (p->total_seg > 0x7fffffffLL) return fail(PULSCAN_ERR_UNSUPPORTED, "too many segments");
  const int rc = ensure_smem(normalise_kernel, smem, g_lim_norm);
  if (rc) return rc;
  float4 *st = d_stats ? reinterpret_cast<float4 *>(d_stats) : reinterpret_cast<float4 *>(p->d_stats);
  normalise_kernel<<<static_cast<unsigned>(p->base_seg), kNormThreads, smem, s>>>(
      reinterpret_cast<const float2 *>(d_spec), d_power, st, p->d_series, p->d_seg_off,
      static_cast<int>(p->n_base), p->seg_len, p->d_counters, bins, d_sel);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // namespace ps
