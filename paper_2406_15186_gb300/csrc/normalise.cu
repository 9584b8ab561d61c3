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

struct SelShared {
  uint32_t hist[2][kBuckets];
  uint32_t wsum[2][kWarpsN / 2];
  float red[kWarpsN][4];
  float lo[kMaxLevels][2], scale[kMaxLevels][2];
  uint32_t b1[kMaxLevels][2], b2[kMaxLevels][2];
  uint32_t rank[2], below[2], cnt[2], list_n[2];
  float list[2][kCap];
  float res[2][2];
  float mm[4];     // block min0, min1, max0, max1
  int done[2];
  uint32_t flag;
};

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
template <class Cand>
__device__ __forceinline__ void block_minmax(SelShared &sh, Cand cand, int n) {
  float a0 = INFINITY, a1 = INFINITY, z0 = -INFINITY, z1 = -INFINITY;
  for (int e = threadIdx.x; e < n; e += kNormThreads) {
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
    for (int w = 0; w < kWarpsN; ++w) r = (lane < 2) ? fminf(r, sh.red[w][lane]) : fmaxf(r, sh.red[w][lane]);
    sh.mm[lane] = r;
  }
  __syncthreads();
}

// Block-wide scan of both histograms: threads [0, 128) scan component 0,
// [128, 256) component 1, kPerThread consecutive buckets each (summed in a
// skewed order to spread banks).  Writes the buckets holding ranks r and
// r + pair, the count below the first and the cumulative count through the
// second.
__device__ __forceinline__ void scan_find(SelShared &sh, int level, bool pair) {
  const int c = threadIdx.x / (kNormThreads / 2);
  const int t = threadIdx.x % (kNormThreads / 2);
  const uint32_t *h = sh.hist[c] + kPerThread * t;
  uint32_t local = 0;
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) local += h[(j + t) & (kPerThread - 1)];
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
    for (int j = 0; j < kPerThread; ++j) {
      const uint32_t nxt = acc + h[j];
      if (r1 >= acc && r1 < nxt) {
        sh.b1[level][c] = kPerThread * t + j;
        sh.below[c] = acc;
      }
      if (r2 >= acc && r2 < nxt) {
        sh.b2[level][c] = kPerThread * t + j;
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
template <class Sh>
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
    for (int w = 0; w < kWarpsN; ++w) {
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
template <class Get>
__device__ void select_levels(SelShared &sh, Get get, int n, uint32_t rank, bool pair,
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
    for (int j = threadIdx.x; j < 2 * kBuckets; j += kNormThreads) (&sh.hist[0][0])[j] = 0u;
    __syncthreads();
    if (sh.done[0] && sh.done[1]) break;
    for (int e = threadIdx.x; e < n; e += kNormThreads) {
      float v0, v1;
      bool c0, c1;
      cand(e, v0, c0, v1, c1, level);
      if (c0) atomicAdd(&sh.hist[0][bucket_of(v0, sh.lo[level][0], sh.scale[level][0])], 1u);
      if (c1) atomicAdd(&sh.hist[1][bucket_of(v1, sh.lo[level][1], sh.scale[level][1])], 1u);
    }
    __syncthreads();
    scan_find(sh, level, pair);
    bool split[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) split[c] = !sh.done[c] && pair && sh.b1[level][c] != sh.b2[level][c];
    if (split[0] || split[1]) {
      float x0 = -INFINITY, x1 = -INFINITY, n0 = INFINITY, n1 = INFINITY;
      for (int e = threadIdx.x; e < n; e += kNormThreads) {
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
      split_pair(sh, split, x0, x1, n0, n1);
      if (threadIdx.x < 2 && split[threadIdx.x]) sh.done[threadIdx.x] = 1;
      __syncthreads();
      if (sh.done[0] && sh.done[1]) break;
    }
    bool gather[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) gather[c] = !sh.done[c] && (sh.cnt[c] - sh.below[c] <= static_cast<uint32_t>(kCap));
    if (gather[0] || gather[1]) {
      for (int e = threadIdx.x; e < n; e += kNormThreads) {
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
  scan_find(sh, 0, pair);
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

// ---------------------------------------------------------------------------
// Register-resident variant (the common case: blocks of at most 256 * 32
// bins).  Thread t holds bins t, t + 256, t + 512, ... in registers, loaded
// with coalesced 8-byte reads straight from global memory, and every pass
// (range, two selects, power) works on those registers: no staging copy,
// fewer instructions per bin, and small shared memory (histograms of 1024
// buckets).  A crowded target bucket falls back to the multi-level select
// above, reading the block from global memory.
constexpr int kFastBuckets = 1024;

struct RegShared {
  uint32_t hist[2][kFastBuckets];
  uint32_t wsum[2][kWarpsN / 2];
  float red[kWarpsN][4];
  uint32_t rank[2], below[2], cnt[2], list_n[2], b1[2], b2[2];
  float list[2][kCap];
  float res[2][2];
  float mm[4];
};

__device__ __forceinline__ uint32_t fast_bucket(float x, float lo, float scale) {
  const float t = (x - lo) * scale;
  return min(static_cast<uint32_t>(fmaxf(t, 0.0f)), static_cast<uint32_t>(kFastBuckets - 1));
}

__device__ __forceinline__ float fast_scale(float lo, float hi) {
  return (hi > lo) ? static_cast<float>(kFastBuckets) / (hi - lo) * (1.0f - 1.0f / 4096.0f) : 0.0f;
}

// Block min (mm[0..1]) and max (mm[2..3]) of the two components.
__device__ __forceinline__ void reg_minmax(RegShared &rs, float a0, float a1, float z0, float z1) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 = fminf(a0, __shfl_xor_sync(0xffffffffu, a0, o));
    a1 = fminf(a1, __shfl_xor_sync(0xffffffffu, a1, o));
    z0 = fmaxf(z0, __shfl_xor_sync(0xffffffffu, z0, o));
    z1 = fmaxf(z1, __shfl_xor_sync(0xffffffffu, z1, o));
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    rs.red[wid][0] = a0;
    rs.red[wid][1] = a1;
    rs.red[wid][2] = z0;
    rs.red[wid][3] = z1;
  }
  __syncthreads();
  if (wid == 0 && lane < 4) {
    float r = (lane < 2) ? INFINITY : -INFINITY;
    for (int w = 0; w < kWarpsN; ++w) r = (lane < 2) ? fminf(r, rs.red[w][lane]) : fmaxf(r, rs.red[w][lane]);
    rs.mm[lane] = r;
  }
  __syncthreads();
}

// Scan of both 1024-bucket histograms (threads [0,128): component 0,
// [128,256): component 1, 8 buckets each): the buckets of ranks r and
// r + pair, the count below the first and the cumulative count through the
// second.
__device__ __forceinline__ void reg_scan(RegShared &rs, bool pair) {
  constexpr int kPer = kFastBuckets / (kNormThreads / 2);
  const int c = threadIdx.x / (kNormThreads / 2);
  const int t = threadIdx.x % (kNormThreads / 2);
  const uint32_t *h = rs.hist[c] + kPer * t;
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
  if (lane == 31) rs.wsum[c][wid] = incl;
  __syncthreads();
  uint32_t base = 0;
  for (int j = 0; j < wid; ++j) base += rs.wsum[c][j];
  const uint32_t excl = base + incl - local;
  const uint32_t r1 = rs.rank[c];
  const uint32_t r2 = r1 + (pair ? 1u : 0u);
  if ((r1 >= excl && r1 < excl + local) || (r2 >= excl && r2 < excl + local)) {
    uint32_t acc = excl;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const uint32_t nxt = acc + h[j];
      if (r1 >= acc && r1 < nxt) {
        rs.b1[c] = kPer * t + j;
        rs.below[c] = acc;
      }
      if (r2 >= acc && r2 < nxt) {
        rs.b2[c] = kPer * t + j;
        rs.cnt[c] = nxt;
      }
      acc = nxt;
    }
  }
  __syncthreads();
}

// Level-0 select of ranks `rank` (and rank + 1 when `pair`) of both
// components over [lo, hi] from this thread's nv register values val(j).
// Returns false, having decided nothing, when a target bucket is crowded.
template <int K, class Val>
__device__ __forceinline__ bool reg_select(RegShared &rs, Val val, int nv, uint32_t rank, bool pair, float lo0,
                                           float lo1, float hi0, float hi1, float (&out_lo)[2],
                                           float (&out_hi)[2]) {
  const float s0 = fast_scale(lo0, hi0), s1 = fast_scale(lo1, hi1);
  const bool flat0 = !(hi0 > lo0), flat1 = !(hi1 > lo1);
  for (int j = threadIdx.x; j < 2 * kFastBuckets; j += kNormThreads) (&rs.hist[0][0])[j] = 0u;
  if (threadIdx.x < 2) {
    rs.rank[threadIdx.x] = rank;
    rs.list_n[threadIdx.x] = 0u;
  }
  __syncthreads();
  uint32_t qq[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j < nv) {
      const float2 f = val(j);
      const uint32_t q0 = fast_bucket(f.x, lo0, s0), q1 = fast_bucket(f.y, lo1, s1);
      atomicAdd(&rs.hist[0][q0], 1u);
      atomicAdd(&rs.hist[1][q1], 1u);
      qq[j] = q0 | (q1 << 16);
    }
  }
  __syncthreads();
  reg_scan(rs, pair);
  // a pair split over two buckets is decided by one max and one min
  const bool split[2] = {!flat0 && pair && rs.b1[0] != rs.b2[0], !flat1 && pair && rs.b1[1] != rs.b2[1]};
  if (split[0] || split[1]) {
    float x0 = -INFINITY, x1 = -INFINITY, n0 = INFINITY, n1 = INFINITY;
    const uint32_t sb10 = rs.b1[0], sb20 = rs.b2[0], sb11 = rs.b1[1], sb21 = rs.b2[1];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (j < nv) {
        const uint32_t q0 = qq[j] & 0xffffu, q1 = qq[j] >> 16;
        if ((split[0] && (q0 == sb10 || q0 == sb20)) || (split[1] && (q1 == sb11 || q1 == sb21))) {
          const float2 f = val(j);
          if (split[0] && q0 == sb10) x0 = fmaxf(x0, f.x);
          if (split[0] && q0 == sb20) n0 = fminf(n0, f.x);
          if (split[1] && q1 == sb11) x1 = fmaxf(x1, f.y);
          if (split[1] && q1 == sb21) n1 = fminf(n1, f.y);
        }
      }
    }
    split_pair(rs, split, x0, x1, n0, n1);
  }
  const bool need0 = !flat0 && !split[0], need1 = !flat1 && !split[1];
  if ((need0 && rs.cnt[0] - rs.below[0] > static_cast<uint32_t>(kCap)) ||
      (need1 && rs.cnt[1] - rs.below[1] > static_cast<uint32_t>(kCap))) {
    __syncthreads();
    return false;
  }
  const uint32_t l0 = need0 ? rs.b1[0] : 1u, h0 = need0 ? rs.b2[0] : 0u;
  const uint32_t l1 = need1 ? rs.b1[1] : 1u, h1 = need1 ? rs.b2[1] : 0u;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j < nv) {
      const uint32_t q0 = qq[j] & 0xffffu, q1 = qq[j] >> 16;
      const bool g0 = q0 >= l0 && q0 <= h0, g1 = q1 >= l1 && q1 <= h1;
      if (g0 || g1) {
        const float2 f = val(j);
        if (g0) rs.list[0][atomicAdd(&rs.list_n[0], 1u)] = f.x;
        if (g1) rs.list[1][atomicAdd(&rs.list_n[1], 1u)] = f.y;
      }
    }
  }
  __syncthreads();
  const bool active[2] = {need0, need1};
  rank_lists(rs, active, pair);
  out_lo[0] = flat0 ? lo0 : rs.res[0][0];
  out_lo[1] = flat1 ? lo1 : rs.res[1][0];
  out_hi[0] = flat0 ? lo0 : (pair ? rs.res[0][1] : rs.res[0][0]);
  out_hi[1] = flat1 ? lo1 : (pair ? rs.res[1][1] : rs.res[1][0]);
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

// Blocks per SM the register budget must allow: all values of a thread plus
// one bucket word per value stay in registers.  Up to K = 17 four blocks per
// SM (64 registers; K = 17 spills ~90 bytes to L1, which costs less than a
// third round of CTAs on 1024-block grids).
constexpr int reg_min_blocks(int k) { return k <= 17 ? 4 : 1; }

template <int K>
__global__ void __launch_bounds__(kNormThreads, reg_min_blocks(K)) normalise_reg_kernel(
    const float2 *__restrict__ spec, float *__restrict__ power, float4 *__restrict__ stats,
    const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off, int n_series, int seg_len,
    float *__restrict__ sel) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  RegShared &rs = *reinterpret_cast<RegShared *>(smem_raw);
  SelShared &sh = *reinterpret_cast<SelShared *>(smem_raw);   // the fallback's (same memory, used after rs)
  const int64_t g = blockIdx.x;
  int lo = 0, hi = n_series - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const SeriesDev S = series[lo];
  const int64_t sl = g - S.seg_off;
  const int64_t b0 = sl * seg_len;
  const int n = static_cast<int>(((sl == S.n_seg - 1) ? S.m : b0 + seg_len) - b0);
  const float2 *src = spec + S.spec_off + b0;
  const int t = threadIdx.x;
  const int nv = (t < n) ? min(K, (n - t + kNormThreads - 1) / kNormThreads) : 0;
  float2 v[K];
#pragma unroll
  for (int j = 0; j < K; ++j) v[j] = (j < nv) ? __ldg(src + j * kNormThreads + t) : make_float2(0.0f, 0.0f);
  const bool dc_here = (b0 == 0);
  if (dc_here && t == 0) v[0] = make_float2(0.0f, 0.0f);   // DC := 0
  auto gval = [&](int e) -> float2 { return (dc_here && e == 0) ? make_float2(0.0f, 0.0f) : src[e]; };

  float a0 = INFINITY, a1 = INFINITY, z0 = -INFINITY, z1 = -INFINITY;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j < nv) {
      a0 = fminf(a0, v[j].x);
      a1 = fminf(a1, v[j].y);
      z0 = fmaxf(z0, v[j].x);
      z1 = fmaxf(z1, v[j].y);
    }
  }
  reg_minmax(rs, a0, a1, z0, z1);
  const float mn0 = rs.mm[0], mn1 = rs.mm[1], mx0 = rs.mm[2], mx1 = rs.mm[3];
  __syncthreads();

  const bool even = (n % 2) == 0;
  const uint32_t rank = even ? static_cast<uint32_t>(n / 2 - 1) : static_cast<uint32_t>(n / 2);
  // Two passes through ONE copy of the select code (a smaller kernel keeps
  // the instruction cache warm): pass 0 selects the median of the values,
  // pass 1 the median of their absolute deviations from it (the MAD).
  float med_re = 0.0f, med_im = 0.0f, mad_re = 0.0f, mad_im = 0.0f;
  float lo0 = mn0, lo1 = mn1, hi0 = mx0, hi1 = mx1;
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const float c0 = med_re, c1 = med_im;
    float lo_v[2], hi_v[2];
    if (!reg_select<K>(rs, [&](int j) {
          return pass ? make_float2(fabsf(v[j].x - c0), fabsf(v[j].y - c1)) : v[j];
        }, nv, rank, even, lo0, lo1, hi0, hi1, lo_v, hi_v))
      select_levels(sh, [&](int e, float &v0, float &v1) {
        const float2 f = gval(e);
        v0 = pass ? fabsf(f.x - c0) : f.x;
        v1 = pass ? fabsf(f.y - c1) : f.y;
      }, n, rank, even, lo_v, hi_v);
    float a, b;
    bcast_mid(rs.mm, lo_v, hi_v, even, a, b);
    if (sel != nullptr && t == 0) {
      sel[8 * g + 2 * pass + 0] = lo_v[0];
      sel[8 * g + 2 * pass + 1] = hi_v[0];
      sel[8 * g + 2 * pass + 4] = lo_v[1];
      sel[8 * g + 2 * pass + 5] = hi_v[1];
    }
    if (pass == 0) {
      med_re = a;
      med_im = b;
      // the deviations lie in [0, max distance of the block's range from the median]
      lo0 = 0.0f;
      lo1 = 0.0f;
      hi0 = fmaxf(fabsf(mx0 - med_re), fabsf(med_re - mn0));
      hi1 = fmaxf(fabsf(mx1 - med_im), fabsf(med_im - mn1));
    } else {
      mad_re = a;
      mad_im = b;
    }
  }
  float inv_re, inv_im;
  bcast_inv(rs.mm, mad_re, mad_im, inv_re, inv_im);
  float *out = power + S.p_off + b0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j < nv) {
      const float a = (v[j].x - med_re) * inv_re;
      const float b = (v[j].y - med_im) * inv_im;
      out[j * kNormThreads + t] = 0.5f * (a * a + b * b);
    }
  }
  if (t == 0 && stats != nullptr) stats[g] = make_float4(med_re, mad_re, med_im, mad_im);
}

// Bins per thread of the register kernel for the plan's largest block (0:
// too large, use the staged kernel).  Power-of-two series leave a last block
// of L + 1 bins, hence the odd sizes.
constexpr int kRegK[] = {1, 2, 3, 4, 5, 6, 8, 9, 12, 16, 17, 24, 32};

int reg_bins_per_thread(pulscan_plan p) {
  int64_t max_n = 0;
  for (int64_t i = 0; i < p->n_base; ++i) {
    const auto &se = p->series[i];
    max_n = std::max<int64_t>(max_n, se.m - (se.n_seg - 1) * p->seg_len);
  }
  for (int k : kRegK)
    if (max_n <= static_cast<int64_t>(k) * kNormThreads) return k;
  return 0;
}

template <int K>
void launch_reg(pulscan_plan p, const float *d_spec, float *d_power, float4 *st4, float *d_sel, cudaStream_t s) {
  normalise_reg_kernel<K><<<static_cast<unsigned>(p->base_seg), kNormThreads, sizeof(SelShared), s>>>(
      reinterpret_cast<const float2 *>(d_spec), d_power, st4, p->d_series, p->d_seg_off,
      static_cast<int>(p->n_base), p->seg_len, d_sel);
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

}  // namespace

SmemLimit g_lim_norm;

int prepare_normalise(pulscan_plan p) { return ensure_smem(normalise_kernel, normalise_smem(p, nullptr), g_lim_norm); }

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
  switch (reg_bins_per_thread(p)) {
    case 0: break;
    case 1: launch_reg<1>(p, d_spec, d_power, st4, d_sel, s); break;
    case 2: launch_reg<2>(p, d_spec, d_power, st4, d_sel, s); break;
    case 3: launch_reg<3>(p, d_spec, d_power, st4, d_sel, s); break;
    case 4: launch_reg<4>(p, d_spec, d_power, st4, d_sel, s); break;
    case 5: launch_reg<5>(p, d_spec, d_power, st4, d_sel, s); break;
    case 6: launch_reg<6>(p, d_spec, d_power, st4, d_sel, s); break;
    case 8: launch_reg<8>(p, d_spec, d_power, st4, d_sel, s); break;
    case 9: launch_reg<9>(p, d_spec, d_power, st4, d_sel, s); break;
    case 12: launch_reg<12>(p, d_spec, d_power, st4, d_sel, s); break;
    case 16: launch_reg<16>(p, d_spec, d_power, st4, d_sel, s); break;
    case 17: launch_reg<17>(p, d_spec, d_power, st4, d_sel, s); break;
    case 24: launch_reg<24>(p, d_spec, d_power, st4, d_sel, s); break;
    default: launch_reg<32>(p, d_spec, d_power, st4, d_sel, s); break;
  }
  if (reg_bins_per_thread(p) > 0) {
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
