// Differentiable extension: a logsumexp relaxation of the per-(segment,
// width) maximum of Algorithm 4 and its hand-written adjoint.
//
//   Y[s, w] = tau * log sum_{k in seg s, k <= M - w} exp(S_w[k] / tau)
//
// tends to the maximum as tau -> 0.  The adjoint goes back through the
// softmax weights, the boxcar bank (whose adjoint is again a boxcar: every
// weight is added to all bins of its window), P = (a^2 + b^2)/2, the median /
// MAD normalisation of Eq. 8 (almost-everywhere derivatives at the selected
// order statistics) and the real FFT, to the time series.
//
// Kernels (one CTA per segment, one warp per 1056 bins: each lane holds one
// 33-bin tile and sweeps widths 1..W as in the search; a form with two tiles
// per lane as packed pairs is kept as the kernels' T = 2 instance):
// * lse_forward_kernel: per width the warp takes the maximum of its windows
//   (one redux.sync), per 33-width block the warps' maxima give
//   M[s, w] = max S_w; only windows within cut = tau * ln 2^24 of M are
//   exponentiated -- every other term weighs < 2^-24 of the largest, and at
//   most 2L of them change Y by < tau 2L 2^-24 -- so exp work is rare;
// * lse_backward_kernel: the same sweep; each window within the cut of Y
//   gets weight g = G exp((S - Y) / tau), entered as a difference pair
//   D[k] += g, D[k + w] -= g (reductions into the segment's own dL/dP and
//   tail slots, which stay in L2); after the sweep one block prefix sum of D
//   gives dL/dP over the segment and a (W - 1)-bin tail that spills into the
//   next segment;
// * the sweep only flags, per width, which 11-bin groups of which lanes
//   hold a window within the cut (six group maxima per lane and step,
//   ballots kept by the lane that owns the step); the flagged (group, width)
//   events of a 33-width block are worked off after it, a lane per event.
//   Keeping the exp / scatter code out of the unrolled ring steps keeps the
//   loop body small enough for the instruction cache;
// * the sweep's FP32 window sums (differences of the prefix's high parts)
//   pick windows only: an exponent (S - M) / tau amplifies an absolute
//   error in S by 1 / tau, and such a sum carries about an ulp of F.  Each
//   picked window's S is recomputed as F[k + w] - F[k] from the per-segment
//   exclusive prefix sum F held in shared memory as an unevaluated pair of
//   floats (hi + lo, built
//   with error-free additions, carried between threads in FP64) and kept as
//   a pair: even one rounding of S (half an ulp, 2.4e-4 at S = 4096) would
//   move a weight by 2.4e-3 at tau = 0.1.  S - M is taken as (hi - M) + lo,
//   whose first difference is exact;
// * Y leaves the forward as a pair too (d_y and its rounding error d_ylo),
//   and the backward's weights use (hi - Y) + (lo - Ylo): an FP32 Y alone
//   would scale every weight of a (segment, width) by exp(dY / tau);
// * normalise_backward_kernel: dL/dP -> dL/d(Re, Im) through Eq. 8, written
//   as the input of a cuFFT C2R transform with the Hermitian weights (DC 0,
//   interior halved, Nyquist real), whose output is dL/dx;
// * inject_kernel / amp_grad_partial_kernel + amp_grad_sum_kernel:
//   x = noise + A template and dL/dA = sum_n dL/dx[n] template[n], per series.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include <cuda_fp16.h>

#include "bank.cuh"
#include "common.cuh"
#include "ptx.cuh"

namespace ps {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kLseMaxWarps = 2;   // segments of at most 2 x 2112 bins

// s + e == a + b exactly (Knuth's two-sum; explicit roundings, no contraction).
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float t = __fadd_rn(a, b);
  const float bb = __fsub_rn(t, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(b, bb));
  return t;
}

// Exclusive prefix F[j] = sum_{i<j} P[i] for j = 0..n as fh[j] + fl[j],
// built in place: fh[0..n) holds P on entry (fh has n + 1 entries).
// fl (at most half an ulp of fh) is kept in FP16, whose 11-bit mantissa
// leaves an error below 2^-12 ulp of F.
// Each thread sums a contiguous chunk with two-sum, the chunk totals are
// scanned in FP64 (wtot: one double per warp), then each chunk is re-walked
// from its FP64 carry split into a float pair (every thread reads and
// overwrites its own chunk only).  Ends with a barrier.
__device__ void build_prefix(float *__restrict__ fh, int n, __half *__restrict__ fl, double *wtot) {
  const int nt = blockDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int chunk = (n + nt - 1) / nt;
  const int a0 = min(n, static_cast<int>(threadIdx.x) * chunk), a1 = min(n, a0 + chunk);
  float h = 0.0f, l = 0.0f, e;
  for (int j = a0; j < a1; ++j) {
    h = two_sum(h, fh[j], e);
    l = __fadd_rn(l, e);
  }
  const double tot = static_cast<double>(h) + static_cast<double>(l);
  double incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  double carry = incl - tot;
  for (int v = 0; v < warp; ++v) carry += wtot[v];
  h = static_cast<float>(carry);
  l = static_cast<float>(carry - static_cast<double>(h));
  // stored normalised (fast two-sum, |l| << |h|): |fl| <= half an ulp of fh
  for (int j = a0; j < a1; ++j) {
    const float v = fh[j];
    const float hs = __fadd_rn(h, l);
    fh[j] = hs;
    fl[j] = __float2half_rn(__fsub_rn(l, __fsub_rn(hs, h)));
    h = two_sum(h, v, e);
    l = __fadd_rn(l, e);
  }
  if (threadIdx.x == nt - 1) {   // its chunk ends at n, or is empty with the full total as carry
    const float hs = __fadd_rn(h, l);
    fh[n] = hs;
    fl[n] = __float2half_rn(__fsub_rn(l, __fsub_rn(hs, h)));
  }
  __syncthreads();
}

// sum buf[a..b) = F[b] - F[a] as an unevaluated pair hi + lo: hi = fh[b] -
// fh[a] rounded, lo = its rounding error plus the difference of the low
// parts, so hi + lo carries about 2^-12 ulp of F of error (not one rounding
// of S).  Callers subtract a nearby reference from hi first (exact by
// Sterbenz's lemma when the two are within a factor of two) and add lo after.
__device__ __forceinline__ float window_sum2(const float *__restrict__ fh, const __half *__restrict__ fl, int a, int b,
                                             float &lo) {
  float e;
  const float d = two_sum(fh[b], -fh[a], e);
  lo = __fadd_rn(e, __fsub_rn(__half2float(fl[b]), __half2float(fl[a])));
  return d;
}

// A lane works on two 33-bin tiles at once, a = warp * kSpan + lane * 33 and
// b = a + kTile, as packed pairs: one add.rn.f32x2 forms a window sum of
// both (two FP32 adds, the same roundings as scalar adds).
constexpr int kTile = 32 * kR;     // 1056 bins: the lanes' first tiles
constexpr int kSpan = 2 * kTile;   // 2112 bins per warp
constexpr int kSub = 11;           // ring steps unrolled at a time (kR = 3 kSub)

__device__ __forceinline__ uint64_t pk2(float x, float y) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(x), "f"(y));
  return d;
}

__device__ __forceinline__ void upk2(uint64_t d, float &x, float &y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(d));
}

__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Runs widths 1..W over the lane's two tiles, calling cb(w, c, sv, full)
// per width: sv(i) gives the pair (S_w[xa + i], S_w[xb + i]) of window sums,
// formed as F[x + i + w] - F[x + i] from the prefix's high parts.  These sums
// only pick windows (the picked ones are recomputed exactly): their error,
// about an ulp of F, is far below any cut.  The lane keeps -F[x + i]
// (-inf for start bins past the segment's end, nva / nvb valid, so those
// never win a maximum) and a ring of F[x + i + w] that advances one bin per
// width (one shared load per tile and width).  Full 33-width blocks run the
// ring unrolled with no per-step branch; full_block(bi, nsteps)
// (warp-uniform) says whether every window of the warp is valid through
// block bi -- cb gets a compile-time flag for it.  Other blocks (the
// spectrum's end, the last partial block) read F straight from shared
// memory in a rolled loop.  block_end(bi, nsteps) follows every block.
template <class Full, class F, class G>
__device__ __forceinline__ void walk_pairs(const float *__restrict__ fh, int xa, int xb, int nva, int nvb, int W,
                                           Full &&full_block, F &&cb, G &&block_end) {
  uint64_t nb2[kR], r2[kR];
#pragma unroll
  for (int i = 0; i < kR; ++i) nb2[i] = pk2(i < nva ? -fh[xa + i] : -INFINITY, i < nvb ? -fh[xb + i] : -INFINITY);
  auto load_ring = [&](int wf) {
#pragma unroll
    for (int j = 0; j < kR - 1; ++j) r2[j] = pk2(fh[xa + wf + j], fh[xb + wf + j]);
  };
  load_ring(1);
  const int nblk = (W + kR - 1) / kR;
  for (int bi = 0; bi < nblk; ++bi) {
    const int wf = bi * kR + 1;
    const int nsteps = min(kR, W - bi * kR);
    if (nsteps == kR && full_block(bi, nsteps)) {
      // three rolled sub-blocks of 11 unrolled steps (a third of the code of
      // 33 unrolled steps, for the instruction cache), each ending with the
      // ring rotated by 11 so that the next starts from the same layout
#pragma unroll 1
      for (int sb = 0; sb < kR; sb += kSub) {
        const int ws = wf + sb;
#pragma unroll
        for (int cc = 0; cc < kSub; ++cc) {
          r2[(cc + kR - 1) % kR] = pk2(fh[xa + ws + cc + kR - 1], fh[xb + ws + cc + kR - 1]);
          cb(ws + cc, sb + cc, [&](int i) { return add2(r2[(i + cc) % kR], nb2[i]); }, std::true_type{});
        }
        uint64_t rot[kR];
#pragma unroll
        for (int i = 0; i < kR; ++i) rot[i] = r2[(i + kSub) % kR];
#pragma unroll
        for (int i = 0; i < kR; ++i) r2[i] = rot[i];
      }
    } else {
      for (int c = 0; c < nsteps; ++c) {
        const int w = wf + c;
        cb(w, c, [&](int i) { return add2(pk2(fh[xa + i + w], fh[xb + i + w]), nb2[i]); }, std::false_type{});
      }
      if (bi + 1 < nblk) load_ring(wf + kR);
    }
    block_end(bi, nsteps);
  }
}

// The one-tile form of walk_pairs: the lane's 33 start bins x .. x + 32 as
// scalars, sv(i) = F[x + i + w] - F[x + i] by one FP32 add; the same ring,
// blocks and sub-blocks (half the registers: 66 instead of 132).
template <class Full, class F, class G>
__device__ __forceinline__ void walk_single(const float *__restrict__ fh, int xa, int nva, int W, Full &&full_block,
                                            F &&cb, G &&block_end) {
  float nb[kR], r[kR];
#pragma unroll
  for (int i = 0; i < kR; ++i) nb[i] = i < nva ? -fh[xa + i] : -INFINITY;
  auto load_ring = [&](int wf) {
#pragma unroll
    for (int j = 0; j < kR - 1; ++j) r[j] = fh[xa + wf + j];
  };
  load_ring(1);
  const int nblk = (W + kR - 1) / kR;
  for (int bi = 0; bi < nblk; ++bi) {
    const int wf = bi * kR + 1;
    const int nsteps = min(kR, W - bi * kR);
    if (nsteps == kR && full_block(bi, nsteps)) {
#pragma unroll 1
      for (int sb = 0; sb < kR; sb += kSub) {
        const int ws = wf + sb;
#pragma unroll
        for (int cc = 0; cc < kSub; ++cc) {
          r[(cc + kR - 1) % kR] = fh[xa + ws + cc + kR - 1];
          cb(ws + cc, sb + cc, [&](int i) { return __fadd_rn(r[(i + cc) % kR], nb[i]); }, std::true_type{});
        }
        float rot[kR];
#pragma unroll
        for (int i = 0; i < kR; ++i) rot[i] = r[(i + kSub) % kR];
#pragma unroll
        for (int i = 0; i < kR; ++i) r[i] = rot[i];
      }
    } else {
      for (int c = 0; c < nsteps; ++c) {
        const int w = wf + c;
        cb(w, c, [&](int i) { return __fadd_rn(fh[xa + i + w], nb[i]); }, std::false_type{});
      }
      if (bi + 1 < nblk) load_ring(wf + kR);
    }
    block_end(bi, nsteps);
  }
}

struct SegTile {
  int64_t m, b0, seg_g;
  int nb;          // bins of this segment
  const float *src;
  float *buf;
};

// Stage P[b0 .. b0 + buf_len) (zeros beyond M) into shared memory.
__device__ __forceinline__ bool stage_segment(const SegTile &t, int buf_len, uint64_t *bar, uint32_t *flag,
                                              uint32_t *counters) {
  const int64_t avail64 = t.m - t.b0;
  const int avail = static_cast<int>(min64(avail64, static_cast<int64_t>(buf_len)));
  const int n_tma = ((reinterpret_cast<uintptr_t>(t.src) & 15u) == 0u && avail > 0) ? (avail & ~3) : 0;
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && n_tma > 0) {
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(n_tma) * 4u);
    tma_load_1d(t.buf, t.src, static_cast<uint32_t>(n_tma) * 4u, bar);
  }
  for (int i = n_tma + threadIdx.x; i < buf_len; i += blockDim.x) t.buf[i] = (i < avail) ? t.src[i] : 0.0f;
  if (threadIdx.x == 0) *flag = (n_tma == 0 || mbar_wait_bounded(bar, 0, 2000000000ull)) ? 1u : 0u;
  __syncthreads();
  if (*flag == 0u) {
    if (threadIdx.x == 0) atomicOr(counters + 2, kErrTimeout);
    return false;
  }
  return true;
}

__device__ __forceinline__ SegTile seg_tile(const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off,
                                            int n_series, int seg_len, const float *power, float *buf) {
  const int64_t g = blockIdx.x;
  int lo = 0, hi = n_series - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const SeriesDev S = series[lo];
  SegTile t;
  const int64_t sl = g - S.seg_off;
  t.m = S.m;
  t.b0 = sl * seg_len;
  t.nb = static_cast<int>(((sl == S.n_seg - 1) ? S.m : t.b0 + seg_len) - t.b0);
  t.seg_g = g;
  t.src = power + S.p_off + t.b0;
  t.buf = buf;
  return t;
}

// Valid windows of the lane starting at local bin x at width w: start inside
// the segment, window inside the spectrum:  lim(w) = clamp(min(a, b - w), 0, 33)
// with a = nb - x and b = M - (b0 + x) + 1 fixed per tile.  The sums of
// bins past a start at -inf (walk_pairs), so only the spectrum's end needs a
// mask: `masked(w)` says whether it cuts one of the tile's windows at width w.
struct LaneLim {
  int a, b;
  __device__ __forceinline__ int at(int w) const { return max(0, min(kR, min(a, b - w))); }
  __device__ __forceinline__ bool masked(int w) const { return a > 0 && b - w < min(a, kR); }
};

__device__ __forceinline__ LaneLim lane_lim(const SegTile &t, int x) {
  const int64_t bb = t.m - (t.b0 + x) + 1;
  return LaneLim{t.nb - x, static_cast<int>(min64(bb, static_cast<int64_t>(1) << 30))};
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Maxima of the lane's six 11-bin groups, g[j] of tile a and g[3 + j] of
// tile b (windows i < lim only; -inf where none), and their maximum.
// kFull: every window valid (the limits are ignored).
constexpr int kGrp = 11;
template <bool kFull, class S>
__device__ __forceinline__ float lane_groups2(S &&sv, int lima, int limb, float (&g)[6]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float a[kGrp], b[kGrp];
#pragma unroll
    for (int i = 0; i < kGrp; ++i) upk2(sv(kGrp * j + i), a[i], b[i]);
    if (kFull) {
      g[j] = max3(max3(max3(a[0], a[1], a[2]), max3(a[3], a[4], a[5]), max3(a[6], a[7], a[8])), a[9], a[10]);
      g[3 + j] = max3(max3(max3(b[0], b[1], b[2]), max3(b[3], b[4], b[5]), max3(b[6], b[7], b[8])), b[9], b[10]);
    } else {
      float ma = -INFINITY, mb = -INFINITY;
#pragma unroll
      for (int i = 0; i < kGrp; ++i) {
        ma = fmaxf(ma, (kGrp * j + i < lima) ? a[i] : -INFINITY);
        mb = fmaxf(mb, (kGrp * j + i < limb) ? b[i] : -INFINITY);
      }
      g[j] = ma;
      g[3 + j] = mb;
    }
  }
  return fmaxf(max3(g[0], g[1], g[2]), max3(g[3], g[4], g[5]));
}

// The one-tile form: maxima of the lane's three 11-bin groups (windows
// i < lim only; -inf where none) and their maximum.
template <bool kFull, class S>
__device__ __forceinline__ float lane_groups1(S &&sv, int lim, float (&g)[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float a[kGrp];
#pragma unroll
    for (int i = 0; i < kGrp; ++i) a[i] = sv(kGrp * j + i);
    if (kFull) {
      g[j] = max3(max3(max3(a[0], a[1], a[2]), max3(a[3], a[4], a[5]), max3(a[6], a[7], a[8])), a[9], a[10]);
    } else {
      float ma = -INFINITY;
#pragma unroll
      for (int i = 0; i < kGrp; ++i) ma = fmaxf(ma, (kGrp * j + i < lim) ? a[i] : -INFINITY);
      g[j] = ma;
    }
  }
  return max3(g[0], g[1], g[2]);
}

// The window limits of a segment in 32-bit form: start bin x of the
// segment has valid windows of width w for its lane's bins up to
// lim = clamp(min(nb - x, room - x - w), 0, 33), room = M - b0 + 1.
struct SegLim {
  int nb, room;
  __device__ __forceinline__ int at(int x, int w) const { return max(0, min(kR, min(nb - x, room - x - w))); }
};

__device__ __forceinline__ SegLim seg_lim(const SegTile &t) {
  return SegLim{t.nb, static_cast<int>(min64(t.m - t.b0 + 1, static_cast<int64_t>(1) << 30))};
}

// All events of one 33-width block at once: (step c, lane l, group j)
// triples, c | l << 6 | j << 11, for every 11-bin group whose bit is set in
// the step masks mk (ballots: bit l of mk[r][j] is group j of lane l, j < 3
// in tile a and j - 3 in tile b; this
// lane holds those of step `lane` in mk[0] and lane 0 also those of step 32
// in mk[1], zero where the lane owns no step); then their windows (11 per
// event) are worked off a thread per event (block_events_cta), in rounds of
// at most kEvCap events per warp of the CTA.  Collecting a block's events
// first gives the window work the whole block's parallelism instead of one
// width's.  f(c, k, w, hi, lo) is called for every window whose exact sum
// lies above thr(c) (S = hi + lo, k the segment-local start bin).
constexpr int kEvCap = 128;

// One event (step c, lane l, group jg, warp wv: c | l << 6 | jg << 11 | wv << 14):
// its 11 windows are screened with the prefix's high parts alone
// (independent loads; within 1.5 ulp of F, margin 4 ulp of the segment's
// largest F), then the few that pass are summed exactly.
template <int NG, class Thr, class F>
__device__ __forceinline__ void work_event(int ev, const SegLim &sl, int wf, Thr &&thr, const float *__restrict__ fh,
                                           const __half *__restrict__ fl, float margin, F &&f) {
  constexpr int kSpanW = (NG / 3) * kTile;   // bins per warp: one or two tiles per lane
  const int c = ev & 63, l = (ev >> 6) & 31, jg = (ev >> 11) & 7, wv = ev >> 14;
  const int w = wf + c;
  const int x = wv * kSpanW + (jg >= 3 ? kTile : 0) + l * kR;   // the tile's first bin
  const int b0 = kGrp * (jg >= 3 ? jg - 3 : jg);                 // the group's first bin in the tile
  const int k0 = x + b0;
  const int lim = sl.at(x, w) - b0;                              // valid windows: i < lim
  const float th = thr(c);
  float ha[kGrp], hb[kGrp];
#pragma unroll
  for (int i = 0; i < kGrp; ++i) {
    ha[i] = fh[k0 + i];
    hb[i] = fh[k0 + w + i];
  }
  const float ths = th - margin;
  uint32_t hot = 0u;
#pragma unroll
  for (int i = 0; i < kGrp; ++i) hot |= (hb[i] - ha[i] > ths) ? (1u << i) : 0u;
  if (lim < kGrp) hot &= (lim > 0) ? ((1u << lim) - 1u) : 0u;
  while (hot != 0u) {
    const int k = k0 + __ffs(static_cast<int>(hot)) - 1;
    hot &= hot - 1u;
    float lo;
    const float hi = window_sum2(fh, fl, k, k + w, lo);
    if (__fadd_rn(__fsub_rn(hi, th), lo) > 0.0f) f(c, k, w, hi, lo);
  }
}

// This lane's events of the block (see block_events_cta) written to evl[pos -
// base] for list positions pos in [base, base + cap), from position `first` on.
template <int NG>
__device__ __forceinline__ void write_events(const uint32_t (&mk)[2][NG], int warp, int lane, int first, int base,
                                             int cap, int *evl) {
  int pos = first;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int c = r ? kR - 1 : lane;
#pragma unroll
    for (int j = 0; j < NG; ++j) {
      for (uint32_t mm = mk[r][j]; mm != 0u; mm &= mm - 1u, ++pos)
        if (pos >= base && pos < base + cap)
          evl[pos - base] = c | ((__ffs(static_cast<int>(mm)) - 1) << 6) | (j << 11) | (warp << 14);
    }
  }
}

template <int NG>
__device__ __forceinline__ uint32_t count_events(const uint32_t (&mk)[2][NG]) {
  uint32_t cnt = 0u;
#pragma unroll
  for (int j = 0; j < NG; ++j) cnt += __popc(mk[0][j]) + __popc(mk[1][j]);
  return cnt;
}

// The CTA's events of the block worked off by all its threads: the warp
// holding the segment's maximum flags nearly all of them, and the others
// would wait for it at the next block's barrier.  wcnt: one int per warp.
// Ends with the list free (a barrier after each full chunk but the last).
template <class Thr, class F, int NG>
__device__ __forceinline__ void block_events_cta(const SegLim &sl, int warp, int lane, int wf,
                                                 const uint32_t (&mk)[2][NG], Thr thr, const float *__restrict__ fh,
                                                 const __half *__restrict__ fl, int *evl, int cap, int *wcnt,
                                                 float margin, F &&f) {
  const uint32_t cnt = count_events(mk);
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wcnt[warp] = static_cast<int>(incl);
  __syncthreads();
  const int warps = blockDim.x >> 5;
  int woff = 0, n_ev = 0;
  for (int v = 0; v < warps; ++v) {
    const int cv = wcnt[v];
    if (v < warp) woff += cv;
    n_ev += cv;
  }
  const int first = woff + static_cast<int>(incl - cnt);
  for (int base = 0; base < n_ev; base += cap) {
    write_events(mk, warp, lane, first, base, cap, evl);
    __syncthreads();
    const int n_round = min(cap, n_ev - base);
    for (int e = threadIdx.x; e < n_round; e += blockDim.x) work_event<NG>(evl[e], sl, wf, thr, fh, fl, margin, f);
    if (base + cap < n_ev) __syncthreads();
  }
}

// The warp's maximum of v (a single reduction instruction on sm_100+).
__device__ __forceinline__ float warp_max(float v) {
  float r;
  asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}

// Per-warp rows of 33 widths, double-buffered by block parity (up to four
// warps: one tile per lane); the backward's four rows per warp.
constexpr int kRows = 4 * kR;
constexpr int kBwdRows = 4 * 4 * kR;

// Per-step ballots of the six group flags g[j] >= lo (or > lo), kept by the
// lane that owns the step (lane c for step c, every lane for step 32).
template <bool kStrict, int NG>
__device__ __forceinline__ void flag_groups(const float (&g)[NG], float lo, int c, int lane, uint32_t (&mk)[2][NG]) {
#pragma unroll
  for (int j = 0; j < NG; ++j) {
    const uint32_t bal = __ballot_sync(kFullMask, kStrict ? g[j] > lo : g[j] >= lo);
    if (c == lane) mk[0][j] = bal;
    if (c == kR - 1) mk[1][j] = bal;
  }
}

template <int T>
__global__ void __launch_bounds__(T == 1 ? 128 : 64, T == 1 ? 5 : 6) lse_forward_kernel(
    const float *__restrict__ power, const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off,
    int n_series, int W, int seg_len, float tau, float cut, float *__restrict__ y, float *__restrict__ ylo,
    uint32_t *__restrict__ counters, int buf_len) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  double *wtot = reinterpret_cast<double *>(smem_raw + 32);
  uint32_t *flag = reinterpret_cast<uint32_t *>(smem_raw + 64);
  int *wcnt = reinterpret_cast<int *>(smem_raw + 80);      // per-warp event counts (four)
  float *fh = reinterpret_cast<float *>(smem_raw + 128);   // P, then the prefix's high part: buf_len + 1
  float *wmax = fh + buf_len + 1;       // [2][warps][33]: each warp's maximum per width
  float *mrow = wmax + 2 * kRows;       // [2][warps][33]: M per width, a copy per warp
  float *lsbw = mrow + 2 * kRows;       // [2][warps][33]: each warp's sums of exp
  const int warps = blockDim.x >> 5;
  int *evl = reinterpret_cast<int *>(lsbw + 2 * kRows);           // the CTA's event list: warps x kEvCap
  __half *fl = reinterpret_cast<__half *>(evl + warps * kEvCap);   // the prefix's low part: buf_len + 1
  const SegTile t = seg_tile(series, seg_off, n_series, seg_len, power, fh);
  if (!stage_segment(t, buf_len, bar, flag, counters)) return;
  build_prefix(fh, buf_len, fl, wtot);
  const float margin = 4.8e-7f * fh[buf_len];   // 4 ulp of the largest prefix value (F is non-decreasing)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NG = 3 * T;   // 11-bin groups per lane
  const int xa = warp * (T * kTile) + lane * kR, xb = xa + kTile;
  const LaneLim la = lane_lim(t, xa), lb = lane_lim(t, xb);
  const SegLim sgl = seg_lim(t);
  const float inv_tau = 1.0f / tau;
  // Y = M + tau log(sum) of block bj's widths as a pair: the FP32 value and
  // its exact rounding error (the backward's weights exp((S - Y) / tau) need
  // Y to better than FP32 resolution: an error dY moves them all by dY / tau).
  // Thread c (< nst) takes width c: the warps' partial sums, its own warp's M.
  auto emit_y = [&](int bj, int nst) {
    const int pp = bj & 1;
    for (int c = threadIdx.x; c < nst; c += blockDim.x) {
      float sum = 0.0f;
      for (int v = 0; v < warps; ++v) sum += lsbw[pp * kRows + v * kR + c];
      float e;
      const float yh = two_sum(mrow[pp * kRows + warp * kR + c], tau * logf(sum), e);
      const int64_t o = t.seg_g * static_cast<int64_t>(W) + bj * kR + c;
      y[o] = yh;
      ylo[o] = e;
    }
  };
  uint32_t mk[2][NG];
#pragma unroll
  for (int j = 0; j < NG; ++j) mk[0][j] = mk[1][j] = 0u;
  float wme = -INFINITY, wm32 = -INFINITY;   // this warp's maximum at step `lane`, and at step 32
  // One sweep over the widths.  Per step the warp takes its maximum wm of
  // all windows and ballots which lanes' 11-bin groups reach wm - cut.
  // After each 33-width block the warps' maxima give M[s, w] (one block
  // barrier), and the flagged groups are screened against M - cut (a group
  // within the cut of M is within the cut of wm <= M; a step whose wm is
  // below M - cut has none).
  auto full_block = [&](int bi, int nsteps) {
    const int w = bi * kR + nsteps;
    return !__any_sync(kFullMask, la.masked(w) || (T == 2 && lb.masked(w)));
  };
  auto step = [&](int w, int c, auto sv, auto full) {
    float g[NG];
    float lm;
    if constexpr (T == 2) lm = lane_groups2<decltype(full)::value>(sv, la.at(w), lb.at(w), g);
    else lm = lane_groups1<decltype(full)::value>(sv, la.at(w), g);
    const float wm = warp_max(lm);
    flag_groups<false>(g, wm - cut, c, lane, mk);
    if (c == lane) wme = wm;
    if (c == kR - 1) wm32 = wm;
  };
  auto block_end = [&](int bi, int nsteps) {
        const int p = bi & 1;
        const float *wm_p = wmax + p * kRows;
        if (lane < nsteps) wmax[p * kRows + warp * kR + lane] = wme;
        if (lane == 0 && nsteps == kR) wmax[p * kRows + warp * kR + kR - 1] = wm32;
        __syncthreads();
        if (bi > 0) emit_y(bi - 1, kR);
        // M per width (each warp its own copy); this warp's sums start at 0
        float *mr = mrow + p * kRows + warp * kR;
        float *ls = lsbw + p * kRows + warp * kR;
        bool drop = true;
        if (lane < nsteps) {
          float m = -INFINITY;
          for (int v = 0; v < warps; ++v) m = fmaxf(m, wm_p[v * kR + lane]);
          mr[lane] = m;
          ls[lane] = 0.0f;
          drop = wme < m - cut;
        }
        bool drop32 = true;
        if (nsteps == kR) {
          float m = -INFINITY;
          for (int v = 0; v < warps; ++v) m = fmaxf(m, wm_p[v * kR + kR - 1]);
          if (lane == 0) {
            mr[kR - 1] = m;
            ls[kR - 1] = 0.0f;
          }
          drop32 = lane != 0 || wm32 < m - cut;
        }
#pragma unroll
        for (int j = 0; j < NG; ++j) {
          if (drop) mk[0][j] = 0u;
          if (drop32) mk[1][j] = 0u;
        }
        block_events_cta(sgl, warp, lane, bi * kR + 1, mk, [&](int c) { return mr[c] - cut; }, fh, fl, evl,
                         warps * kEvCap, wcnt, margin, [&](int c, int, int, float hi, float lo) {
                           atomicAdd(&ls[c], __expf(__fadd_rn(__fsub_rn(hi, mr[c]), lo) * inv_tau));
                         });
      };
  if constexpr (T == 2) walk_pairs(fh, xa, xb, la.a, lb.a, W, full_block, step, block_end);
  else walk_single(fh, xa, la.a, W, full_block, step, block_end);
  __syncthreads();
  const int nb = (W + kR - 1) / kR;
  emit_y(nb - 1, W - (nb - 1) * kR);
}

template <int T>
__global__ void __launch_bounds__(T == 1 ? 128 : 64, T == 1 ? 5 : 6) lse_backward_kernel(
    const float *__restrict__ power, const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off,
    int n_series, int W, int seg_len, float tau, float cut, const float *__restrict__ y,
    const float *__restrict__ ylo, const float *__restrict__ gy, float *__restrict__ dp, float *__restrict__ tail,
    uint32_t *__restrict__ counters, int buf_len) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  double *wtot = reinterpret_cast<double *>(smem_raw + 32);
  uint32_t *flag = reinterpret_cast<uint32_t *>(smem_raw + 64);
  int *wcnt = reinterpret_cast<int *>(smem_raw + 80);      // per-warp event counts (four)
  float *fh = reinterpret_cast<float *>(smem_raw + 128);   // P, then the prefix's high part: buf_len + 1
  float *rows = fh + buf_len + 1;                // warps x [Y, Y low part, G, Y - cut] x 33 widths of a block
  float *wsum = rows + kBwdRows;                 // per-warp scan totals
  int *evl = reinterpret_cast<int *>(wsum + 32);                                  // warps x kEvCap event lists
  __half *fl = reinterpret_cast<__half *>(evl + (blockDim.x >> 5) * kEvCap);     // prefix: low part, buf_len + 1
  const SegTile t = seg_tile(series, seg_off, n_series, seg_len, power, fh);
  if (!stage_segment(t, buf_len, bar, flag, counters)) return;
  // The difference array D over the segment's bins and the W - 1 after it
  // (k + w <= nb + W - 1) lives in global memory, in this segment's own
  // output slots: its dL/dP bins, then its tail.  Updates are fire-and-forget
  // reductions that stay in L2; the CTA scans it after the sweep, staged
  // into shared memory over the then-unused prefix.
  float *out = dp + (t.src - power);   // same offset in the dP buffer
  float *tl = tail + t.seg_g * static_cast<int64_t>(W);
  const int d_seg = t.nb + W - 1;
  for (int j = threadIdx.x; j < t.nb; j += blockDim.x) out[j] = 0.0f;
  for (int j = threadIdx.x; j < W; j += blockDim.x) tl[j] = 0.0f;   // W - 1 read; the last takes k + w = nb + W - 1
  build_prefix(fh, buf_len, fl, wtot);   // ends with a barrier: the zeros come first
  const float margin = 4.8e-7f * fh[buf_len];   // 4 ulp of the largest prefix value (F is non-decreasing)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this warp's row of the block's widths: Y, its low part, G and the
  // threshold Y - cut (+inf where G = 0: no window of that width counts)
  float *yrow = rows + warp * 4 * kR, *ylrow = yrow + kR, *grow = ylrow + kR, *trow = grow + kR;
  auto load_rows = [&](int bi) {
    const int nst = min(kR, W - bi * kR);
    for (int c = lane; c < nst; c += 32) {
      const int64_t o = t.seg_g * static_cast<int64_t>(W) + bi * kR + c;
      const float yv = y[o], gv = gy[o];
      yrow[c] = yv;
      ylrow[c] = ylo[o];
      grow[c] = gv;
      trow[c] = (gv != 0.0f) ? yv - cut : INFINITY;
    }
    __syncwarp();
  };
  load_rows(0);
  constexpr int NG = 3 * T;   // 11-bin groups per lane
  const int xa = warp * (T * kTile) + lane * kR, xb = xa + kTile;
  const float inv_tau = 1.0f / tau;
  const LaneLim la = lane_lim(t, xa), lb = lane_lim(t, xb);
  const SegLim sgl = seg_lim(t);
  uint32_t mk[2][NG];
#pragma unroll
  for (int j = 0; j < NG; ++j) mk[0][j] = mk[1][j] = 0u;
  // Per step the warp ballots which lanes' 11-bin groups reach Y - cut;
  // after each 33-width block the flagged groups' windows are weighted.  Y
  // is known: no block barrier.
  auto full_block = [&](int bi, int nsteps) {
    const int w = bi * kR + nsteps;
    return !__any_sync(kFullMask, la.masked(w) || (T == 2 && lb.masked(w)));
  };
  auto step = [&](int w, int c, auto sv, auto full) {
    float g[NG];
    if constexpr (T == 2) lane_groups2<decltype(full)::value>(sv, la.at(w), lb.at(w), g);
    else lane_groups1<decltype(full)::value>(sv, la.at(w), g);
    flag_groups<true>(g, trow[c], c, lane, mk);
  };
  auto block_end = [&](int bi, int nsteps) {
        const bool drop = lane >= nsteps, drop32 = lane != 0 || nsteps != kR;
#pragma unroll
        for (int j = 0; j < NG; ++j) {
          if (drop) mk[0][j] = 0u;
          if (drop32) mk[1][j] = 0u;
        }
        const int wf = bi * kR + 1;
        block_events_cta(sgl, warp, lane, wf, mk, [&](int c) { return trow[c]; }, fh, fl, evl,
                         (blockDim.x >> 5) * kEvCap, wcnt, margin,
                     [&](int c, int k, int w, float hi, float lo) {
                       // (S - Y) from the two pairs: hi - Y is exact (Sterbenz)
                       const float g =
                           grow[c] * __expf(__fadd_rn(__fsub_rn(hi, yrow[c]), __fsub_rn(lo, ylrow[c])) * inv_tau);
                       atomicAdd(out + k, g);   // k < nb
                       const int e = k + w;
                       atomicAdd(e < t.nb ? out + e : tl + (e - t.nb), -g);
                     });
        if (bi + 1 < (W + kR - 1) / kR) load_rows(bi + 1);
      };
  if constexpr (T == 2) walk_pairs(fh, xa, xb, la.a, lb.a, W, full_block, step, block_end);
  else walk_single(fh, xa, la.a, W, full_block, step, block_end);
  __syncthreads();
  float *dd = fh;   // d_seg <= buf_len entries
  for (int j = threadIdx.x; j < d_seg; j += blockDim.x) dd[j] = __ldcg(j < t.nb ? out + j : tl + (j - t.nb));
  __syncthreads();
  // inclusive prefix sum of dd: thread t owns a contiguous chunk
  const int nt = blockDim.x;
  const int chunk = (d_seg + nt - 1) / nt;
  const int a0 = threadIdx.x * chunk, a1 = min(d_seg, a0 + chunk);
  float run = 0.0f;
  for (int j = a0; j < a1; ++j) run += dd[j];
  float incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  float base = incl - run;
  for (int v = 0; v < warp; ++v) base += wsum[v];
  float acc = base;
  for (int j = a0; j < a1; ++j) {
    acc += dd[j];
    dd[j] = acc;
  }
  __syncthreads();
  // bins of this segment, then the spill into the next one
  for (int j = threadIdx.x; j < t.nb; j += nt) out[j] = dd[j];
  for (int j = threadIdx.x; j < W - 1; j += nt) tl[j] = dd[t.nb + j];
}

// dL/dP -> C2R input, per segment (256 threads).
constexpr double kKappaB = 1.482602218505602;

__global__ void __launch_bounds__(256) normalise_backward_kernel(
    const float2 *__restrict__ spec, const float *__restrict__ dp, const float *__restrict__ tail,
    const float4 *__restrict__ stats, const float *__restrict__ sel, const SeriesDev *__restrict__ series,
    const int64_t *__restrict__ seg_off, int n_series, int seg_len, int W, float2 *__restrict__ out) {
  __shared__ float red[8][4];
  __shared__ int idx_all[8][8];
  __shared__ int idx_sh[8];
  __shared__ float sums[4];
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
  const float2 *x = spec + S.spec_off + b0;
  const float *dpp = dp + S.p_off + b0;
  const float *prev_tail = (sl > 0) ? tail + (g - 1) * static_cast<int64_t>(W) : nullptr;
  const float4 st = stats[g];
  const float med[2] = {st.x, st.z}, mad[2] = {st.y, st.w};
  const float *sv = sel + 8 * g;
  const bool even = (n % 2) == 0;
  const float inv[2] = {static_cast<float>(1.0 / (kKappaB * static_cast<double>(mad[0]))),
                        static_cast<float>(1.0 / (kKappaB * static_cast<double>(mad[1])))};
  const bool ok = mad[0] > 0.0f && mad[1] > 0.0f;
  auto val = [&](int j) -> float2 { return (b0 + j == 0) ? make_float2(0.0f, 0.0f) : x[j]; };
  auto dpv = [&](int j) -> float { return dpp[j] + ((prev_tail && j < W - 1) ? prev_tail[j] : 0.0f); };
  // block sums: S1_c = sum g_a, S2_c = sum g_a (x - med); and the selected indices
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  int idx[8] = {n, n, n, n, n, n, n, n};
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int j = tid; j < n; j += 256) {
    const float2 v = val(j);
    const float d = dpv(j);
    const float a = (v.x - med[0]) * inv[0], b = (v.y - med[1]) * inv[1];
    acc[0] += d * a;
    acc[1] += d * a * (v.x - med[0]);
    acc[2] += d * b;
    acc[3] += d * b * (v.y - med[1]);
    const float xv[2] = {v.x, v.y};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float dev = fabsf(xv[c] - med[c]);
      if (xv[c] == sv[4 * c + 0] && j < idx[4 * c + 0]) idx[4 * c + 0] = j;
      if (xv[c] == sv[4 * c + 1] && j < idx[4 * c + 1]) idx[4 * c + 1] = j;
      if (dev == sv[4 * c + 2] && j < idx[4 * c + 2]) idx[4 * c + 2] = j;
      if (dev == sv[4 * c + 3] && j < idx[4 * c + 3]) idx[4 * c + 3] = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(kFullMask, acc[q], o);
#pragma unroll
    for (int q = 0; q < 8; ++q) idx[q] = min(idx[q], __shfl_xor_sync(kFullMask, idx[q], o));
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) red[wid][q] = acc[q];
#pragma unroll
    for (int q = 0; q < 8; ++q) idx_all[wid][q] = idx[q];
  }
  __syncthreads();
  if (tid < 8) {
    int m = n;
    for (int v = 0; v < 8; ++v) m = min(m, idx_all[v][tid]);
    idx_sh[tid] = m;
  }
  if (tid < 4) {
    float z = 0.0f;
    for (int v = 0; v < 8; ++v) z += red[v][tid];
    sums[tid] = z;
  }
  __syncthreads();
  // the second middle statistic may tie with the first: then take the next occurrence
  if (even) {
    if (tid < 4) {
      const int c = tid >> 1, q = (tid & 1) ? 2 : 0;   // (median | deviation) pair of component c
      const int first = idx_sh[4 * c + q], second = idx_sh[4 * c + q + 1];
      if (second == first) {
        int nxt = n;
        for (int j = first + 1; j < n; ++j) {
          const float2 v = val(j);
          const float xv = c ? v.y : v.x;
          const float test = q ? fabsf(xv - med[c]) : xv;
          if (test == sv[4 * c + q + 1]) {
            nxt = j;
            break;
          }
        }
        idx_sh[4 * c + q + 1] = nxt;
      }
    }
    __syncthreads();
  }
  const float wsel = even ? 0.5f : 1.0f;
  const int64_t half = S.m - 1;   // Nyquist bin index = N / 2
  for (int j = tid; j < n; j += 256) {
    const float2 v = val(j);
    const float d = dpv(j);
    const float xv[2] = {v.x, v.y};
    float gx[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float scale_inv = inv[c];
      const float ac = (xv[c] - med[c]) * scale_inv;
      const float ga = d * ac;
      const int m_lo = idx_sh[4 * c + 0], m_hi = even ? idx_sh[4 * c + 1] : -1;
      const int d_lo = idx_sh[4 * c + 2], d_hi = even ? idx_sh[4 * c + 3] : -1;
      const float dmed = wsel * ((j == m_lo) ? 1.0f : 0.0f) + wsel * ((j == m_hi) ? 1.0f : 0.0f);
      // sign(x_m - med) at the selected deviations (read from the staged spectrum)
      const float x_dlo = (d_lo < n) ? (c ? val(d_lo).y : val(d_lo).x) : med[c];
      const float x_dhi = (even && d_hi < n) ? (c ? val(d_hi).y : val(d_hi).x) : med[c];
      const float sg_lo = (x_dlo > med[c]) ? 1.0f : ((x_dlo < med[c]) ? -1.0f : 0.0f);
      const float sg_hi = even ? ((x_dhi > med[c]) ? 1.0f : ((x_dhi < med[c]) ? -1.0f : 0.0f)) : 0.0f;
      const float dmad = wsel * sg_lo * ((j == d_lo) ? 1.0f : 0.0f) + wsel * sg_hi * ((j == d_hi) ? 1.0f : 0.0f) -
                         wsel * (sg_lo + sg_hi) * dmed;
      const float s1 = sums[2 * c], s2 = sums[2 * c + 1];
      gx[c] = ok ? (ga * scale_inv - s1 * scale_inv * dmed - s2 * scale_inv / mad[c] * dmad) : 0.0f;
    }
    const int64_t k = b0 + j;
    float2 o;
    if (k == 0) {
      o = make_float2(0.0f, 0.0f);           // DC := 0 carries no gradient
    } else if (k == half) {
      o = make_float2(gx[0], 0.0f);          // Nyquist: real
    } else {
      o = make_float2(0.5f * gx[0], 0.5f * gx[1]);
    }
    out[S.spec_off + k] = o;
  }
}

__global__ void inject_kernel(const float *__restrict__ noise, const float *__restrict__ tmpl,
                              const float *__restrict__ amp, const SeriesDev *__restrict__ series,
                              const int64_t *__restrict__ x_off, const int64_t *__restrict__ x_len, int n_series,
                              float *__restrict__ x) {
  const int si = blockIdx.y;
  if (si >= n_series) return;
  const int64_t off = x_off[si], len = x_len[si];
  const float a = amp[series[si].user_index];
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < len;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[off + i] = fmaf(a, tmpl[off + i], noise[off + i]);
}

// dL/dA per series in two steps: CTA (chunk, series) reduces its 1/kAmpChunks of
// the series (FP32 runs of 64 products folded into FP64) into a partial;
// then one warp per series adds its partials in chunk order (deterministic).
// Many CTAs per series keep the read of dL/dx and the template at HBM rate.
constexpr int kAmpChunks = 16;

__global__ void __launch_bounds__(256) amp_grad_partial_kernel(const float *__restrict__ gx,
                                                               const float *__restrict__ tmpl,
                                                               const int64_t *__restrict__ x_off,
                                                               const int64_t *__restrict__ x_len, int n_series,
                                                               double *__restrict__ part_out) {
  const int si = blockIdx.y, ch = blockIdx.x;
  if (si >= n_series) return;
  const int64_t off = x_off[si], len = x_len[si];
  const int64_t lo = len * ch / kAmpChunks, hi = len * (ch + 1) / kAmpChunks;
  double acc = 0.0;
  float part = 0.0f;
  int cnt = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    part = fmaf(__ldg(gx + off + i), __ldg(tmpl + off + i), part);
    if (++cnt == 64) {   // fold into FP64 every 64 terms
      acc += part;
      part = 0.0f;
      cnt = 0;
    }
  }
  acc += part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFullMask, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double z = 0.0;
    for (int v = 0; v < static_cast<int>(blockDim.x >> 5); ++v) z += red[v];
    part_out[static_cast<int64_t>(si) * kAmpChunks + ch] = z;
  }
}

__global__ void amp_grad_sum_kernel(const double *__restrict__ part, const SeriesDev *__restrict__ series,
                                    int n_series, float *__restrict__ gamp) {
  const int si = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (si >= n_series) return;
  double z = (lane < kAmpChunks) ? part[static_cast<int64_t>(si) * kAmpChunks + lane] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(kFullMask, z, o);
  if (lane == 0) gamp[series[si].user_index] = static_cast<float>(z);
}

// Tiles per lane of the logsumexp kernels: one (scalar adds; 66 ring and
// window registers, about 20 warps per SM) measured 1.33x faster than two
// packed tiles (132 registers, 12 warps per SM) on the forward kernel.
constexpr int kLseTiles = 1;

// Warps per segment CTA for warps of `span` bins.

int lse_warps(pulscan_plan p, int span = kSpan) {
  int64_t max_n = 0;
  for (const auto &se : p->series) max_n = std::max<int64_t>(max_n, se.m - (se.n_seg - 1) * p->seg_len);
  return static_cast<int>((max_n + span - 1) / span);
}

int lse_buf_len(pulscan_plan p, int warps, int span = kSpan) {
  const int nb = (p->z_max + kR - 1) / kR;
  return ((span * warps + nb * kR + 3 * kR) + 3) & ~3;
}

SmemLimit g_lim_fwd, g_lim_bwd;

int lse_prepare(pulscan_plan p) {
  if (p->numharm > 1) return fail(PULSCAN_ERR_UNSUPPORTED, "logsumexp path on a harmonic plan");
  if (p->fidelity != PULSCAN_FIDELITY_EXACT)
    return fail(PULSCAN_ERR_UNSUPPORTED, "logsumexp path in the median-of-medians mode");
  if (lse_warps(p) > kLseMaxWarps)
    return fail(PULSCAN_ERR_UNSUPPORTED, "logsumexp path needs segments of at most 4224 bins");
  return PULSCAN_OK;
}

int lse_backward_buffers(pulscan_plan p) {
  if (!p->d_dp) PS_CUDA(cudaMalloc(reinterpret_cast<void **>(&p->d_dp), sizeof(float) * p->p_floats));
  if (!p->d_tail)
    PS_CUDA(cudaMalloc(reinterpret_cast<void **>(&p->d_tail), sizeof(float) * p->total_seg * p->z_max));
  if (!p->d_gspec) PS_CUDA(cudaMalloc(reinterpret_cast<void **>(&p->d_gspec), 2 * sizeof(float) * p->spec_bins));
  if (p->ifft.empty()) {
    for (const auto &f : p->fft) {
      FftClass g = f;
      g.handle = 0;
      long long nn = f.n, inembed = f.spec_stride, onembed = f.n;
      size_t work = 0;
      cufftResult r = cufftCreate(&g.handle);
      if (r == CUFFT_SUCCESS)
        r = cufftMakePlanMany64(g.handle, 1, &nn, &inembed, 1, f.spec_stride, &onembed, 1, f.n, CUFFT_C2R, f.count,
                                &work);
      if (r != CUFFT_SUCCESS) {
        if (g.handle) cufftDestroy(g.handle);
        return fail(r == CUFFT_ALLOC_FAILED ? PULSCAN_ERR_NOMEM : PULSCAN_ERR_CUDA, "cuFFT C2R plan failed");
      }
      p->ifft.push_back(g);
    }
  }
  return PULSCAN_OK;
}

float lse_cut(pulscan_plan p, float tau) {
  // windows more than tau ln 2^24 below the maximum each weigh < 2^-24 of it;
  // at most 2L of them (a segment's start bins) add < 2L 2^-24 to the sum
  // (>= 1), i.e. < tau 2L 2^-24 to Y (1.2e-5 tau per 1000 bins of segment),
  // below Y's FP32 resolution except for the smallest widths, and each
  // dropped weight changes dL/dP by < 2^-24 of the largest one
  (void)p;
  return tau * static_cast<float>(std::log(16777216.0));
}

}  // namespace

}  // namespace ps

using namespace ps;

extern "C" {

int pulscan_lse_forward(pulscan_plan p, const float *d_x, float *d_spec, float *d_power, float *d_stats,
                        float *d_sel, float *d_y, float *d_ylo, float tau, pulscan_stream stream) {
  if (!p || !d_x || !d_spec || !d_power || !d_stats || !d_sel || !d_y || !d_ylo)
    return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (!(tau > 0.0f) || !std::isfinite(tau)) return fail(PULSCAN_ERR_INVALID_ARG, "tau must be finite and > 0");
  int rc = lse_prepare(p);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rc = pulscan_rfft(p, d_x, d_spec, stream);
  if (rc) return rc;
  rc = launch_normalise_sel(p, d_spec, d_power, d_stats, d_sel, s);
  if (rc) return rc;
  constexpr int span = kLseTiles * kTile;
  const int warps = lse_warps(p, span);
  const int buf_len = lse_buf_len(p, warps, span);
  const int smem = 128 + 4 * (buf_len + 1 + 6 * kRows + warps * kEvCap) + 2 * (buf_len + 1) + 16;
  rc = ensure_smem(lse_forward_kernel<kLseTiles>, smem, g_lim_fwd);
  if (rc) return rc;
  lse_forward_kernel<kLseTiles><<<static_cast<unsigned>(p->total_seg), 32 * warps, smem, s>>>(
      d_power, p->d_series, p->d_seg_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len, tau,
      lse_cut(p, tau), d_y, d_ylo, p->d_counters, buf_len);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

int pulscan_lse_backward(pulscan_plan p, const float *d_spec, const float *d_power, const float *d_stats,
                         const float *d_sel, const float *d_y, const float *d_ylo, const float *d_gy, float *d_gx,
                         float tau, pulscan_stream stream) {
  if (!p || !d_spec || !d_power || !d_stats || !d_sel || !d_y || !d_ylo || !d_gy || !d_gx)
    return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  if (!(tau > 0.0f) || !std::isfinite(tau)) return fail(PULSCAN_ERR_INVALID_ARG, "tau must be finite and > 0");
  int rc = lse_prepare(p);
  if (rc) return rc;
  rc = lse_backward_buffers(p);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  constexpr int span = kLseTiles * kTile;
  const int warps = lse_warps(p, span);
  const int buf_len = lse_buf_len(p, warps, span);
  const int smem = 128 + 4 * (buf_len + 1 + kBwdRows + 32 + warps * kEvCap) + 2 * (buf_len + 1) + 16;
  rc = ensure_smem(lse_backward_kernel<kLseTiles>, smem, g_lim_bwd);
  if (rc) return rc;
  lse_backward_kernel<kLseTiles><<<static_cast<unsigned>(p->total_seg), 32 * warps, smem, s>>>(
      d_power, p->d_series, p->d_seg_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len, tau,
      lse_cut(p, tau), d_y, d_ylo, d_gy, p->d_dp, p->d_tail, p->d_counters, buf_len);
  PS_CUDA(cudaGetLastError());
  normalise_backward_kernel<<<static_cast<unsigned>(p->total_seg), 256, 0, s>>>(
      reinterpret_cast<const float2 *>(d_spec), p->d_dp, p->d_tail, reinterpret_cast<const float4 *>(d_stats),
      d_sel, p->d_series, p->d_seg_off, static_cast<int>(p->series.size()), p->seg_len, p->z_max,
      reinterpret_cast<float2 *>(p->d_gspec));
  PS_CUDA(cudaGetLastError());
  for (auto &f : p->ifft) {
    cufftResult r = cufftSetStream(f.handle, s);
    if (r == CUFFT_SUCCESS)
      r = cufftExecC2R(f.handle, reinterpret_cast<cufftComplex *>(p->d_gspec) + f.spec_off, d_gx + f.x_off);
    if (r != CUFFT_SUCCESS) return fail(PULSCAN_ERR_CUDA, "cufftExecC2R failed");
  }
  return PULSCAN_OK;
}

int pulscan_inject(pulscan_plan p, const float *d_noise, const float *d_template, const float *d_amp, float *d_x,
                   pulscan_stream stream) {
  if (!p || !d_noise || !d_template || !d_amp || !d_x) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int ns = static_cast<int>(p->n_base);
  if (ns > 65535) return fail(PULSCAN_ERR_UNSUPPORTED, "too many series for one launch");
  inject_kernel<<<dim3(64, ns), 256, 0, s>>>(d_noise, d_template, d_amp, p->d_series, p->d_x_off, p->d_x_len, ns,
                                             d_x);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

int pulscan_amplitude_grad(pulscan_plan p, const float *d_gx, const float *d_template, float *d_gamp,
                           pulscan_stream stream) {
  if (!p || !d_gx || !d_template || !d_gamp) return fail(PULSCAN_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int ns = static_cast<int>(p->n_base);
  if (ns > 65535) return fail(PULSCAN_ERR_UNSUPPORTED, "too many series for one launch");
  if (!p->d_amp_part)
    PS_CUDA(cudaMalloc(reinterpret_cast<void **>(&p->d_amp_part), sizeof(double) * kAmpChunks * ns));
  amp_grad_partial_kernel<<<dim3(kAmpChunks, ns), 256, 0, s>>>(d_gx, d_template, p->d_x_off, p->d_x_len, ns,
                                                                p->d_amp_part);
  PS_CUDA(cudaGetLastError());
  amp_grad_sum_kernel<<<(ns + 7) / 8, 256, 0, s>>>(p->d_amp_part, p->d_series, ns, d_gamp);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // extern "C"
