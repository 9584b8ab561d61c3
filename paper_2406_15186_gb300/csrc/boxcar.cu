// Boxcar filter bank + per-(segment, width) maximum (paper §2.2.5 and
// Algorithm 4), GB300 design.
//
// Work decomposition: a CTA of 1 to 4 warps owns a tile of 1056 bins per
// warp (consecutive start bins of one series); lane l of warp v owns the
// kR = 33 start bins k0 .. k0+32, k0 = tile + 33 (32 v + l).  The tile plus its halo
// of z_max bins is staged into shared memory by one TMA bulk copy.  Each lane
// keeps its 33 running sums s_i = S_w[k0+i] in registers and walks w = 1..W:
// step w adds P[k0+i+w-1] to s_i (one FP32 add per (bin, width), the
// recursion Y_w = Y_{w-1}[:end-1] + X[w:end] of §2.2.5 applied per bin).  The
// 33 window values live in a register ring that takes one new shared-memory
// load per step; the stride between lanes (33 floats) is odd, so those loads
// are bank-conflict free.  The width loop is unrolled by 33 so every ring
// index is a compile-time constant.
//
// Search mode only needs the maxima that reach the threshold T_w.  Because
// P >= 0, a block of 33 bins x 33 widths starting at width w0 satisfies
//   S_w[k0+i] <= S_{w0-1}[k0] + sum_{x=k0+w0-1}^{k0+w0+63} P[x]
// for all i < 33, w0 <= w < w0+33, and the second term is one pre-summed
// 66-bin window.  Only when some lane's bound reaches T_{w0} does the warp
// run the block in "exact" mode: the same adds, plus a compare of every sum
// with T_w and a segmented warp max-reduction of the hits.  For the first
// widths (w <= 132), where T_w is far above w but the block bound is loose,
// the bound is taken per 11 bins x 11 widths.  The maxima themselves are
// merged across warps and CTAs with a 64-bit atomicMax on
// (power bits << 32 | ~bin) per (segment, width) slot: the largest power
// wins, ties go to the lowest bin (the first index of Algorithm 4's scan).
//
// Dump mode (pulscan_segment_maxima) runs every block exactly and merges the
// maximum of every (segment, width) with no threshold.
#include <algorithm>

#include "bank.cuh"
#include "common.cuh"
#include "ptx.cuh"

namespace ps {

namespace {

constexpr unsigned kFull = 0xffffffffu;


struct LaneCtx {
  int64_t k0;          // series-relative first bin of the lane
  int64_t m;           // bins of the series
  int lim_tile;        // lane bins that belong to this tile (may be <= 0)
  int64_t seg_a;       // global segment of bin k0 (clamped to the series)
  int ib;              // first lane bin index that lies in segment seg_a + 1 (33 if none)
  int64_t seg_last;    // global index of the series' last segment
  int seg_len;
  int64_t seg_base;    // global index of the series' first segment
  int W;
  unsigned long long *slots;
  uint32_t *dirty;
};

__device__ __forceinline__ unsigned long long slot_key(float v, uint32_t bin) {
  return (static_cast<unsigned long long>(__float_as_uint(v)) << 32) |
         static_cast<unsigned long long>(0xffffffffu - bin);
}

// Merge one (segment, width) maximum into its slot.  Both updates are
// fire-and-forget reductions (no value returned, so the warp does not wait
// for the round trip): the 64-bit max on the slot, and in search mode one bit
// in the dirty bitmap that tells the finaliser which slots to visit.
template <bool kSearch>
__device__ __forceinline__ void emit_slot(unsigned long long *slots, uint32_t *dirty, uint64_t idx,
                                          unsigned long long key) {
  atomicMax(slots + idx, key);
  if (kSearch) atomicOr(dirty + (idx >> 5), 1u << (idx & 31u));
}

// Lowest lane-bin index i in [ia, ib) with s_i == v (kR if none).
__device__ __forceinline__ int first_equal(const float (&s)[kR], float v, int ia, int ib) {
  int idx = kR;
#pragma unroll
  for (int i = kR - 1; i >= 0; --i) idx = (s[i] == v && i >= ia && i < ib) ? i : idx;
  return idx;
}

// Three-input maximum (one instruction on sm_100 and later); like fmaxf it
// returns one of its operands and ignores NaN operands.
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// One exact step's merge.  Each lane offers the maximum of its valid bins in
// segment seg_a (bins [0, ib)) and, for the one lane that straddles a
// segment boundary, in seg_a + 1 (bins [ib, lim)); v < 0 means no valid bin.
// For each of the warp's first two segments the warp reduces the maximum,
// drops it if it is below T (search mode), finds the lowest bin holding it,
// and lane 0 merges it into the (segment, width) slot.  Parts in a third
// segment (segment_len < 1056 only) are merged lane by lane.
template <bool kSearch>
__device__ __forceinline__ void merge_step(const float (&s)[kR], const LaneCtx &c, int w, float T, float vA,
                                           float vB, int lim) {
  const int64_t s_first = __shfl_sync(kFull, c.seg_a, 0);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int64_t X = s_first + t;
    const bool isA = (c.seg_a == X);
    const bool isB = (c.seg_a + 1 == X);
    const float v = isA ? vA : (isB ? vB : -1.0f);
    const uint32_t bits = (v >= 0.0f) ? __float_as_uint(v) : 0u;
    const unsigned has = __ballot_sync(kFull, v >= 0.0f);
    if (has == 0u) continue;
    const uint32_t bmax = __reduce_max_sync(kFull, bits);
    const float vmax = __uint_as_float(bmax);
    if (kSearch && !(vmax >= T)) continue;
    uint32_t bin = 0xffffffffu;
    if (v >= 0.0f && bits == bmax) {
      const int i = isA ? first_equal(s, vmax, 0, min(c.ib, lim)) : first_equal(s, vmax, c.ib, lim);
      bin = static_cast<uint32_t>(c.k0 + i);
    }
    const uint32_t bmin = __reduce_min_sync(kFull, bin);
    if ((threadIdx.x & 31) == 0)
      emit_slot<kSearch>(c.slots, c.dirty, static_cast<uint64_t>(X) * c.W + (w - 1), slot_key(vmax, bmin));
  }
  // parts outside the warp's first two segments
  if (vA >= 0.0f && c.seg_a > s_first + 1 && (!kSearch || vA >= T)) {
    const int i = first_equal(s, vA, 0, min(c.ib, lim));
    emit_slot<kSearch>(c.slots, c.dirty, static_cast<uint64_t>(c.seg_a) * c.W + (w - 1),
                       slot_key(vA, static_cast<uint32_t>(c.k0 + i)));
  }
  if (vB >= 0.0f && c.seg_a + 1 > s_first + 1 && (!kSearch || vB >= T)) {
    const int i = first_equal(s, vB, c.ib, lim);
    emit_slot<kSearch>(c.slots, c.dirty, static_cast<uint64_t>(c.seg_a + 1) * c.W + (w - 1),
                       slot_key(vB, static_cast<uint32_t>(c.k0 + i)));
  }
}

// Exact mode: steps w = wf + cb .. wf + ce - 1 with every window inspected.
// The sums stay in registers (static index i); the window is read straight
// from shared memory (33 loads per step).  Branch-free per bin: the lane's
// maxima over its valid bins are max-reductions with selects, and the bin
// index is searched only by the lane(s) holding the warp maximum.
// kSearch: only maxima >= T_w are merged; otherwise every maximum is.
// wshift: lane_buf[w - 1 - wshift + i] is the window value of bin i at width
// w (a window staged from width wshift + 1 on).
template <bool kSearch>
__device__ __forceinline__ void exact_steps(float (&s)[kR], const float *__restrict__ lane_buf, int wf,
                                            int cb, int ce, const float *__restrict__ thr,
                                            const LaneCtx &c, int wshift = 0) {
  // segment_len < 66 lets a lane's 33 bins reach a third segment: then every
  // bin is merged on its own (only tiny test shapes take this branch)
  const bool small_seg = c.seg_len < 2 * kR;
  const bool any_split = __any_sync(kFull, c.ib < kR);
  for (int cc = cb; cc < ce; ++cc) {
    const int w = wf + cc;
    const float *pw = lane_buf + (w - 1 - wshift);
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] += pw[i];
    // valid bins: inside the tile, and the window inside the spectrum
    const int64_t lim64 = c.m - w + 1 - c.k0;
    const int lim = static_cast<int>(min64(static_cast<int64_t>(c.lim_tile), max64(lim64, 0)));
    const float T = kSearch ? thr[w - 1] : 0.0f;
    if (small_seg) {
#pragma unroll
      for (int i = 0; i < kR; ++i) {
        if (i < lim && (!kSearch || s[i] >= T)) {
          const int64_t sg = c.seg_base + min64((c.k0 + i) / c.seg_len, c.seg_last - c.seg_base);
          emit_slot<kSearch>(c.slots, c.dirty, static_cast<uint64_t>(sg) * c.W + (w - 1),
                             slot_key(s[i], static_cast<uint32_t>(c.k0 + i)));
        }
      }
      continue;
    }
    const int la = min(c.ib, lim);   // part A: bins [0, la)
    float vA = -1.0f, vB = -1.0f;
#pragma unroll
    for (int i = 0; i < kR; ++i) vA = fmaxf(vA, (i < la) ? s[i] : -1.0f);
    if (any_split) {
#pragma unroll
      for (int i = 0; i < kR; ++i) vB = fmaxf(vB, (i >= c.ib && i < lim) ? s[i] : -1.0f);
    }
    // nothing to merge if no valid bin reaches T anywhere in the warp
    if (kSearch && !__any_sync(kFull, vA >= T || vB >= T)) continue;
    merge_step<kSearch>(s, c, w, T, vA, vB, lim);
  }
}

// Bound test of one 11-width sub-block of an early block: three groups of
// 11 bins, each bounded by s_{11 j} plus a pre-summed window of 22 bins.
__device__ __forceinline__ bool early_bound(const float (&s)[kR], const float *__restrict__ q11, int qb, float tb) {
  return (s[0] + q11[qb] + q11[qb + 1] >= tb) || (s[kSub] + q11[qb + 1] + q11[qb + 2] >= tb) ||
         (s[2 * kSub] + q11[qb + 2] + q11[qb + 3] >= tb);
}

// Lane context for lane `lane` of warp `warp` of the tile starting at bin t0.
__device__ __forceinline__ LaneCtx lane_ctx(const SeriesDev &S, int64_t t0, int tile_bins, int warp, int lane,
                                            int W, int seg_len, unsigned long long *slots, uint32_t *dirty) {
  LaneCtx c;
  c.k0 = t0 + warp * (32 * kR) + lane * kR;
  c.m = S.m;
  const int64_t tile_end = min64(t0 + static_cast<int64_t>(tile_bins), S.m);
  c.lim_tile = static_cast<int>(max64(min64(tile_end - c.k0, kR), -1));
  c.seg_len = seg_len;
  c.seg_base = S.seg_off;
  c.seg_last = S.seg_off + S.n_seg - 1;
  const int64_t sa_local = min64(c.k0 / seg_len, S.n_seg - 1);
  c.seg_a = S.seg_off + sa_local;
  c.ib = (sa_local < S.n_seg - 1) ? static_cast<int>(min64((sa_local + 1) * seg_len - c.k0, kR)) : kR;
  c.W = W;
  c.slots = slots;
  c.dirty = dirty;
  return c;
}

__device__ __forceinline__ int series_of_tile(const int64_t *__restrict__ tile_off, int n_series, int64_t tile) {
  int lo = 0, hi = n_series - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_off[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Deferred block: (tile, virtual warp, block, first step) packed in 64 bits:
// tile in bits 0-39, the virtual warp (the 1056-bin slice of the tile, 0..7)
// in 40-42, the 33-width block in 43-55, the first step in 56-63.
__device__ __forceinline__ unsigned long long pack_item(int64_t tile, int warp, int bi, int cx) {
  return static_cast<unsigned long long>(tile) | (static_cast<unsigned long long>(warp) << 40) |
         (static_cast<unsigned long long>(bi) << 43) | (static_cast<unsigned long long>(cx) << 56);
}

// Defer the rest of block bi (steps cx..) of this warp: append a work item
// and snapshot the 33 running sums (coalesced, [item][bin][lane]).  Returns
// false when the list is full; the caller then runs the block exactly inline.
__device__ __forceinline__ bool defer_block(const float (&s)[kR], unsigned long long *__restrict__ items,
                                            float *__restrict__ snaps, uint32_t *__restrict__ counters,
                                            uint32_t cap, int64_t tile, int warp, int bi, int cx) {
  const int lane = threadIdx.x & 31;
  uint32_t idx = 0;
  if (lane == 0) idx = atomicAdd(counters + 0, 1u);
  idx = __shfl_sync(kFull, idx, 0);
  if (idx >= cap) return false;
  if (lane == 0) items[idx] = pack_item(tile, warp, bi, cx);
  float *sp = snaps + static_cast<size_t>(idx) * (kR * 32) + lane;
#pragma unroll
  for (int i = 0; i < kR; ++i) sp[i * 32] = s[i];
  return true;
}

// Two adds in one instruction: (a, b) += (x, y) by add.rn.f32x2, the packed
// FP32 add of sm_100 and later.  Each half rounds exactly as a scalar
// add.rn.f32 would, so the sums are bit-identical to the scalar bank's.
__device__ __forceinline__ void add_pair(float &a, float &b, float x, float y) {
  asm("{\n\t.reg .b64 s, v;\n\t"
      "mov.b64 s, {%0, %1};\n\t"
      "mov.b64 v, {%2, %3};\n\t"
      "add.rn.f32x2 s, s, v;\n\t"
      "mov.b64 {%0, %1}, s;\n\t}"
      : "+f"(a), "+f"(b)
      : "f"(x), "f"(y));
}

// Packed form of fast_steps: a lane carries two 33-bin groups (A and B, 1056
// bins apart) with one ring each, and adds them pairwise.
template <int C0, int NC>
__device__ __forceinline__ void fast_steps2(float (&sA)[kR], float (&sB)[kR], float (&bA)[kR], float (&bB)[kR],
                                            const float *__restrict__ pA, const float *__restrict__ pB) {
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    const int c = C0 + cc;
    bA[(c + kR - 1) % kR] = pA[c + kR - 1];
    bB[(c + kR - 1) % kR] = pB[c + kR - 1];
#pragma unroll
    for (int i = 0; i < kR; ++i) add_pair(sA[i], sB[i], bA[(i + c) % kR], bB[(i + c) % kR]);
  }
}

// The search over one staged tile with packed adds (two virtual warps per
// warp).  The block logic is the scalar one's, once per group: a group whose
// bound reaches the threshold is deferred (its own item and snapshot) while
// both groups go on with packed adds; if the item list is full, the rest of
// that block runs in scalar code for both groups (the flagged one exactly).
// The lane contexts are only needed on that rare path and are formed there
// (from the series descriptor in global memory), so they hold no registers
// in the packed loop.
__device__ __forceinline__ void packed_bank(const float *__restrict__ buf, const float *__restrict__ q11,
                                         const float *__restrict__ q33, const SeriesDev &S0, int si, int64_t tile,
                                         int64_t t0, int tile_bins, int W, int seg_len, const float *__restrict__ thr,
                                         const float *__restrict__ thrb, unsigned long long *__restrict__ slots,
                                         uint32_t *__restrict__ dirty, uint32_t *__restrict__ counters,
                                         unsigned long long *__restrict__ items, float *__restrict__ snaps,
                                         uint32_t item_cap, const SeriesDev *__restrict__ series) {
  (void)S0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vA = 2 * warp, vB = 2 * warp + 1;
  const int xA = vA * (32 * kR) + lane * kR, xB = xA + 32 * kR;
  const float *lA = buf + xA, *lB = buf + xB;
  float sA[kR], sB[kR], bA[kR], bB[kR];
#pragma unroll
  for (int i = 0; i < kR; ++i) {
    sA[i] = 0.0f;
    sB[i] = 0.0f;
  }
#pragma unroll
  for (int j = 0; j < kR - 1; ++j) {
    bA[j] = lA[j];
    bB[j] = lB[j];
  }
  bA[kR - 1] = 0.0f;
  bB[kR - 1] = 0.0f;
  const int nb = (W + kR - 1) / kR;
  const int qbA = xA / kSub, qcA = xA / kR, qbB = xB / kSub, qcB = xB / kR;
  // the rest of block bi from step cb in scalar code; a group flagged ex
  // runs exactly (every window compared), the other one plain adds
  auto finish_scalar = [&](int bi, int cb, int nsteps, bool exA, bool exB) {
    const SeriesDev S = series[si];
    const int wf = bi * kR + 1;
    if (exA) {
      const LaneCtx c = lane_ctx(S, t0, tile_bins, vA, lane, W, seg_len, slots, dirty);
      exact_steps<true>(sA, lA, wf, cb, nsteps, thr, c);
    } else {
      tail_steps(sA, lA, wf + cb, wf + nsteps);
    }
    if (exB) {
      const LaneCtx c = lane_ctx(S, t0, tile_bins, vB, lane, W, seg_len, slots, dirty);
      exact_steps<true>(sB, lB, wf, cb, nsteps, thr, c);
    } else {
      tail_steps(sB, lB, wf + cb, wf + nsteps);
    }
    reload_ring<kR>(bA, lA + bi * kR);
    reload_ring<kR>(bB, lB + bi * kR);
  };
  for (int bi = 0; bi < nb; ++bi) {
    const float *pA = lA + bi * kR, *pB = lB + bi * kR;
    const int wf = bi * kR + 1;
    const int nsteps = min(kR, W - bi * kR);
    const bool early = bi < kEarlyBlocks;
    bool defA = false, defB = false, exA = false, exB = false;
    {
      const float tb = thrb[wf - 1];
      const bool hA = early ? early_bound(sA, q11, qbA + 3 * bi, tb)
                            : (sA[0] + q33[qcA + bi] + q33[qcA + bi + 1] >= tb);
      const bool hB = early ? early_bound(sB, q11, qbB + 3 * bi, tb)
                            : (sB[0] + q33[qcB + bi] + q33[qcB + bi + 1] >= tb);
      if (__any_sync(kFull, hA)) {
        if (defer_block(sA, items, snaps, counters, item_cap, tile, vA, bi, 0)) defA = true;
        else exA = true;
      }
      if (__any_sync(kFull, hB)) {
        if (defer_block(sB, items, snaps, counters, item_cap, tile, vB, bi, 0)) defB = true;
        else exB = true;
      }
    }
    if (exA || exB) {
      finish_scalar(bi, 0, nsteps, exA, exB);
      continue;
    }
    if (nsteps < kSub) {
      tail_steps(sA, lA, wf, wf + nsteps);
      tail_steps(sB, lB, wf, wf + nsteps);
      continue;
    }
    fast_steps2<0, kSub>(sA, sB, bA, bB, pA, pB);
    if (early && nsteps > kSub) {
      const float tb = thrb[wf + kSub - 1];
      if (!defA && __any_sync(kFull, early_bound(sA, q11, qbA + 3 * bi + 1, tb))) {
        if (defer_block(sA, items, snaps, counters, item_cap, tile, vA, bi, kSub)) defA = true;
        else exA = true;
      }
      if (!defB && __any_sync(kFull, early_bound(sB, q11, qbB + 3 * bi + 1, tb))) {
        if (defer_block(sB, items, snaps, counters, item_cap, tile, vB, bi, kSub)) defB = true;
        else exB = true;
      }
      if (exA || exB) {
        finish_scalar(bi, kSub, nsteps, exA, exB);
        continue;
      }
    }
    if (nsteps < 2 * kSub) {
      tail_steps(sA, lA, wf + kSub, wf + nsteps);
      tail_steps(sB, lB, wf + kSub, wf + nsteps);
      continue;
    }
    fast_steps2<kSub, kSub>(sA, sB, bA, bB, pA, pB);
    if (early && nsteps > 2 * kSub) {
      const float tb = thrb[wf + 2 * kSub - 1];
      if (!defA && __any_sync(kFull, early_bound(sA, q11, qbA + 3 * bi + 2, tb))) {
        if (!defer_block(sA, items, snaps, counters, item_cap, tile, vA, bi, 2 * kSub)) exA = true;
      }
      if (!defB && __any_sync(kFull, early_bound(sB, q11, qbB + 3 * bi + 2, tb))) {
        if (!defer_block(sB, items, snaps, counters, item_cap, tile, vB, bi, 2 * kSub)) exB = true;
      }
      if (exA || exB) {
        finish_scalar(bi, 2 * kSub, nsteps, exA, exB);
        continue;
      }
    }
    if (nsteps < kR) {
      tail_steps(sA, lA, wf + 2 * kSub, wf + nsteps);
      tail_steps(sB, lB, wf + 2 * kSub, wf + nsteps);
      continue;
    }
    fast_steps2<2 * kSub, kSub>(sA, sB, bA, bB, pA, pB);
  }
}

// One tile: stage P[t0, t0 + buf_len) by a TMA bulk copy, form the bound
// sums, run the bank.  Returns false when the copy timed out (flagged).
// groups = 1: warp v owns bins [1056 v, 1056 (v + 1)) of the tile, a lane 33
// of them.  groups = 2 (tiles twice as wide): warp v owns the two slices
// ("virtual warps") 2v and 2v + 1; in search mode (kPacked) each lane carries
// one 33-bin group of each and adds both with packed instructions, in dump
// mode the warp runs the two slices one after the other.  A virtual warp is
// the unit of the deferred-block items either way.
// The fused search (normalisation on the fly, Eq. 8): P of series bin k from
// the spectrum and its segment's (med_re, 1 / (kappa MAD_re), med_im,
// 1 / (kappa MAD_im)), the DC bin taken as 0 + 0i; the segment of bin k is
// min(k / L, n_seg - 1).  Bit-identical to the normalisation kernel's P.
__device__ __forceinline__ float fused_power(const float2 *__restrict__ spec, const float4 *__restrict__ norm,
                                            const SeriesDev &S, int64_t k, int seg_len) {
  const float2 x = (k == 0) ? make_float2(0.0f, 0.0f) : __ldg(spec + S.spec_off + k);
  const uint32_t sg = min(static_cast<uint32_t>(k) / static_cast<uint32_t>(seg_len),
                          static_cast<uint32_t>(S.n_seg - 1));
  return power_of(x.x, x.y, __ldg(norm + S.seg_off + sg));
}

// buf[i] = P[t0 + i] for i < avail, 0 up to buf_len, formed from the
// spectrum segment by segment (one statistics load per segment).
__device__ __forceinline__ void stage_fused(float *buf, int buf_len, int avail, const SeriesDev &S, int64_t t0,
                                            int seg_len, const float2 *__restrict__ spec,
                                            const float4 *__restrict__ norm) {
  const int64_t last = S.n_seg - 1;
  int64_t seg = min64(t0 / seg_len, last);
  for (int a = 0; a < avail; ++seg) {
    const int64_t seg_end = (seg == last) ? S.m : (seg + 1) * seg_len;
    const int b = static_cast<int>(min64(seg_end - t0, static_cast<int64_t>(avail)));
    const float4 nrm = __ldg(norm + S.seg_off + seg);
    for (int i = a + static_cast<int>(threadIdx.x); i < b; i += blockDim.x) {
      const int64_t k = t0 + i;
      const float2 x = (k == 0) ? make_float2(0.0f, 0.0f) : __ldg(spec + S.spec_off + k);
      buf[i] = power_of(x.x, x.y, nrm);
    }
    a = b;
  }
  for (int i = avail + static_cast<int>(threadIdx.x); i < buf_len; i += blockDim.x) buf[i] = 0.0f;
}

// ---------------------------------------------------------------------------
// Dump mode: every (segment, width) maximum, no threshold.
//
// A slice whose lanes each lie in one of two segments X0, X0 + 1 (at most one
// lane straddles the boundary) walks the widths at which all its windows are
// inside the tile and the series with a lean per-step merge: each lane's
// maximum from eleven 3-bin group maxima, one warp max-reduction per segment,
// and the lowest lane holding the warp maximum alone finds its bin and merges
// the key.  A whole lane finds the bin through its group maxima (the first
// group holding the value, then the first of that group's three bins); the
// straddling lane takes masked maxima and a masked scan of its part.  The
// remaining widths (windows past the end of the series or the tile) and
// slices that touch three segments take the general exact steps.
constexpr int kGroups = kR / 3;

// Maximum of the lane's 33 sums; g receives the eleven 3-bin group maxima and
// t the maxima of groups 0-2, 3-5 and 6-8.
__device__ __forceinline__ float lane_max33(const float (&s)[kR], float (&g)[kGroups], float (&t)[3]) {
#pragma unroll
  for (int j = 0; j < kGroups; ++j) g[j] = max3f(s[3 * j], s[3 * j + 1], s[3 * j + 2]);
#pragma unroll
  for (int r = 0; r < 3; ++r) t[r] = max3f(g[3 * r], g[3 * r + 1], g[3 * r + 2]);
  return max3f(max3f(t[0], t[1], t[2]), g[9], g[10]);
}

// First of three values equal to v (the third if neither of the first two).
__device__ __forceinline__ int first_of3(float a, float b, float v) { return a == v ? 0 : (b == v ? 1 : 2); }

// Lowest i with s_i == v, for v the lane's own maximum: the first of the
// triple maxima t (then groups 9, 10) holding v, its first group, then that
// group's first bin.  Each level reads static registers picked by a switch,
// so the one lane that searches executes a few instructions per level.
__device__ __forceinline__ int first_bin33(const float (&s)[kR], const float (&g)[kGroups], const float (&t)[3],
                                           float v) {
  int q;
  if (t[0] == v) q = first_of3(g[0], g[1], v);
  else if (t[1] == v) q = 3 + first_of3(g[3], g[4], v);
  else if (t[2] == v) q = 6 + first_of3(g[6], g[7], v);
  else q = g[9] == v ? 9 : 10;
  switch (q) {
#define PS_BIN_CASE(k) \
  case k: return 3 * (k) + first_of3(s[3 * (k)], s[3 * (k) + 1], v);
    PS_BIN_CASE(0) PS_BIN_CASE(1) PS_BIN_CASE(2) PS_BIN_CASE(3) PS_BIN_CASE(4) PS_BIN_CASE(5)
    PS_BIN_CASE(6) PS_BIN_CASE(7) PS_BIN_CASE(8) PS_BIN_CASE(9)
#undef PS_BIN_CASE
    default: return 30 + first_of3(s[30], s[31], v);
  }
}

// Maximum of s[A..B), B > A, as a tree of 3-input maxima.
template <int A, int B>
__device__ __forceinline__ float range_max(const float (&s)[kR]) {
  if constexpr (B - A == 1) {
    return s[A];
  } else if constexpr (B - A == 2) {
    return fmaxf(s[A], s[A + 1]);
  } else if constexpr (B - A == 3) {
    return max3f(s[A], s[A + 1], s[A + 2]);
  } else {
    constexpr int T = (B - A) / 3;
    return max3f(range_max<A, A + T>(s), range_max<A + T, A + 2 * T>(s), range_max<A + 2 * T, B>(s));
  }
}

// Maxima of the lane's bins [0, ib) and [ib, 33), 0 < ib < 33 (the lane that
// straddles a segment boundary), through a switch on ib.
__device__ __forceinline__ void split_max(const float (&s)[kR], int ib, float &a, float &b) {
  switch (ib) {
#define PS_SPLIT_CASE(k)        \
  case k:                       \
    a = range_max<0, k>(s);     \
    b = range_max<k, kR>(s);    \
    break;
    PS_SPLIT_CASE(1) PS_SPLIT_CASE(2) PS_SPLIT_CASE(3) PS_SPLIT_CASE(4) PS_SPLIT_CASE(5) PS_SPLIT_CASE(6)
    PS_SPLIT_CASE(7) PS_SPLIT_CASE(8) PS_SPLIT_CASE(9) PS_SPLIT_CASE(10) PS_SPLIT_CASE(11) PS_SPLIT_CASE(12)
    PS_SPLIT_CASE(13) PS_SPLIT_CASE(14) PS_SPLIT_CASE(15) PS_SPLIT_CASE(16) PS_SPLIT_CASE(17) PS_SPLIT_CASE(18)
    PS_SPLIT_CASE(19) PS_SPLIT_CASE(20) PS_SPLIT_CASE(21) PS_SPLIT_CASE(22) PS_SPLIT_CASE(23) PS_SPLIT_CASE(24)
    PS_SPLIT_CASE(25) PS_SPLIT_CASE(26) PS_SPLIT_CASE(27) PS_SPLIT_CASE(28) PS_SPLIT_CASE(29) PS_SPLIT_CASE(30)
    PS_SPLIT_CASE(31)
#undef PS_SPLIT_CASE
    default:
      a = range_max<0, 32>(s);
      b = s[32];
  }
}

// Merge the warp maximum of v into slot (X, col); in search mode only a
// maximum >= T is merged (and its slot marked dirty).  v < 0: the lane holds
// no bin of segment X.  The lane's candidate bins are [ia, ie).
template <bool kSearch>
__device__ __forceinline__ void lean_emit(const float (&s)[kR], const float (&g)[kGroups], const float (&t)[3],
                                          float v, int ia, int ie, const LaneCtx &c, int64_t X, int col, int lane,
                                          float T) {
  const bool ok = v >= 0.0f;
  const uint32_t bits = ok ? __float_as_uint(v) : 0u;
  const uint32_t wb = __reduce_max_sync(kFull, bits);
  const float vm = __uint_as_float(wb);
  if (kSearch && !(vm >= T)) return;
  const unsigned hit = __ballot_sync(kFull, ok && bits == wb);
  if (hit != 0u && lane == __ffs(static_cast<int>(hit)) - 1) {
    const int i = (ia == 0 && ie == kR) ? first_bin33(s, g, t, vm) : first_equal(s, vm, ia, ie);
    emit_slot<kSearch>(c.slots, c.dirty, static_cast<uint64_t>(X) * c.W + col,
                       slot_key(vm, static_cast<uint32_t>(c.k0 + i)));
  }
}

// Steps w = wa..wb (every window valid) of a slice in segment X0 alone.
__device__ __forceinline__ void dump_steps_one(float (&s)[kR], const float *__restrict__ lane_buf, const LaneCtx &c,
                                               int64_t X0, int wa, int wb, int lane) {
  for (int w = wa; w <= wb; ++w) {
    const float *pw = lane_buf + (w - 1);
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] += pw[i];
    float g[kGroups], t[3];
    const float M = lane_max33(s, g, t);
    lean_emit<false>(s, g, t, M, 0, kR, c, X0, w - 1, lane, 0.0f);
  }
}

// Steps w = wa..wb (every window valid) of a slice that reaches segment
// X0 + 1; lane bl (or none, bl < 0) straddles the boundary at its bin c.ib.
__device__ __forceinline__ void dump_steps_two(float (&s)[kR], const float *__restrict__ lane_buf, const LaneCtx &c,
                                               int64_t X0, int bl, int wa, int wb, int lane) {
  for (int w = wa; w <= wb; ++w) {
    const float *pw = lane_buf + (w - 1);
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] += pw[i];
    float g[kGroups], t[3];
    const float M = lane_max33(s, g, t);
    const bool inA = c.seg_a == X0;
    float vA = inA ? M : -1.0f, vB = inA ? -1.0f : M;
    int ea = kR, ib = 0;
    if (lane == bl) {
      // the straddling lane's two parts
      split_max(s, c.ib, vA, vB);
      ea = c.ib;
      ib = c.ib;
    }
    lean_emit<false>(s, g, t, vA, 0, ea, c, X0, w - 1, lane, 0.0f);
    lean_emit<false>(s, g, t, vB, ib, kR, c, X0 + 1, w - 1, lane, 0.0f);
  }
}

// Every (segment, width) maximum of slice vw of the tile.
__device__ __forceinline__ void dump_slice(const float *__restrict__ buf, const SeriesDev &S, int64_t t0,
                                           int tile_bins, int vw, int lane, int W, int seg_len,
                                           unsigned long long *__restrict__ slots) {
  const LaneCtx c = lane_ctx(S, t0, tile_bins, vw, lane, W, seg_len, slots, nullptr);
  const float *lane_buf = buf + vw * (32 * kR) + lane * kR;
  float s[kR];
#pragma unroll
  for (int i = 0; i < kR; ++i) s[i] = 0.0f;
  const int64_t X0 = __shfl_sync(kFull, c.seg_a, 0);
  // each lane in X0 (possibly straddling into X0 + 1) or wholly in X0 + 1
  const bool two = seg_len >= 2 * kR && __all_sync(kFull, c.seg_a == X0 || (c.seg_a == X0 + 1 && c.ib == kR));
  // the lane's windows are all valid up to width m - (k0 + 32) when its 33
  // bins belong to the tile
  const int64_t wl = c.lim_tile >= kR ? max64(0, min64(static_cast<int64_t>(W), c.m - c.k0 - (kR - 1))) : 0;
  const int w_fast = two ? static_cast<int>(__reduce_min_sync(kFull, static_cast<unsigned>(wl))) : 0;
  if (w_fast > 0) {
    const bool split = __any_sync(kFull, c.seg_a != X0 || c.ib < kR);
    const int bl = __ffs(static_cast<int>(__ballot_sync(kFull, c.ib < kR))) - 1;
    if (split) dump_steps_two(s, lane_buf, c, X0, bl, 1, w_fast, lane);
    else dump_steps_one(s, lane_buf, c, X0, 1, w_fast, lane);
  }
  if (w_fast < W) exact_steps<false>(s, lane_buf, w_fast + 1, 0, W - w_fast, nullptr, c);
}

template <bool kSearch, bool kPacked>
__device__ __forceinline__ bool boxcar_tile(
    int64_t tile, unsigned char *smem_raw, const float *__restrict__ power, const SeriesDev *__restrict__ series,
    const int64_t *__restrict__ tile_off, int n_series, int W, int seg_len, const float *__restrict__ thr_all,
    const float *__restrict__ thrb_all, unsigned long long *__restrict__ slots, uint32_t *__restrict__ dirty,
    uint32_t *__restrict__ counters, unsigned long long *__restrict__ items, float *__restrict__ snaps,
    uint32_t item_cap, int tile_bins, int buf_len, int groups, uint32_t wait_test, const float2 *__restrict__ spec,
    const float4 *__restrict__ norm) {
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  float *buf = reinterpret_cast<float *>(smem_raw + 128);
  const int nq33 = buf_len / kR;        // 33-bin block sums
  const int nq11 = buf_len / kSub;      // 11-bin block sums
  float *q33 = buf + buf_len;
  float *q11 = q33 + nq33 + 1;
  const int nthreads = blockDim.x;

  const int si = series_of_tile(tile_off, n_series, tile);
  const SeriesDev S = series[si];
  const int64_t t0 = (tile - S.tile_off) * static_cast<int64_t>(tile_bins);
  const float *src = power + S.p_off + t0;
  const int64_t avail64 = S.m - t0;
  const int avail = static_cast<int>(min64(avail64, static_cast<int64_t>(buf_len)));
  // a 16-byte multiple from a 16-byte aligned source; the rest by plain loads
  const int n_tma = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0u && avail > 0) ? (avail & ~3) : 0;

  if (norm != nullptr) {
    // fused: P formed from the spectrum while it is staged
    stage_fused(buf, buf_len, avail, S, t0, seg_len, spec, norm);
    __syncthreads();
  } else {
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  // wait_test != 0 (a test of the timeout path): no copy is issued, so the
  // barrier never completes and the bounded wait below gives up after
  // wait_test microseconds with nothing in flight
  if (threadIdx.x == 0 && n_tma > 0 && wait_test == 0u) {
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(n_tma) * 4u);
    tma_load_1d(buf, src, static_cast<uint32_t>(n_tma) * 4u, bar);
  }
  for (int i = n_tma + threadIdx.x; i < buf_len; i += nthreads) buf[i] = (i < avail) ? src[i] : 0.0f;
  // one thread waits on the copy (bounded); the others sleep in the barrier
  const uint64_t limit_ns = wait_test ? 1000ull * wait_test : 2000000000ull;
  if (threadIdx.x == 0)
    q33[0] = ((n_tma == 0 && wait_test == 0u) || mbar_wait_bounded(bar, 0, limit_ns)) ? 1.0f : 0.0f;
  __syncthreads();
  if (q33[0] == 0.0f) {
    if (threadIdx.x == 0) atomicOr(counters + 2, kErrTimeout);
    return false;   // nothing else is in flight: the only copy is this one
  }
  __syncthreads();
  }

  // block sums for the bounds: q11[j] = sum of 11 bins from 11 j,
  // q33[j] = sum of 33 bins from 33 j
  for (int j = threadIdx.x; j < nq11; j += nthreads) {
    const float *p = buf + kSub * j;
    float a = 0.0f;
#pragma unroll
    for (int x = 0; x < kSub; ++x) a += p[x];
    q11[j] = a;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nq33; j += nthreads) q33[j] = q11[3 * j] + q11[3 * j + 1] + q11[3 * j + 2];
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float *thr = thr_all + static_cast<int64_t>(si) * W;
  const float *thrb = thrb_all + static_cast<int64_t>(si) * W;

  if (!kSearch) {
    // every (segment, width) maximum: each of the warp's slices in turn
    for (int g = 0; g < groups; ++g) dump_slice(buf, S, t0, tile_bins, warp * groups + g, lane, W, seg_len, slots);
    return true;
  }
  if (kPacked) {
    packed_bank(buf, q11, q33, S, si, tile, t0, tile_bins, W, seg_len, thr, thrb, slots, dirty, counters, items,
                snaps, item_cap, series);
    return true;
  }

  const int x0 = warp * (32 * kR) + lane * kR;   // buffer-relative first bin
  const LaneCtx c = lane_ctx(S, t0, tile_bins, warp, lane, W, seg_len, slots, dirty);
  float s[kR], b[kR];
#pragma unroll
  for (int i = 0; i < kR; ++i) s[i] = 0.0f;
  const float *lane_buf = buf + x0;

#pragma unroll
  for (int j = 0; j < kR - 1; ++j) b[j] = lane_buf[j];
  b[kR - 1] = 0.0f;

  // One 33-step body serves every block.  A block first tests its bound
  // (per 11 x 11 sub-block for the early widths, per 33 x 33 block after);
  // early blocks test again before steps 11 and 22.  When a bound reaches the
  // threshold the rest of the block is deferred (snapshot + work item for the
  // deferred kernel) and the warp carries on with plain adds; only when the
  // work list is full does the warp inspect the block itself (exact mode).
  const int nb = (W + kR - 1) / kR;
  const int qb0 = x0 / kSub;
  const int qc0 = x0 / kR;
  for (int bi = 0; bi < nb; ++bi) {
    const float *pb = lane_buf + bi * kR;
    const int wf = bi * kR + 1;
    const int nsteps = min(kR, W - bi * kR);
    const bool early = bi < kEarlyBlocks;
    bool deferred = false;
    {
      const bool hit = early ? early_bound(s, q11, qb0 + 3 * bi, thrb[wf - 1])
                             : (s[0] + q33[qc0 + bi] + q33[qc0 + bi + 1] >= thrb[wf - 1]);
      if (__any_sync(kFull, hit)) {
        if (!defer_block(s, items, snaps, counters, item_cap, tile, warp, bi, 0)) {
          exact_steps<true>(s, lane_buf, wf, 0, nsteps, thr, c);
          reload_ring<kR>(b, pb);
          continue;
        }
        deferred = true;
      }
    }
    if (nsteps < kSub) {
      tail_steps(s, lane_buf, wf, wf + nsteps);
      continue;
    }
    fast_steps<0, kSub>(s, b, pb);
    if (early && !deferred && nsteps > kSub &&
        __any_sync(kFull, early_bound(s, q11, qb0 + 3 * bi + 1, thrb[wf + kSub - 1]))) {
      if (!defer_block(s, items, snaps, counters, item_cap, tile, warp, bi, kSub)) {
        exact_steps<true>(s, lane_buf, wf, kSub, nsteps, thr, c);
        reload_ring<kR>(b, pb);
        continue;
      }
      deferred = true;
    }
    if (nsteps < 2 * kSub) {
      tail_steps(s, lane_buf, wf + kSub, wf + nsteps);
      continue;
    }
    fast_steps<kSub, kSub>(s, b, pb);
    if (early && !deferred && nsteps > 2 * kSub &&
        __any_sync(kFull, early_bound(s, q11, qb0 + 3 * bi + 2, thrb[wf + 2 * kSub - 1]))) {
      if (!defer_block(s, items, snaps, counters, item_cap, tile, warp, bi, 2 * kSub)) {
        exact_steps<true>(s, lane_buf, wf, 2 * kSub, nsteps, thr, c);
        reload_ring<kR>(b, pb);
        continue;
      }
    }
    if (nsteps < kR) {
      tail_steps(s, lane_buf, wf + 2 * kSub, wf + nsteps);
      continue;
    }
    fast_steps<2 * kSub, kSub>(s, b, pb);
  }
  return true;
}

__device__ __forceinline__ uint32_t sm_id() {
  uint32_t id;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
  return id;
}

// The bank over all tiles.  With tile_ctr == nullptr every CTA takes tile
// tile_base + blockIdx.x.  Otherwise the launch is persistent (a few CTAs per SM): the
// tiles are split into n_ranges contiguous ranges [range_lo[r],
// range_lo[r + 1]), one per SM, each with a claim counter in tile_ctr
// (zeroed before the launch).  A CTA claims tiles from the range of the SM
// it runs on (%smid modulo n_ranges), one atomic per tile, issued before the
// current tile runs so its latency is hidden; when that range is drained,
// warp 0 reads all counters at once and claims from any range with tiles
// left.  So every SM gets the same share of the work however the hardware
// places the CTAs, and no tile is left while any CTA runs.  (A
// one-CTA-per-tile grid refills the SMs that free their slots first, which
// leaves a partial last wave on some SMs only.)
// kPacked (search mode only): two virtual warps per warp with packed adds,
// at most 170 registers per thread (three 4-warp CTAs per SM).  Dump mode
// targets kDumpMinBlocks resident 4-warp CTAs per SM.
constexpr int kDumpMinBlocks = 4;

template <bool kSearch, bool kPacked>
__global__ void __launch_bounds__(kMaxThreads, kSearch ? (kPacked ? 3 : kMinBlocks) : kDumpMinBlocks) boxcar_kernel(
    const float *__restrict__ power, const SeriesDev *__restrict__ series, const int64_t *__restrict__ tile_off,
    int n_series, int W, int seg_len, const float *__restrict__ thr_all, const float *__restrict__ thrb_all,
    unsigned long long *__restrict__ slots, uint32_t *__restrict__ dirty, uint32_t *__restrict__ counters,
    unsigned long long *__restrict__ items, float *__restrict__ snaps, uint32_t item_cap, int tile_bins,
    int buf_len, uint32_t *__restrict__ tile_ctr, const int64_t *__restrict__ range_lo, int n_ranges, int groups,
    uint32_t wait_test, int64_t tile_base, const float2 *__restrict__ spec, const float4 *__restrict__ norm) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (tile_ctr == nullptr) {
    boxcar_tile<kSearch, kPacked>(tile_base + blockIdx.x, smem_raw, power, series, tile_off, n_series, W, seg_len, thr_all,
                                  thrb_all, slots, dirty, counters, items, snaps, item_cap, tile_bins, buf_len, groups,
                                  wait_test, spec, norm);
    return;
  }
  int64_t *claim = reinterpret_cast<int64_t *>(smem_raw + 64);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int home = static_cast<int>(sm_id() % static_cast<uint32_t>(n_ranges));
  const int64_t home_lo = range_lo[home], home_hi = range_lo[home + 1];
  bool home_open = true;   // thread 0
  auto claim_home = [&]() -> int64_t {
    if (!home_open) return -1;
    const int64_t t = home_lo + atomicAdd(tile_ctr + home, 1u);
    if (t < home_hi) return t;
    home_open = false;
    return -1;
  };
  int64_t mine = (threadIdx.x == 0) ? claim_home() : -1;
  for (;;) {
    if (warp == 0) {
      int64_t t = __shfl_sync(kFull, mine, 0);
      // home drained: claim from any range with tiles left (every range is
      // visited once per pass; claims only grow, so the pass ends)
      for (int base = 0; t < 0 && base < n_ranges; base += 32) {
        const int r = base + lane;
        bool left = false;
        if (r < n_ranges) left = static_cast<int64_t>(__ldcg(tile_ctr + r)) < range_lo[r + 1] - range_lo[r];
        uint32_t m = __ballot_sync(kFull, left);
        while (m != 0u && t < 0) {
          const int rr = base + __ffs(static_cast<int>(m)) - 1;
          m &= m - 1u;
          int64_t c = -1;
          if (lane == 0) {
            const int64_t v = range_lo[rr] + atomicAdd(tile_ctr + rr, 1u);
            c = (v < range_lo[rr + 1]) ? v : -1;
          }
          t = __shfl_sync(kFull, c, 0);
        }
      }
      if (lane == 0) *claim = t;
    }
    __syncthreads();
    const int64_t tile = *claim;
    __syncthreads();
    if (tile < 0) return;
    if (threadIdx.x == 0) mine = claim_home();
    if (!boxcar_tile<kSearch, kPacked>(tile, smem_raw, power, series, tile_off, n_series, W, seg_len, thr_all,
                                       thrb_all, slots, dirty, counters, items, snaps, item_cap, tile_bins, buf_len,
                                       groups, wait_test, spec, norm))
      return;
    __syncthreads();   // the tile's shared memory is free for the next one
  }
}

// Deferred blocks, one CTA of three warps per work item.  The item is the
// block of 32 x 33 = 1056 consecutive start bins x 33 widths that one warp of
// the search kernel left, with the 1056 running sums saved in a snapshot.
// Thread t carries the sums of bins 11t .. 11t + 10 of the block through its
// remaining widths -- the same adds in the same order as the search kernel,
// so the sums are bit-identical -- and after each step stores the best of its
// eleven sums (a max tree) and the first of its bins holding it; the window
// values come from an 11-register ring (one shared-memory load per step), and
// the step loop has no cross-thread work.  A thread whose bins straddle a
// segment boundary keeps the two parts apart (a second best/bin pair); its
// warp runs that variant, so no thread diverges.  Every 11 steps the chunk's
// widths are merged into one 64-bit maximum per (segment, width): when the
// block touches at most two segments (segment_len >= 1056, the usual case),
// 8 threads per width each scan 12 threads' entries in bin order and a
// 3-round shuffle combines them; otherwise lane l of a warp scans the three
// threads that cover bins 33 l .. 33 l + 32 and keeps, per segment there (at
// most two), the largest sum reaching T_w and its lowest bin, the second part
// moves to lane l + 1 (whose segment it is), and the warp reduces each
// segment it holds with two 32-bit reductions (power bits, then bin).  Each
// key has one writer, so no atomics.  A last pass sends every maximum to its
// slot.
// The P window (1056 bins plus the 66-bin reach of one block) and the
// snapshot are staged in shared memory.  Blocks at the very end of a series
// (windows that leave the spectrum) take a plain per-step loop.
constexpr int kDeferThreads = 96;
constexpr int kDeferBins = 32 * kR / kDeferThreads;        // bins per thread (11)
constexpr int kDeferWarps = kDeferThreads / 32;
constexpr int kDeferChunk = 11;                             // steps per merge
constexpr int kRegion = 32 * kR + 2 * kR;
constexpr int kItemSegs = 32 * kR / (2 * kR) + 2;           // segments one item can touch (segment_len >= 66)
static_assert(kDeferBins == 11 && kDeferChunk == 11, "the unrolled ring assumes 11 bins and 11 steps");
static_assert(kDeferBins * kDeferThreads == 32 * kR, "the threads' bins cover the block");
static_assert(kR % kDeferBins == 0 && kR / kDeferBins * 32 == kDeferThreads, "a lane's 33 bins are whole threads");
constexpr int kThreadsPerLane = kR / kDeferBins;            // 3
constexpr int kRegionLoads = (kRegion + kDeferThreads - 1) / kDeferThreads;
constexpr int kSnapLoads = 32 * kR / kDeferThreads;
static_assert(kSnapLoads * kDeferThreads == 32 * kR, "whole snapshot loads");

__device__ __forceinline__ unsigned long long best_key(float v, uint32_t bin) {
  return (static_cast<unsigned long long>(__float_as_uint(v)) << 32) |
         static_cast<unsigned long long>(0xffffffffu - bin);
}

__device__ __forceinline__ float max11(const float (&v)[kDeferBins]) {
  return max3f(max3f(max3f(v[0], v[1], v[2]), max3f(v[3], v[4], v[5]), max3f(v[6], v[7], v[8])), v[9], v[10]);
}

// First j with v[j] == m (11 if none).
__device__ __forceinline__ int first_of(const float (&v)[kDeferBins], float m) {
  uint32_t eq = 0u;
#pragma unroll
  for (int j = 0; j < kDeferBins; ++j) eq |= (v[j] == m) ? (1u << j) : 0u;
  return __ffs(static_cast<int>(eq | (1u << kDeferBins))) - 1;
}

struct DeferShared {
  float region[kRegion];
  float snap[kR * (32 + 1)];                    // [bin i][lane l], rows of 33
  float cval[kDeferChunk][kDeferThreads + 1];   // per step of the chunk: best sum of each thread (part A);
  float cvalB[kDeferChunk][kDeferThreads + 1];  // part B (bins past a segment boundary), -1 if none; rows
                                                // padded so the 8-thread merge reads are conflict-free
  uint8_t cidx[kDeferChunk][kDeferThreads + 1];   // first bin within the thread holding it
  uint8_t cidxB[kDeferChunk][kDeferThreads + 1];
  unsigned long long keys[kItemSegs][kR];
  float tcache[kR];                             // T_w of the block's widths
};

// One chunk of 11 steps from the register ring rg (positions p of the chunk's
// window rb[] in rg[p % 11]; on exit positions 11..21, i.e. the next chunk's
// 0..10).  kSplit: bins from jc on form part B.
template <bool kSplit>
__device__ __forceinline__ void defer_chunk(float (&s)[kDeferBins], float (&rg)[kDeferBins],
                                            const float *__restrict__ rb, int jc, DeferShared &sh, int t) {
#pragma unroll
  for (int u = 0; u < kDeferChunk; ++u) {
#pragma unroll
    for (int j = 0; j < kDeferBins; ++j) s[j] += rg[(u + j) % kDeferBins];
    rg[u] = rb[u + kDeferBins];   // position u + 11 takes the slot of position u
    if (!kSplit) {
      const float best = max11(s);
      sh.cval[u][t] = best;
      sh.cidx[u][t] = static_cast<uint8_t>(first_of(s, best));
    } else {
      float va[kDeferBins], vb[kDeferBins];
#pragma unroll
      for (int j = 0; j < kDeferBins; ++j) {
        va[j] = (j < jc) ? s[j] : -1.0f;
        vb[j] = (j < jc) ? -1.0f : s[j];
      }
      const float ba = max11(va), bb = max11(vb);
      sh.cval[u][t] = ba;
      sh.cidx[u][t] = static_cast<uint8_t>(first_of(va, ba));
      sh.cvalB[u][t] = bb;
      sh.cidxB[u][t] = static_cast<uint8_t>(first_of(vb, bb));
    }
  }
}

__global__ void __launch_bounds__(kDeferThreads, 8) deferred_kernel(
    const float *__restrict__ power, const SeriesDev *__restrict__ series, const int64_t *__restrict__ tile_off,
    int n_series, int W, int seg_len, const float *__restrict__ thr_all, unsigned long long *__restrict__ slots,
    uint32_t *__restrict__ dirty, const uint32_t *__restrict__ counters,
    const unsigned long long *__restrict__ items, const float *__restrict__ snaps, uint32_t item_cap,
    int tile_bins, const float2 *__restrict__ spec,
    const float4 *__restrict__ norm) {
  __shared__ DeferShared sh;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t n_items = min(counters[0], item_cap);
  for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const unsigned long long item = items[it];
    const int64_t tile = static_cast<int64_t>(item & 0xffffffffffull);
    const int wv = static_cast<int>((item >> 40) & 7ull);
    const int bi = static_cast<int>((item >> 43) & 0x1fffull);
    const int cx = static_cast<int>((item >> 56) & 0xffull);
    const int si = series_of_tile(tile_off, n_series, tile);
    const SeriesDev S = series[si];
    const int64_t t0 = (tile - S.tile_off) * static_cast<int64_t>(tile_bins);
    const int64_t k0 = t0 + wv * (32 * kR);             // first start bin of the block
    const int64_t r0 = k0 + bi * kR + cx;               // first bin of the staged window
    const float *src = power + S.p_off;
    const int nsteps = min(kR, W - bi * kR);
    const int wf = bi * kR + 1;
    const int64_t seg_hi = S.n_seg - 1;
    const int64_t g0 = min64(k0 / seg_len, seg_hi);     // series-relative segment of the first bin
    const int n_segs = static_cast<int>(min64((k0 + 32 * kR - 1) / seg_len, seg_hi) - g0 + 1);
    // all global loads of the item are issued before any is used (registers),
    // so staging costs one memory latency, not one per loop trip
    const float *sp = snaps + static_cast<size_t>(it) * (kR * 32);
    float ld_r[kRegionLoads], ld_s[kSnapLoads];
    if (norm == nullptr) {
#pragma unroll
      for (int q = 0; q < kRegionLoads; ++q) {
        const int j = t + q * kDeferThreads;
        ld_r[q] = (j < kRegion && r0 + j < S.m) ? __ldg(src + r0 + j) : 0.0f;
      }
    } else {
#pragma unroll
      for (int q = 0; q < kRegionLoads; ++q) {
        const int j = t + q * kDeferThreads;
        ld_r[q] = (j < kRegion && r0 + j < S.m) ? fused_power(spec, norm, S, r0 + j, seg_len) : 0.0f;
      }
    }
#pragma unroll
    for (int q = 0; q < kSnapLoads; ++q) ld_s[q] = sp[t + q * kDeferThreads];
    const float thr_t = (t < nsteps) ? __ldg(thr_all + static_cast<int64_t>(si) * W + wf - 1 + t) : 0.0f;
    __syncthreads();   // the previous item is finished with the shared arrays
#pragma unroll
    for (int q = 0; q < kRegionLoads; ++q) {
      const int j = t + q * kDeferThreads;
      if (j < kRegion) sh.region[j] = ld_r[q];
    }
#pragma unroll
    for (int q = 0; q < kSnapLoads; ++q) {
      const int j = t + q * kDeferThreads;
      sh.snap[(j >> 5) * 33 + (j & 31)] = ld_s[q];
    }
    for (int j = t; j < n_segs * kR; j += kDeferThreads) (&sh.keys[0][0])[j] = 0ull;
#pragma unroll
    for (int u = 0; u < kDeferChunk; ++u) sh.cvalB[u][t] = -1.0f;
    if (t < nsteps) sh.tcache[t] = thr_t;
    __syncthreads();

    // this thread's bins b0 + j, b0 = 11 t (bin b of the block = lane b / 33's bin b % 33)
    const int b0 = kDeferBins * t;
    float s[kDeferBins];
#pragma unroll
    for (int j = 0; j < kDeferBins; ++j) s[j] = sh.snap[((b0 + j) % kR) * 33 + (b0 + j) / kR];
    const int sg0 = static_cast<int>(min64((k0 + b0) / seg_len, seg_hi) - g0);
    const int sg1 = static_cast<int>(min64((k0 + b0 + kDeferBins - 1) / seg_len, seg_hi) - g0);
    // straddling thread: bins from jc on lie in segment sg1
    const int jc = (sg1 != sg0) ? static_cast<int>((g0 + sg1) * seg_len - k0) - b0 : kDeferBins;
    const bool split_warp = __any_sync(kFull, jc != kDeferBins);
    // bin b has a whole window at width w iff b < base - w; all_valid: every
    // bin of the block at every remaining width
    const int64_t base = S.m + 1 - k0;
    const bool all_valid = base - (wf + nsteps - 1) >= 32 * kR;
    // merge lanes: lane l covers bins 33 l .. 33 l + 32, from segment segA on;
    // bins from cut on lie in segA + 1
    const int segA = static_cast<int>(min64((k0 + kR * lane) / seg_len, seg_hi) - g0);
    const int cut = (g0 + segA < seg_hi) ? static_cast<int>((g0 + segA + 1) * seg_len - k0) : (1 << 30);
    // with at most two segments: the block's first bin of the second one
    const int bcut = (n_segs == 2) ? static_cast<int>((g0 + 1) * seg_len - k0) : (1 << 30);

    float rg[kDeferBins];
    bool ring = false;
    for (int c0 = cx; c0 < nsteps; c0 += kDeferChunk) {
      const int c1 = min(c0 + kDeferChunk, nsteps);
      if (all_valid && c1 - c0 == kDeferChunk) {
        const float *rb = sh.region + (c0 - cx) + b0;
        if (!ring) {
#pragma unroll
          for (int j = 0; j < kDeferBins; ++j) rg[j] = rb[j];
          ring = true;
        }
        if (split_warp) defer_chunk<true>(s, rg, rb, jc, sh, t);
        else defer_chunk<false>(s, rg, rb, jc, sh, t);
      } else {
        // windows leaving the spectrum (or a short last block): plain steps
        for (int cc = c0; cc < c1; ++cc) {
          const float *pw = sh.region + (cc - cx) + b0;
          const int64_t lim = base - (wf + cc);
          float va[kDeferBins], vb[kDeferBins];
#pragma unroll
          for (int j = 0; j < kDeferBins; ++j) {
            s[j] += pw[j];
            const bool ok = b0 + j < lim;
            va[j] = (ok && j < jc) ? s[j] : -1.0f;
            vb[j] = (ok && j >= jc) ? s[j] : -1.0f;
          }
          const float ba = max11(va), bb = max11(vb);
          sh.cval[cc - c0][t] = ba;
          sh.cidx[cc - c0][t] = static_cast<uint8_t>(first_of(va, ba));
          sh.cvalB[cc - c0][t] = bb;
          sh.cidxB[cc - c0][t] = static_cast<uint8_t>(first_of(vb, bb));
        }
      }
      __syncthreads();
      if (n_segs <= 2) {
        // at most one segment boundary (bcut) in the block: 8 threads per
        // width of the chunk, each scanning 12 threads' entries in bin order,
        // then a 3-round shuffle over the 8; no atomics (one writer per key)
        const int mw = t >> 3, q = t & 7;
        const int u = mw;
        unsigned long long kk0 = 0ull, kk1 = 0ull;
        if (c0 + mw < c1) {
          const float T = sh.tcache[c0 + mw];
#pragma unroll
          for (int e = 0; e < kDeferThreads / 8; ++e) {
            const int tt = (kDeferThreads / 8) * q + e;
            const float v = sh.cval[u][tt];
            if (v >= T && v >= 0.0f) {
              const int bin = kDeferBins * tt + sh.cidx[u][tt];
              const unsigned long long key = best_key(v, static_cast<uint32_t>(k0 + bin));
              if (bin < bcut) kk0 = max(kk0, key);
              else kk1 = max(kk1, key);
            }
            const float v2 = sh.cvalB[u][tt];   // part B: past the boundary
            if (v2 >= T && v2 >= 0.0f)
              kk1 = max(kk1, best_key(v2, static_cast<uint32_t>(k0 + kDeferBins * tt + sh.cidxB[u][tt])));
          }
        }
#pragma unroll
        for (int d = 4; d >= 1; d >>= 1) {
          kk0 = max(kk0, __shfl_xor_sync(kFull, kk0, d));
          kk1 = max(kk1, __shfl_xor_sync(kFull, kk1, d));
        }
        if (q == 0 && c0 + mw < c1) {
          if (kk0 != 0ull) sh.keys[0][c0 + mw] = max(sh.keys[0][c0 + mw], kk0);
          if (kk1 != 0ull) sh.keys[1][c0 + mw] = max(sh.keys[1][c0 + mw], kk1);
        }
      } else for (int cc = c0 + warp; cc < c1; cc += kDeferWarps) {
        const int u = cc - c0;
        const float T = sh.tcache[cc];
        // the lane's best per segment part, scanning its bins in order (a
        // strict > keeps the lowest bin among equal sums)
        float vA = -1.0f, vB = -1.0f;
        int binA = 0, binB = 0;
#pragma unroll
        for (int q = 0; q < kThreadsPerLane; ++q) {
          const int tt = kThreadsPerLane * lane + q;
          const float v = sh.cval[u][tt];
          if (v >= T && v >= 0.0f) {
            const int bin = kDeferBins * tt + sh.cidx[u][tt];
            if (bin < cut) {
              if (v > vA) { vA = v; binA = bin; }
            } else if (v > vB) {
              vB = v;
              binB = bin;
            }
          }
          const float v2 = sh.cvalB[u][tt];
          if (v2 >= T && v2 >= 0.0f) {
            const int bin = kDeferBins * tt + sh.cidxB[u][tt];
            if (v2 > vB) { vB = v2; binB = bin; }
          }
        }
        // part B of lane l lies in segment segA + 1 = lane l + 1's segA (a
        // segment of >= 66 bins covers the rest of lane l and all of lane l + 1);
        // its bins come first there, so it wins ties
        const float vP = __shfl_up_sync(kFull, vB, 1);
        const int binP = __shfl_up_sync(kFull, binB, 1);
        if (lane > 0 && vP >= 0.0f && vP >= vA) { vA = vP; binA = binP; }
        if (lane == 31 && vB >= 0.0f) {
          unsigned long long &kk = sh.keys[segA + 1][cc];
          kk = max(kk, best_key(vB, static_cast<uint32_t>(k0 + binB)));
        }
        // each segment the warp holds: max power bits, then the lowest bin
        unsigned todo = __ballot_sync(kFull, vA >= 0.0f);
        while (todo != 0u) {
          const int sgs = __shfl_sync(kFull, segA, __ffs(static_cast<int>(todo)) - 1);
          const bool in = segA == sgs && vA >= 0.0f;
          const uint32_t bits = in ? __float_as_uint(vA) : 0u;
          const uint32_t mx = __reduce_max_sync(kFull, bits);
          const uint32_t bn = (in && bits == mx) ? static_cast<uint32_t>(k0 + binA) : 0xffffffffu;
          const uint32_t bmin = __reduce_min_sync(kFull, bn);
          if (lane == 0) {
            unsigned long long &kk = sh.keys[sgs][cc];
            kk = max(kk, best_key(__uint_as_float(mx), bmin));
          }
          todo &= ~__ballot_sync(kFull, segA == sgs);
        }
      }
      __syncthreads();   // the next chunk overwrites the chunk arrays
    }
    for (int j = t; j < n_segs * kR; j += kDeferThreads) {
      const unsigned long long key = (&sh.keys[0][0])[j];
      if (key != 0ull)
        emit_slot<true>(slots, dirty, static_cast<uint64_t>(S.seg_off + g0 + j / kR) * W + (wf + j % kR - 1), key);
    }
  }
}

// Deferred blocks, one warp per item (segment_len >= 66).  The warp takes
// its lanes' 33 running sums straight from the snapshot ([bin][lane]:
// coalesced), stages the item's window (1056 bins plus the 66-bin reach of
// one block) in its own shared-memory region and runs the block's remaining
// steps in the bank's lane layout.  Where every window of the item lies in
// the series and each lane lies in one of two segments, a step costs the
// adds, the lane maximum from its group maxima and one warp max-reduction
// compared with T_w; only a maximum that passes takes the per-segment merge
// (the leader's bin search and the slot reduction of the dump mode's lean
// merge).  Other items take the general exact steps.
constexpr int kDwWarps = 4;                               // items per CTA at a time
constexpr int kDwLoads = (kRegion + 31) / 32;             // window loads per lane

template <bool kTwo>
__device__ __forceinline__ void defer_lean_steps(float (&s)[kR], const float *__restrict__ lane_win,
                                                 const LaneCtx &c, int64_t X0, int bl, int wf, int c0, int c1,
                                                 const float *__restrict__ thr, int lane) {
  for (int cc = c0; cc < c1; ++cc) {
    const float *pw = lane_win + (cc - c0);
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] += pw[i];
    const int w = wf + cc;
    const float T = __ldg(thr + (w - 1));
    float g[kGroups], t[3];
    const float M = lane_max33(s, g, t);
    if (!kTwo) {
      lean_emit<true>(s, g, t, M, 0, kR, c, X0, w - 1, lane, T);
      continue;
    }
    // nothing reaches T anywhere in the slice: no part can pass
    const uint32_t any = __reduce_max_sync(kFull, M >= 0.0f ? __float_as_uint(M) : 0u);
    if (!(__uint_as_float(any) >= T)) continue;
    const bool inA = c.seg_a == X0;
    float vA = inA ? M : -1.0f, vB = inA ? -1.0f : M;
    int ea = kR, ib = 0;
    if (lane == bl) {
      split_max(s, c.ib, vA, vB);
      ea = c.ib;
      ib = c.ib;
    }
    lean_emit<true>(s, g, t, vA, 0, ea, c, X0, w - 1, lane, T);
    lean_emit<true>(s, g, t, vB, ib, kR, c, X0 + 1, w - 1, lane, T);
  }
}

__global__ void __launch_bounds__(32 * kDwWarps) deferred_warp_kernel(
    const float *__restrict__ power, const SeriesDev *__restrict__ series, const int64_t *__restrict__ tile_off,
    int n_series, int W, int seg_len, const float *__restrict__ thr_all, unsigned long long *__restrict__ slots,
    uint32_t *__restrict__ dirty, const uint32_t *__restrict__ counters,
    const unsigned long long *__restrict__ items, const float *__restrict__ snaps, uint32_t item_cap,
    int tile_bins, const float2 *__restrict__ spec, const float4 *__restrict__ norm) {
  __shared__ float region_all[kDwWarps][kRegion];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *region = region_all[warp];
  const uint32_t n_items = min(counters[0], item_cap);
  for (uint32_t it = blockIdx.x * kDwWarps + warp; it < n_items; it += gridDim.x * kDwWarps) {
    const unsigned long long item = items[it];
    const int64_t tile = static_cast<int64_t>(item & 0xffffffffffull);
    const int wv = static_cast<int>((item >> 40) & 7ull);
    const int bi = static_cast<int>((item >> 43) & 0x1fffull);
    const int cx = static_cast<int>((item >> 56) & 0xffull);
    const int si = series_of_tile(tile_off, n_series, tile);
    const SeriesDev S = series[si];
    const int64_t t0 = (tile - S.tile_off) * static_cast<int64_t>(tile_bins);
    const int64_t k0s = t0 + wv * (32 * kR);            // first start bin of the slice
    const int64_t r0 = k0s + bi * kR + cx;              // first bin of the staged window
    const int nsteps = min(kR, W - bi * kR);
    const int wf = bi * kR + 1;
    // every load of the item issued before any is used
    const float *sp = snaps + static_cast<size_t>(it) * (kR * 32) + lane;
    float s[kR], ld[kDwLoads];
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] = sp[i * 32];
    const float *src = power + S.p_off;
    if (norm == nullptr) {
#pragma unroll
      for (int q = 0; q < kDwLoads; ++q) {
        const int j = lane + 32 * q;
        ld[q] = (j < kRegion && r0 + j < S.m) ? __ldg(src + r0 + j) : 0.0f;
      }
    } else {
#pragma unroll
      for (int q = 0; q < kDwLoads; ++q) {
        const int j = lane + 32 * q;
        ld[q] = (j < kRegion && r0 + j < S.m) ? fused_power(spec, norm, S, r0 + j, seg_len) : 0.0f;
      }
    }
    __syncwarp();   // the previous item's reads of the region are done
#pragma unroll
    for (int q = 0; q < kDwLoads; ++q) {
      const int j = lane + 32 * q;
      if (j < kRegion) region[j] = ld[q];
    }
    __syncwarp();
    const LaneCtx c = lane_ctx(S, t0, tile_bins, wv, lane, W, seg_len, slots, dirty);
    const float *thr = thr_all + static_cast<int64_t>(si) * W;
    const float *lane_win = region + lane * kR;       // bin i at step cc: lane_win[cc - cx + i]
    const int64_t X0 = __shfl_sync(kFull, c.seg_a, 0);
    const bool two = __all_sync(kFull, c.seg_a == X0 || (c.seg_a == X0 + 1 && c.ib == kR));
    // every bin of the slice has its whole window at the block's last width
    const bool all_valid = S.m + 1 - k0s - (wf + nsteps - 1) >= 32 * kR;
    if (two && all_valid) {
      const bool split = __any_sync(kFull, c.seg_a != X0 || c.ib < kR);
      const int bl = __ffs(static_cast<int>(__ballot_sync(kFull, c.ib < kR))) - 1;
      if (split) defer_lean_steps<true>(s, lane_win, c, X0, bl, wf, cx, nsteps, thr, lane);
      else defer_lean_steps<false>(s, lane_win, c, X0, bl, wf, cx, nsteps, thr, lane);
    } else {
      exact_steps<true>(s, lane_win, wf, cx, nsteps, thr, c, bi * kR + cx);
    }
  }
}

// Deferred blocks when segments are shorter than 66 bins (a lane's 33 bins
// may then reach a third segment, and every bin is merged on its own; only
// tiny test shapes): one warp per item with all 33 sums.
__global__ void __launch_bounds__(128) deferred_small_kernel(
    const float *__restrict__ power, const SeriesDev *__restrict__ series, const int64_t *__restrict__ tile_off,
    int n_series, int W, int seg_len, const float *__restrict__ thr_all, unsigned long long *__restrict__ slots,
    uint32_t *__restrict__ dirty, const uint32_t *__restrict__ counters,
    const unsigned long long *__restrict__ items, const float *__restrict__ snaps, uint32_t item_cap,
    int tile_bins, const float2 *__restrict__ spec,
    const float4 *__restrict__ norm) {
  __shared__ float region_all[4][kRegion];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *region = region_all[warp];
  const uint32_t n_items = min(counters[0], item_cap);
  for (uint32_t it = blockIdx.x * 4 + warp; it < n_items; it += gridDim.x * 4) {
    const unsigned long long item = items[it];
    const int64_t tile = static_cast<int64_t>(item & 0xffffffffffull);
    const int wv = static_cast<int>((item >> 40) & 7ull);
    const int bi = static_cast<int>((item >> 43) & 0x1fffull);
    const int cx = static_cast<int>((item >> 56) & 0xffull);
    const int si = series_of_tile(tile_off, n_series, tile);
    const SeriesDev S = series[si];
    const int64_t t0 = (tile - S.tile_off) * static_cast<int64_t>(tile_bins);
    const int64_t r0 = t0 + wv * (32 * kR) + bi * kR + cx;
    const float *src = power + S.p_off;
    __syncwarp();
    for (int j = lane; j < kRegion; j += 32)
      region[j] = (r0 + j < S.m) ? (norm != nullptr ? fused_power(spec, norm, S, r0 + j, seg_len) : src[r0 + j]) : 0.0f;
    __syncwarp();
    const LaneCtx c = lane_ctx(S, t0, tile_bins, wv, lane, W, seg_len, slots, dirty);
    float s[kR];
    const float *sp = snaps + static_cast<size_t>(it) * (kR * 32) + lane;
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] = sp[i * 32];
    exact_steps<true>(s, region + lane * kR - (bi * kR + cx), bi * kR + 1, cx, min(kR, W - bi * kR),
                      thr_all + static_cast<int64_t>(si) * W, c);
  }
}

// Dump mode epilogue: slots -> (max, argmax) arrays, clearing the slots.
__global__ void unpack_kernel(unsigned long long *__restrict__ slots, int64_t n, float *__restrict__ mx,
                              uint64_t *__restrict__ am) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long k = slots[i];
    if (k == 0ull) {
      mx[i] = __int_as_float(0x7fc00000);
      am[i] = ~0ull;
    } else {
      mx[i] = __uint_as_float(static_cast<uint32_t>(k >> 32));
      am[i] = static_cast<uint64_t>(0xffffffffu - static_cast<uint32_t>(k & 0xffffffffull));
      slots[i] = 0ull;
    }
  }
}

}  // namespace

int search_tile_bins(int warps, int groups) { return 32 * kR * warps * groups; }

int search_smem_bytes(int W, int warps, int groups, int *buf_len_out) {
  const int nb = (W + kR - 1) / kR;
  int buf_len = search_tile_bins(warps, groups) + nb * kR + 3 * kR;
  buf_len = (buf_len + 3) & ~3;
  const int nq33 = buf_len / kR, nq11 = buf_len / kSub;
  if (buf_len_out) *buf_len_out = buf_len;
  return 128 + 4 * (buf_len + nq33 + 1 + nq11 + 1);
}

SmemLimit g_lim_search, g_lim_search2, g_lim_dump;

int prepare_bank(pulscan_plan p) {
  const int smem = search_smem_bytes(p->z_max, p->search_warps, p->search_groups, nullptr);
  if (smem > 220 * 1024) return fail(PULSCAN_ERR_UNSUPPORTED, "z_max too large for the shared-memory tile");
  int rc = p->search_groups == 2 ? ensure_smem(boxcar_kernel<true, true>, smem, g_lim_search2)
                                 : ensure_smem(boxcar_kernel<true, false>, smem, g_lim_search);
  if (!rc) rc = ensure_smem(boxcar_kernel<false, false>, smem, g_lim_dump);
  if (rc) return rc;
  // persistent grid: as many CTAs as fit on the GPU at once
  int b0 = 0, b1 = 0;
  if (p->search_groups == 2)
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, boxcar_kernel<true, true>, 32 * p->search_warps, smem));
  else
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, boxcar_kernel<true, false>, 32 * p->search_warps,
                                                          smem));
  PS_CUDA(
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, boxcar_kernel<false, false>, 32 * p->search_warps, smem));
  p->persist_grid[0] = b0 * p->n_ranges;
  p->persist_grid[1] = b1 * p->n_ranges;
  return PULSCAN_OK;
}

// The deferred blocks the bank left in the item list (after every bank launch
// of the search).
int launch_deferred(pulscan_plan p, const float *d_power, cudaStream_t s, const float *d_spec) {
  const int tile_bins = search_tile_bins(p->search_warps, p->search_groups);
  const uint32_t cap = static_cast<uint32_t>(p->item_cap);
  const float2 *spec = reinterpret_cast<const float2 *>(d_spec);
  const float4 *norm = d_spec ? reinterpret_cast<const float4 *>(p->d_norm) : nullptr;
  if (p->seg_len >= 2 * kR && p->defer_form == 1)
    deferred_warp_kernel<<<p->defer_grid_warp, 32 * kDwWarps, 0, s>>>(
        d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
        p->d_thresh, p->d_slots, p->d_dirty, p->d_counters, p->d_items, p->d_snaps, cap, tile_bins, spec, norm);
  else if (p->seg_len >= 2 * kR)
    deferred_kernel<<<p->defer_grid, kDeferThreads, 0, s>>>(
        d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
        p->d_thresh, p->d_slots, p->d_dirty, p->d_counters, p->d_items, p->d_snaps, cap, tile_bins, spec, norm);
  else
    deferred_small_kernel<<<p->defer_grid, 128, 0, s>>>(
        d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
        p->d_thresh, p->d_slots, p->d_dirty, p->d_counters, p->d_items, p->d_snaps, cap, tile_bins, spec, norm);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

// The search bank over tiles [tile_lo, tile_lo + n_tiles) only, one CTA per
// tile (a part of a pipelined batch: its deferred blocks wait for
// launch_deferred after the last part).
int launch_search_tiles(pulscan_plan p, const float *d_power, int64_t tile_lo, int64_t n_tiles, cudaStream_t s) {
  if (n_tiles <= 0) return PULSCAN_OK;
  if (n_tiles > 0x7fffffffLL) return fail(PULSCAN_ERR_UNSUPPORTED, "too many search tiles");
  int buf_len = 0;
  const int groups = p->search_groups;
  const int smem = search_smem_bytes(p->z_max, p->search_warps, groups, &buf_len);
  const int tile_bins = search_tile_bins(p->search_warps, groups);
  const uint32_t cap = static_cast<uint32_t>(p->item_cap);
  const int rc = groups == 2 ? ensure_smem(boxcar_kernel<true, true>, smem, g_lim_search2)
                             : ensure_smem(boxcar_kernel<true, false>, smem, g_lim_search);
  if (rc) return rc;
  const dim3 grid(static_cast<unsigned>(n_tiles)), block(32 * p->search_warps);
  if (groups == 2)
    boxcar_kernel<true, true><<<grid, block, smem, s>>>(
        d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
        p->d_thresh, p->d_thresh_bound, p->d_slots, p->d_dirty, p->d_counters, p->d_items, p->d_snaps, cap,
        tile_bins, buf_len, nullptr, nullptr, 1, groups, 0u, tile_lo, nullptr, nullptr);
  else
    boxcar_kernel<true, false><<<grid, block, smem, s>>>(
        d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
        p->d_thresh, p->d_thresh_bound, p->d_slots, p->d_dirty, p->d_counters, p->d_items, p->d_snaps, cap,
        tile_bins, buf_len, nullptr, nullptr, 1, groups, 0u, tile_lo, nullptr, nullptr);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

// d_spec != nullptr: the fused search (P formed from d_spec and p->d_norm;
// d_power is neither read nor written).
static int launch_bank(pulscan_plan p, const float *d_power, bool search, cudaStream_t s,
                       const float *d_spec = nullptr) {
  const float2 *spec = reinterpret_cast<const float2 *>(d_spec);
  const float4 *norm = d_spec ? reinterpret_cast<const float4 *>(p->d_norm) : nullptr;
  int buf_len = 0;
  const int groups = p->search_groups;
  const int smem = search_smem_bytes(p->z_max, p->search_warps, groups, &buf_len);
  if (p->total_tiles > 0x7fffffffLL) return fail(PULSCAN_ERR_UNSUPPORTED, "too many search tiles");
  // persistent for grids of three or more full waves (claim counters zeroed
  // by the caller); a smaller grid keeps one CTA per tile, since each SM
  // needs all its resident warps busy for full issue and a persistent grid
  // would run its last round with fewer CTAs per SM
  const int pg0 = p->persist_grid[search ? 0 : 1];
  const bool persist = p->persist_mode < 0 ? p->total_tiles >= 3LL * pg0 : p->persist_mode > 0;
  const int pg = (pg0 > 0 && persist) ? pg0 : 0;
  uint32_t *ctr = pg > 0 ? p->d_counters + 4 : nullptr;
  const dim3 grid(static_cast<unsigned>(pg > 0 ? std::min<int64_t>(p->total_tiles, pg) : p->total_tiles));
  const dim3 block(32 * p->search_warps);
  const int tile_bins = search_tile_bins(p->search_warps, groups);
  const uint32_t cap = static_cast<uint32_t>(p->item_cap);
  // a timeout test applies to the next search only
  const uint32_t wait_test = search ? p->wait_test_us : 0u;
  if (search) p->wait_test_us = 0u;
  int rc = PULSCAN_OK;
  if (!search) rc = ensure_smem(boxcar_kernel<false, false>, smem, g_lim_dump);
  else if (groups == 2) rc = ensure_smem(boxcar_kernel<true, true>, smem, g_lim_search2);
  else rc = ensure_smem(boxcar_kernel<true, false>, smem, g_lim_search);
  if (rc) return rc;
  if (search) {
    if (groups == 2)
      boxcar_kernel<true, true><<<grid, block, smem, s>>>(
          d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
          p->d_thresh, p->d_thresh_bound, p->d_slots, p->d_dirty, p->d_counters, p->d_items, p->d_snaps, cap,
          tile_bins, buf_len, ctr, p->d_ranges, p->n_ranges, groups, wait_test, 0, spec, norm);
    else
      boxcar_kernel<true, false><<<grid, block, smem, s>>>(
          d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
          p->d_thresh, p->d_thresh_bound, p->d_slots, p->d_dirty, p->d_counters, p->d_items, p->d_snaps, cap,
          tile_bins, buf_len, ctr, p->d_ranges, p->n_ranges, groups, wait_test, 0, spec, norm);
    PS_CUDA(cudaGetLastError());
    record(p, 5, s);
    record(p, 6, s);
    rc = launch_deferred(p, d_power, s, d_spec);
    if (rc) return rc;
    record(p, 7, s);
  } else {
    boxcar_kernel<false, false><<<grid, block, smem, s>>>(
        d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
        p->d_thresh, p->d_thresh_bound, p->d_slots, p->d_dirty, p->d_counters, p->d_items, p->d_snaps, 0u,
        tile_bins, buf_len, ctr, p->d_ranges, p->n_ranges, groups, 0u, 0, nullptr, nullptr);
  }
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

// Dump-mode launch with caller-supplied descriptor and scratch pointers
// (used by the allocation-free entry point; no plan involved).
int prepare_bank_raw(int W, int warps) {
  return ensure_smem(boxcar_kernel<false, false>, search_smem_bytes(W, warps, 1, nullptr), g_lim_dump);
}

int launch_segmax_raw(const float *d_power, const SeriesDev *d_series, const int64_t *d_tile_off, int64_t tiles,
                      int warps, int W, int seg_len, unsigned long long *d_slots, uint32_t *d_counters,
                      int64_t n_slots, float *d_max, uint64_t *d_argmax, cudaStream_t s) {
  int buf_len = 0;
  const int smem = search_smem_bytes(W, warps, 1, &buf_len);
  const int rc = ensure_smem(boxcar_kernel<false, false>, smem, g_lim_dump);
  if (rc) return rc;
  boxcar_kernel<false, false><<<static_cast<unsigned>(tiles), 32 * warps, smem, s>>>(
      d_power, d_series, d_tile_off, 1, W, seg_len, nullptr, nullptr, d_slots, nullptr, d_counters, nullptr,
      nullptr, 0u, search_tile_bins(warps, 1), buf_len, nullptr, nullptr, 1, 1, 0u, 0, nullptr, nullptr);
  PS_CUDA(cudaGetLastError());
  unpack_kernel<<<1024, 256, 0, s>>>(d_slots, n_slots, d_max, d_argmax);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

int launch_maxima_only(pulscan_plan p, const float *d_power, cudaStream_t s) {
  return launch_bank(p, d_power, false, s);   // tile claim counters zeroed with the others by the caller
}

int launch_search(pulscan_plan p, const float *d_power, cudaStream_t s, const float *d_spec) {
  return launch_bank(p, d_power, true, s, d_spec);
}

int launch_segmax(pulscan_plan p, const float *d_power, float *d_max, uint64_t *d_argmax, cudaStream_t s) {
  const int64_t n = p->total_seg * static_cast<int64_t>(p->z_max);
  PS_CUDA(cudaMemsetAsync(p->d_slots, 0, static_cast<size_t>(n) * sizeof(unsigned long long), s));
  PS_CUDA(cudaMemsetAsync(p->d_counters + 4, 0, static_cast<size_t>(p->n_ranges) * sizeof(uint32_t), s));
  record(p, 10, s);
  int rc = launch_bank(p, d_power, false, s);
  if (rc) return rc;
  record(p, 11, s);
  unpack_kernel<<<1024, 256, 0, s>>>(p->d_slots, n, d_max, d_argmax);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // namespace ps
