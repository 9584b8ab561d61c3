// Boxcar filter bank + per-(segment, width) maximum (paper §2.2.5 and
// Algorithm 4), GB300 design.
//
// Work decomposition: a CTA of kWarps warps owns a tile of kTileBins
// consecutive start bins of one series; lane l of warp v owns the kR = 33
// start bins k0 .. k0+32, k0 = tile + 33 (32 v + l).  The tile plus its halo
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
#include "common.cuh"
#include "ptx.cuh"

namespace ps {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

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
  uint32_t *touched;
  uint32_t touched_cap;
  uint32_t *counters;
};

__device__ __forceinline__ unsigned long long slot_key(float v, uint32_t bin) {
  return (static_cast<unsigned long long>(__float_as_uint(v)) << 32) |
         static_cast<unsigned long long>(0xffffffffu - bin);
}

// Merge one (segment, width) maximum into its slot; in search mode record the
// slot the first time it is touched so the finaliser can visit (and clear)
// only touched slots.
template <bool kSearch>
__device__ __noinline__ void emit_slot(unsigned long long *slots, uint32_t *touched, uint32_t cap,
                                       uint32_t *counters, uint64_t idx, unsigned long long key) {
  const unsigned long long old = atomicMax(slots + idx, key);
  if (kSearch && old == 0ull) {
    const uint32_t t = atomicAdd(counters + 0, 1u);
    if (t < cap) touched[t] = static_cast<uint32_t>(idx);
  }
}

// Segmented warp max-reduction of this step's per-lane bests and merge into
// the slots.  Each lane offers at most two parts: bins [0, ib) in segment
// seg_a and bins [ib, 33) in segment seg_a + 1 (v < 0: no entry).  The warp
// reduces the parts that fall into its first two segments; any part beyond
// (only possible when segment_len < 66) is merged lane by lane.
template <bool kSearch>
__device__ __forceinline__ void merge_step(const LaneCtx &c, int w, float vA, int iA, float vB, int iB) {
  const int64_t s_first = __shfl_sync(kFull, c.seg_a, 0);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int64_t X = s_first + t;
    float v = -1.0f;
    int i = -1;
    if (c.seg_a == X) {
      v = vA;
      i = iA;
    } else if (c.seg_a + 1 == X) {
      v = vB;
      i = iB;
    }
    const bool has = (i >= 0);
    const unsigned any = __ballot_sync(kFull, has);
    if (any == 0u) continue;
    const uint32_t bits = has ? __float_as_uint(v) : 0u;
    const uint32_t bmax = __reduce_max_sync(kFull, bits);
    const uint32_t bin = (has && bits == bmax) ? static_cast<uint32_t>(c.k0 + i) : 0xffffffffu;
    const uint32_t bmin = __reduce_min_sync(kFull, bin);
    if ((threadIdx.x & 31) == 0) {
      const uint64_t idx = static_cast<uint64_t>(X) * c.W + (w - 1);
      emit_slot<kSearch>(c.slots, c.touched, c.touched_cap, c.counters, idx,
                         slot_key(__uint_as_float(bmax), bmin));
    }
  }
  // parts outside the warp's first two segments
  if (iA >= 0 && c.seg_a > s_first + 1) {
    emit_slot<kSearch>(c.slots, c.touched, c.touched_cap, c.counters,
                       static_cast<uint64_t>(c.seg_a) * c.W + (w - 1),
                       slot_key(vA, static_cast<uint32_t>(c.k0 + iA)));
  }
  if (iB >= 0 && c.seg_a + 1 > s_first + 1) {
    emit_slot<kSearch>(c.slots, c.touched, c.touched_cap, c.counters,
                       static_cast<uint64_t>(c.seg_a + 1) * c.W + (w - 1),
                       slot_key(vB, static_cast<uint32_t>(c.k0 + iB)));
  }
}

// Exact mode: steps w = wf + cb .. wf + ce - 1 with every sum compared.  The
// sums stay in registers (static index i); the window is read straight from
// shared memory (33 loads per step: this path is rare in search mode).
// kSearch: emit maxima of bins with s_i >= T_w; otherwise emit every maximum.
template <bool kSearch>
__device__ __forceinline__ void exact_steps(float (&s)[kR], const float *__restrict__ lane_buf, int wf,
                                            int cb, int ce, const float *__restrict__ thr,
                                            const LaneCtx &c) {
  // segment_len < 66 lets a lane's 33 bins reach a third segment: then every
  // bin is merged on its own (only tiny test shapes take this branch)
  const bool small_seg = c.seg_len < 2 * kR;
  for (int cc = cb; cc < ce; ++cc) {
    const int w = wf + cc;
    const float *pw = lane_buf + (w - 1);
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
          const int64_t sg = c.seg_base + min((c.k0 + i) / c.seg_len, c.seg_last - c.seg_base);
          emit_slot<kSearch>(c.slots, c.touched, c.touched_cap, c.counters,
                             static_cast<uint64_t>(sg) * c.W + (w - 1),
                             slot_key(s[i], static_cast<uint32_t>(c.k0 + i)));
        }
      }
      continue;
    }
    float vA = -1.0f, vB = -1.0f;
    int iA = -1, iB = -1;
#pragma unroll
    for (int i = 0; i < kR; ++i) {
      if (i < lim && (!kSearch || s[i] >= T)) {
        if (i < c.ib) {
          if (s[i] > vA) { vA = s[i]; iA = i; }
        } else {
          if (s[i] > vB) { vB = s[i]; iB = i; }
        }
      }
    }
    if (!__any_sync(kFull, (iA >= 0) || (iB >= 0))) continue;
    merge_step<kSearch>(c, w, vA, iA, vB, iB);
  }
}

// Fast mode: steps C0 .. C0+NC-1 of the 33-step ring, adds only.
template <int C0, int NC>
__device__ __forceinline__ void fast_steps(float (&s)[kR], float (&b)[kR], const float *__restrict__ pb) {
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    const int c = C0 + cc;
    b[(c + kR - 1) % kR] = pb[c + kR - 1];
#pragma unroll
    for (int i = 0; i < kR; ++i) s[i] += b[(i + c) % kR];
  }
}

// Reload the ring after an exact run that ended at step CE of the block:
// the ring must hold positions [33 bi + CE, 33 bi + CE + 31].
template <int CE>
__device__ __forceinline__ void reload_ring(float (&b)[kR], const float *__restrict__ pb) {
#pragma unroll
  for (int j = 0; j < kR - 1; ++j) b[(CE + j) % kR] = pb[CE + j];
}

template <bool kSearch>
__global__ void __launch_bounds__(kThreads) boxcar_kernel(
    const float *__restrict__ power, const SeriesDev *__restrict__ series, const int64_t *__restrict__ tile_off,
    int n_series, int W, int seg_len, const float *__restrict__ thr_all, const float *__restrict__ thrb_all,
    unsigned long long *__restrict__ slots, uint32_t *__restrict__ touched, uint32_t touched_cap,
    uint32_t *__restrict__ counters, int buf_len) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  float *buf = reinterpret_cast<float *>(smem_raw + 128);
  const int nq33 = buf_len / kR;        // 33-bin block sums
  const int nq11 = buf_len / kSub;      // 11-bin block sums
  float *q33 = buf + buf_len;
  float *q11 = q33 + nq33 + 1;

  // tile -> series (largest i with tile_off[i] <= tile)
  const int64_t tile = blockIdx.x;
  int lo = 0, hi = n_series - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_off[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  const SeriesDev S = series[lo];
  const int64_t t0 = (tile - S.tile_off) * static_cast<int64_t>(kTileBins);
  const float *src = power + S.p_off + t0;
  const int64_t avail64 = S.m - t0;
  const int avail = static_cast<int>(min64(avail64, static_cast<int64_t>(buf_len)));
  // a 16-byte multiple from a 16-byte aligned source; the rest by plain loads
  const int n_tma = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0u && avail > 0) ? (avail & ~3) : 0;

  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && n_tma > 0) {
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(n_tma) * 4u);
    tma_load_1d(buf, src, static_cast<uint32_t>(n_tma) * 4u, bar);
  }
  for (int i = n_tma + threadIdx.x; i < buf_len; i += kThreads) buf[i] = (i < avail) ? src[i] : 0.0f;
  if (n_tma > 0) {
    if (!mbar_wait_bounded(bar, 0, 2000000000ull)) {
      if (threadIdx.x == 0) atomicOr(counters + 2, kErrTimeout);
      return;   // nothing else is in flight: the only copy is this one
    }
  }
  __syncthreads();

  // block sums for the bounds: q11[j] = sum of 11 bins from 11 j,
  // q33[j] = sum of 33 bins from 33 j
  for (int j = threadIdx.x; j < nq11; j += kThreads) {
    const float *p = buf + kSub * j;
    float a = 0.0f;
#pragma unroll
    for (int x = 0; x < kSub; ++x) a += p[x];
    q11[j] = a;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nq33; j += kThreads) q33[j] = q11[3 * j] + q11[3 * j + 1] + q11[3 * j + 2];
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x0 = warp * (32 * kR) + lane * kR;   // buffer-relative first bin
  LaneCtx c;
  c.k0 = t0 + x0;
  c.m = S.m;
  const int64_t tile_end = min(t0 + static_cast<int64_t>(kTileBins), S.m);
  c.lim_tile = static_cast<int>(max64(min64(tile_end - c.k0, kR), -1));
  c.seg_len = seg_len;
  c.seg_base = S.seg_off;
  c.seg_last = S.seg_off + S.n_seg - 1;
  const int64_t sa_local = min(c.k0 / seg_len, S.n_seg - 1);
  c.seg_a = S.seg_off + sa_local;
  c.ib = (sa_local < S.n_seg - 1) ? static_cast<int>(min64((sa_local + 1) * seg_len - c.k0, kR)) : kR;
  c.W = W;
  c.slots = slots;
  c.touched = touched;
  c.touched_cap = touched_cap;
  c.counters = counters;
  const float *thr = thr_all + static_cast<int64_t>(lo) * W;
  const float *thrb = thrb_all + static_cast<int64_t>(lo) * W;

  float s[kR], b[kR];
#pragma unroll
  for (int i = 0; i < kR; ++i) s[i] = 0.0f;
  const float *lane_buf = buf + x0;

  if (!kSearch) {
    exact_steps<false>(s, lane_buf, 1, 0, W, thr, c);
    return;
  }

#pragma unroll
  for (int j = 0; j < kR - 1; ++j) b[j] = lane_buf[j];
  b[kR - 1] = 0.0f;

  const int nb = (W + kR - 1) / kR;
  for (int bi = 0; bi < nb; ++bi) {
    const float *pb = lane_buf + bi * kR;
    const int wf = bi * kR + 1;
    const int nsteps = min(kR, W - bi * kR);
    if (bi < kEarlyBlocks) {
      // three sub-blocks of 11 widths, bound per 11 bins
#pragma unroll
      for (int sub = 0; sub < 3; ++sub) {
        const int cb = sub * kSub;
        if (cb >= nsteps) break;
        const int ce = min(cb + kSub, nsteps);
        const int qj = (x0 + bi * kR + cb) / kSub;
        const float tb = thrb[wf + cb - 1];
        const bool hit = (s[0] + q11[qj] + q11[qj + 1] >= tb) ||
                         (s[kSub] + q11[qj + 1] + q11[qj + 2] >= tb) ||
                         (s[2 * kSub] + q11[qj + 2] + q11[qj + 3] >= tb);
        const bool exact = __any_sync(kFull, hit) || (ce - cb < kSub);
        if (exact) {
          exact_steps<true>(s, lane_buf, wf, cb, ce, thr, c);
          if (sub == 0) reload_ring<kSub>(b, pb);
          else if (sub == 1) reload_ring<2 * kSub>(b, pb);
          else reload_ring<3 * kSub>(b, pb);
        } else {
          if (sub == 0) fast_steps<0, kSub>(s, b, pb);
          else if (sub == 1) fast_steps<kSub, kSub>(s, b, pb);
          else fast_steps<2 * kSub, kSub>(s, b, pb);
        }
      }
    } else {
      const int qj = (x0 + bi * kR) / kR;
      const bool hit = s[0] + q33[qj] + q33[qj + 1] >= thrb[wf - 1];
      const bool exact = __any_sync(kFull, hit) || (nsteps < kR);
      if (exact) {
        exact_steps<true>(s, lane_buf, wf, 0, nsteps, thr, c);
        reload_ring<kR>(b, pb);
      } else {
        fast_steps<0, kR>(s, b, pb);
      }
    }
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

int search_smem_bytes(int W, int *buf_len_out) {
  const int nb = (W + kR - 1) / kR;
  int buf_len = kTileBins + nb * kR + 3 * kR;
  buf_len = (buf_len + 3) & ~3;
  const int nq33 = buf_len / kR, nq11 = buf_len / kSub;
  if (buf_len_out) *buf_len_out = buf_len;
  return 128 + 4 * (buf_len + nq33 + 1 + nq11 + 1);
}

static int launch_bank(pulscan_plan p, const float *d_power, bool search, cudaStream_t s) {
  int buf_len = 0;
  const int smem = search_smem_bytes(p->z_max, &buf_len);
  if (p->total_tiles > 0x7fffffffLL) return fail(PULSCAN_ERR_UNSUPPORTED, "too many search tiles");
  if (search) {
    boxcar_kernel<true><<<static_cast<unsigned>(p->total_tiles), kThreads, smem, s>>>(
        d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
        p->d_thresh, p->d_thresh_bound, p->d_slots, p->d_touched, static_cast<uint32_t>(p->touched_cap),
        p->d_counters, buf_len);
  } else {
    boxcar_kernel<false><<<static_cast<unsigned>(p->total_tiles), kThreads, smem, s>>>(
        d_power, p->d_series, p->d_tile_off, static_cast<int>(p->series.size()), p->z_max, p->seg_len,
        p->d_thresh, p->d_thresh_bound, p->d_slots, p->d_touched, static_cast<uint32_t>(p->touched_cap),
        p->d_counters, buf_len);
  }
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

int prepare_bank(pulscan_plan p) {
  const int smem = search_smem_bytes(p->z_max, nullptr);
  if (smem > 220 * 1024) return fail(PULSCAN_ERR_UNSUPPORTED, "z_max too large for the shared-memory tile");
  PS_CUDA(cudaFuncSetAttribute(boxcar_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  PS_CUDA(cudaFuncSetAttribute(boxcar_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return PULSCAN_OK;
}

int launch_search(pulscan_plan p, const float *d_power, cudaStream_t s) {
  return launch_bank(p, d_power, true, s);
}

int launch_segmax(pulscan_plan p, const float *d_power, float *d_max, uint64_t *d_argmax, cudaStream_t s) {
  const int64_t n = p->total_seg * static_cast<int64_t>(p->z_max);
  PS_CUDA(cudaMemsetAsync(p->d_slots, 0, static_cast<size_t>(n) * sizeof(unsigned long long), s));
  record(p, 8, s);
  int rc = launch_bank(p, d_power, false, s);
  if (rc) return rc;
  record(p, 9, s);
  unpack_kernel<<<1024, 256, 0, s>>>(p->d_slots, n, d_max, d_argmax);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // namespace ps
