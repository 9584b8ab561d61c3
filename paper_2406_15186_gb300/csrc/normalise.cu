// Per-segment median/MAD normalisation and power (paper §2.2.3, Eq. 8).
//
// One CTA per segment (normalisation block).  The block's complex bins are
// staged into shared memory by one TMA bulk copy (or read from global memory
// when the block is too large for shared memory).  The real and imaginary
// parts are normalised separately, as Eq. 8 prescribes, with EXACT order
// statistics: a radix select on order-preserving 32-bit keys of the FP32
// values (digits of 11, 11 and 10 bits, one shared-memory histogram per
// component, both components in the same pass) finds the rank-j element; an
// even count takes the mean of ranks n/2-1 and n/2, the second found from the
// first's multiplicity or by one min-reduction.  The MAD is the same select on
// |x - median|.  Then a = (x - med) / (kappa MAD), kappa = 1/Phi^{-1}(3/4),
// and P = (a^2 + b^2)/2, written coalesced.  The DC bin of a series is taken
// as 0 + 0i.  A segment whose MAD is 0 gets P = 0.
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
constexpr int kMaxSmemBins = 24576;            // float2 elements staged in shared memory

__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float kfloat(uint32_t k) {
  const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

struct SelShared {
  uint32_t hist[2][kHistBins];
  uint32_t wsum[2][8];
  uint32_t prefix[2];
  uint32_t rem[2];
  uint32_t cnt[2];
  uint32_t minkey[2];
  float med[2];
  float mad[2];
};

// Block-wide: component c = threadIdx / 256 scans its 2048-bin histogram
// (8 bins per thread) and locates the digit holding rank rem[c].
__device__ __forceinline__ void find_digit(SelShared &sh, int shift) {
  const int c = threadIdx.x >> 8;
  const int t = threadIdx.x & 255;
  const uint32_t *h = sh.hist[c] + 8 * t;
  uint32_t local = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) local += h[j];
  // inclusive scan of `local` over the 256 threads of this component
  const int lane = t & 31, wid = t >> 5;
  uint32_t v = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) sh.wsum[c][wid] = v;
  __syncthreads();
  uint32_t base = 0;
  for (int j = 0; j < wid; ++j) base += sh.wsum[c][j];
  const uint32_t excl = base + v - local;
  const uint32_t r = sh.rem[c];
  __syncthreads();   // everyone has read rem before it is updated
  if (r >= excl && r < excl + local) {
    uint32_t acc = excl;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (r < acc + h[j]) {
        sh.prefix[c] |= static_cast<uint32_t>(8 * t + j) << shift;
        sh.rem[c] = r - acc;
        sh.cnt[c] = h[j];
        break;
      }
      acc += h[j];
    }
  }
}

// Keys of the rank-`rank` and rank-`rank+1` (if `pair`) elements of both
// components; get(e) returns the element's (re-key, im-key).
template <class Get>
__device__ __forceinline__ void select2(SelShared &sh, Get get, int n, uint32_t rank, bool pair,
                                        uint32_t (&k_lo)[2], uint32_t (&k_hi)[2]) {
  if (threadIdx.x < 2) {
    sh.prefix[threadIdx.x] = 0u;
    sh.rem[threadIdx.x] = rank;
    sh.cnt[threadIdx.x] = 0u;
    sh.minkey[threadIdx.x] = 0xffffffffu;
  }
  uint32_t mask = 0u;
  const int shifts[3] = {21, 10, 0};
  const uint32_t dmasks[3] = {0x7ffu, 0x7ffu, 0x3ffu};
#pragma unroll
  for (int pass = 0; pass < 3; ++pass) {
    for (int j = threadIdx.x; j < 2 * kHistBins; j += kNormThreads) (&sh.hist[0][0])[j] = 0u;
    __syncthreads();
    const uint32_t p0 = sh.prefix[0], p1 = sh.prefix[1];
    const int sh_ = shifts[pass];
    const uint32_t dm = dmasks[pass];
    for (int e = threadIdx.x; e < n; e += kNormThreads) {
      const uint2 k = get(e);
      if ((k.x & mask) == p0) atomicAdd(&sh.hist[0][(k.x >> sh_) & dm], 1u);
      if ((k.y & mask) == p1) atomicAdd(&sh.hist[1][(k.y >> sh_) & dm], 1u);
    }
    __syncthreads();
    find_digit(sh, sh_);
    __syncthreads();
    mask |= dm << sh_;
  }
  k_lo[0] = sh.prefix[0];
  k_lo[1] = sh.prefix[1];
  if (!pair) {
    __syncthreads();   // all reads of sh done before the next select resets it
    return;
  }
  // rank+1: the same key if it repeats, else the smallest larger key
  const bool need0 = sh.rem[0] + 1 >= sh.cnt[0];
  const bool need1 = sh.rem[1] + 1 >= sh.cnt[1];
  if (need0 || need1) {
    uint32_t m0 = 0xffffffffu, m1 = 0xffffffffu;
    for (int e = threadIdx.x; e < n; e += kNormThreads) {
      const uint2 k = get(e);
      if (k.x > k_lo[0]) m0 = min(m0, k.x);
      if (k.y > k_lo[1]) m1 = min(m1, k.y);
    }
    m0 = __reduce_min_sync(0xffffffffu, m0);
    m1 = __reduce_min_sync(0xffffffffu, m1);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&sh.minkey[0], m0);
      atomicMin(&sh.minkey[1], m1);
    }
    __syncthreads();
  }
  k_hi[0] = need0 ? sh.minkey[0] : k_lo[0];
  k_hi[1] = need1 ? sh.minkey[1] : k_lo[1];
  __syncthreads();
}

__device__ __forceinline__ float mean_of(float a, float b) {
  return static_cast<float>(0.5 * (static_cast<double>(a) + static_cast<double>(b)));
}

__global__ void __launch_bounds__(kNormThreads) normalise_kernel(
    const float2 *__restrict__ spec, float *__restrict__ power, float4 *__restrict__ stats,
    const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off, int n_series, int seg_len,
    uint32_t *__restrict__ counters) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  SelShared &sh = *reinterpret_cast<SelShared *>(smem_raw + 128);
  float2 *data = reinterpret_cast<float2 *>(smem_raw + 128 + ((sizeof(SelShared) + 127) & ~size_t(127)));

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
  const bool in_smem = n <= kMaxSmemBins;

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
    if (n_tma > 0 && !mbar_wait_bounded(bar, 0, 2000000000ull)) {
      if (threadIdx.x == 0) atomicOr(counters + 2, kErrTimeout);
      return;
    }
    __syncthreads();
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

  // medians
  uint32_t klo[2], khi[2];
  select2(sh, [&](int e) { const float2 v = val(e); return make_uint2(fkey(v.x), fkey(v.y)); }, n, rank,
          even, klo, khi);
  const float med_re = even ? mean_of(kfloat(klo[0]), kfloat(khi[0])) : kfloat(klo[0]);
  const float med_im = even ? mean_of(kfloat(klo[1]), kfloat(khi[1])) : kfloat(klo[1]);
  // MADs: the same select on |x - med| (non-negative floats)
  select2(sh,
          [&](int e) {
            const float2 v = val(e);
            return make_uint2(fkey(fabsf(v.x - med_re)), fkey(fabsf(v.y - med_im)));
          },
          n, rank, even, klo, khi);
  const float mad_re = even ? mean_of(kfloat(klo[0]), kfloat(khi[0])) : kfloat(klo[0]);
  const float mad_im = even ? mean_of(kfloat(klo[1]), kfloat(khi[1])) : kfloat(klo[1]);

  const bool degenerate = !(mad_re > 0.0f) || !(mad_im > 0.0f);
  const float inv_re = degenerate ? 0.0f : static_cast<float>(1.0 / (kKappa * static_cast<double>(mad_re)));
  const float inv_im = degenerate ? 0.0f : static_cast<float>(1.0 / (kKappa * static_cast<double>(mad_im)));
  float *out = power + S.p_off + b0;
  for (int e = threadIdx.x; e < n; e += kNormThreads) {
    const float2 v = val(e);
    const float a = (v.x - med_re) * inv_re;
    const float b = (v.y - med_im) * inv_im;
    out[e] = 0.5f * (a * a + b * b);
  }
  if (threadIdx.x == 0 && stats != nullptr) stats[g] = make_float4(med_re, mad_re, med_im, mad_im);
}

}  // namespace

static int normalise_smem(pulscan_plan p) {
  int64_t max_n = 0;
  for (const auto &se : p->series) {
    const int64_t last = se.m - (se.n_seg - 1) * p->seg_len;
    max_n = std::max<int64_t>(max_n, last);
  }
  const int data_bins = static_cast<int>(std::min<int64_t>(max_n, kMaxSmemBins));
  return 128 + static_cast<int>((sizeof(SelShared) + 127) & ~size_t(127)) + 8 * data_bins;
}

int prepare_normalise(pulscan_plan p) {
  PS_CUDA(cudaFuncSetAttribute(normalise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, normalise_smem(p)));
  return PULSCAN_OK;
}

int launch_normalise(pulscan_plan p, const float *d_spec, float *d_power, float *d_stats, cudaStream_t s) {
  const int smem = normalise_smem(p);
  if (p->total_seg > 0x7fffffffLL) return fail(PULSCAN_ERR_UNSUPPORTED, "too many segments");
  float4 *st = d_stats ? reinterpret_cast<float4 *>(d_stats) : reinterpret_cast<float4 *>(p->d_stats);
  normalise_kernel<<<static_cast<unsigned>(p->total_seg), kNormThreads, smem, s>>>(
      reinterpret_cast<const float2 *>(d_spec), d_power, st, p->d_series, p->d_seg_off,
      static_cast<int>(p->series.size()), p->seg_len, p->d_counters);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // namespace ps
