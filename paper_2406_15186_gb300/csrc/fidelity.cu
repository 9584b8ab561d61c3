// "Paper-GPU fidelity" mode: the GPU version's approximations of §2.5 and
// §2.6, for comparison with the exact path.
//
// * mom_normalise_kernel: per block, median and MAD of each component by
//   median of medians over the block's first L = 4^k bins (the appendix
//   listing: each level with stride s replaces v[t], t < s, by the local
//   median of v[t], v[t+s], v[t+2s], v[t+3s]; s = L/4, L/16, ..., 1), MAD =
//   the same reduction over |x - median|, scale 1.4826; then
//   P = (a^2 + b^2)/2 over all the block's bins.  The local median is the
//   mean of the two middle values, which the listing writes as
//   (a + b + c + d - min - max)/2; here the two middle values are selected
//   with min/max and averaged, the same number without that form's
//   cancellation when min or max is large.
// * poly_finalize_kernel: Algorithm 4's per-(chunk, width) maxima (all of
//   them: the polynomial is not monotone in the power, so no power threshold
//   can stand in for it) -> log p by the fitted polynomial of §2.6 in FP64
//   (pow = 2 S, dof = 2 a, a the gamma shape of S), Bonferroni, and a record
//   for every maximum whose sigma reaches the threshold.  Every slot is read
//   and cleared.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "signif.cuh"

namespace ps {

namespace {

constexpr int kMomThreads = 256;
constexpr double kMomScale = 1.4826;

__device__ __forceinline__ float local_median(float a, float b, float c, float d) {
  const float lo = fmaxf(fminf(a, b), fminf(c, d));
  const float hi = fminf(fmaxf(a, b), fmaxf(c, d));
  return 0.5f * (lo + hi);
}

// In-place reduction of x[0..L) and y[0..L) to x[0], y[0]; ends with a barrier.
__device__ void mom_reduce(float *x, float *y, int L) {
  for (int s = L / 4; s >= 1; s /= 4) {
    for (int t = threadIdx.x; t < s; t += blockDim.x) {
      x[t] = local_median(x[t], x[t + s], x[t + 2 * s], x[t + 3 * s]);
      y[t] = local_median(y[t], y[t + s], y[t + 2 * s], y[t + 3 * s]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kMomThreads) mom_normalise_kernel(
    const float2 *__restrict__ spec, float *__restrict__ power, float4 *__restrict__ stats,
    const SeriesDev *__restrict__ series, const int64_t *__restrict__ seg_off, int n_series, int seg_len) {
  extern __shared__ __align__(16) float msh[];
  float *xr = msh, *xi = msh + seg_len;
  __shared__ float bc[6];
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
  const bool dc = b0 == 0;
  auto val = [&](int i) { return (dc && i == 0) ? make_float2(0.0f, 0.0f) : src[i]; };
  for (int i = threadIdx.x; i < seg_len; i += blockDim.x) {
    const float2 v = val(i);
    xr[i] = v.x;
    xi[i] = v.y;
  }
  __syncthreads();
  mom_reduce(xr, xi, seg_len);
  const float med_re = xr[0], med_im = xi[0];
  __syncthreads();
  for (int i = threadIdx.x; i < seg_len; i += blockDim.x) {
    const float2 v = val(i);
    xr[i] = fabsf(v.x - med_re);
    xi[i] = fabsf(v.y - med_im);
  }
  __syncthreads();
  mom_reduce(xr, xi, seg_len);
  if (threadIdx.x == 0) {
    const float mad_re = xr[0], mad_im = xi[0];
    const bool degenerate = !(mad_re > 0.0f) || !(mad_im > 0.0f);
    bc[0] = degenerate ? 0.0f : static_cast<float>(1.0 / (kMomScale * static_cast<double>(mad_re)));
    bc[1] = degenerate ? 0.0f : static_cast<float>(1.0 / (kMomScale * static_cast<double>(mad_im)));
    if (stats != nullptr) stats[g] = make_float4(med_re, mad_re, med_im, mad_im);
  }
  __syncthreads();
  const float inv_re = bc[0], inv_im = bc[1];
  float *out = power + S.p_off + b0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 v = val(i);
    const float a = (v.x - med_re) * inv_re;
    const float b = (v.y - med_im) * inv_im;
    out[i] = 0.5f * (a * a + b * b);
  }
}

// §2.6's fit: natural log p of a chi-square value pw with dof degrees of
// freedom; 0 when dof >= 1.05 pw.
__device__ __forceinline__ double poly_logp(double pw, double dof) {
  if (dof >= 1.05 * pw) return 0.0;
  const double x = 1500.0 * dof / pw;
  double f = -4.4604059e-46;
  f = f * x + 9.4927863e-42;
  f = f * x - 9.1470451e-38;
  f = f * x + 5.2810851e-34;
  f = f * x - 2.0376166e-30;
  f = f * x + 5.5480334e-27;
  f = f * x - 1.0973877e-23;
  f = f * x + 1.5991804e-20;
  f = f * x - 1.7231488e-17;
  f = f * x + 1.3660070e-14;
  f = f * x - 7.8617952e-12;
  f = f * x + 3.2136336e-09;
  f = f * x - 9.0466418e-07;
  f = f * x + 0.00016945948;
  f = f * x - 0.021494231;
  f = f * x + 2.9515954;
  f = f * x - 755.24091;
  return pw * f / 1500.0;
}

__global__ void poly_finalize_kernel(unsigned long long *__restrict__ slots, int64_t n_slots,
                                     uint32_t *__restrict__ counters, int W, const SeriesDev *__restrict__ series,
                                     const int64_t *__restrict__ seg_off, int n_series,
                                     const double *__restrict__ ln_trials, const uint8_t *__restrict__ searched,
                                     double ln_target, pulscan_cand *__restrict__ cands, uint32_t max_cands) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  // whole warps walk consecutive slots so the output reservation is per warp
  for (int64_t i0 = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) & ~int64_t(31); i0 < n_slots;
       i0 += stride) {
    const int64_t idx = i0 + lane;
    unsigned long long key = 0ull;
    if (idx < n_slots) {
      key = slots[idx];
      if (key != 0ull) slots[idx] = 0ull;
    }
    bool pass = false;
    float lpf = 0.0f, pw = 0.0f;
    uint32_t bin = 0u, hh = 1u;
    int w = 0, sidx = 0;
    if (key != 0ull) {
      const int64_t gseg = idx / W;
      w = static_cast<int>(idx % W) + 1;
      int lo = 0, hi = n_series - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= gseg) lo = mid; else hi = mid - 1;
      }
      sidx = lo;
      hh = series[lo].harm;
      pw = __uint_as_float(static_cast<uint32_t>(key >> 32));
      bin = 0xffffffffu - static_cast<uint32_t>(key & 0xffffffffull);
      const double a = 0.5 * hh * (hh + 1) * w;
      const double lp = fmin(0.0, poly_logp(2.0 * pw, 2.0 * a) + ln_trials[lo]);
      pass = searched[w - 1] && lp <= ln_target;
      lpf = static_cast<float>(lp);
    }
    const unsigned act = __ballot_sync(0xffffffffu, pass);
    uint32_t base = 0;
    if (lane == 0 && act) base = atomicAdd(counters + 1, static_cast<uint32_t>(__popc(act)));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!pass) continue;
    const uint32_t o = base + static_cast<uint32_t>(__popc(act & ((1u << lane) - 1u)));
    if (o < max_cands) {
      pulscan_cand c;
      c.series = series[sidx].user_index;
      c.width = static_cast<uint32_t>(w);
      c.bin = bin;
      c.power = pw;
      c.sigma = sigma_from_log_p_f32(lpf);
      c.harmonics = hh;
      c.reserved = 0u;
      cands[o] = c;
    }
  }
}

}  // namespace

bool is_power_of_four(int64_t v) { return v >= 1 && (v & (v - 1)) == 0 && ((63 - __builtin_clzll(v)) % 2) == 0; }

int launch_normalise_mom(pulscan_plan p, const float *d_spec, float *d_power, float *d_stats, cudaStream_t s) {
  const int smem = 2 * p->seg_len * static_cast<int>(sizeof(float));
  static SmemLimit lim;
  const int rc = ensure_smem(mom_normalise_kernel, smem, lim);
  if (rc) return rc;
  float4 *st = d_stats ? reinterpret_cast<float4 *>(d_stats) : reinterpret_cast<float4 *>(p->d_stats);
  mom_normalise_kernel<<<static_cast<unsigned>(p->base_seg), kMomThreads, smem, s>>>(
      reinterpret_cast<const float2 *>(d_spec), d_power, st, p->d_series, p->d_seg_off,
      static_cast<int>(p->n_base), p->seg_len);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

int launch_poly_finalize(pulscan_plan p, cudaStream_t s) {
  const int64_t n_slots = p->total_seg * static_cast<int64_t>(p->z_max);
  const int grid = static_cast<int>(std::min<int64_t>(std::max<int64_t>((n_slots + 255) / 256, 1), 4 * 152 * 4));
  const double ln_target = host_log_sf_normal(p->sigma_thr);
  poly_finalize_kernel<<<grid, 256, 0, s>>>(p->d_slots, n_slots, p->d_counters, p->z_max, p->d_series,
                                            p->d_seg_off, static_cast<int>(p->series.size()), p->d_ln_trials,
                                            p->d_searched, ln_target, p->d_cands,
                                            static_cast<uint32_t>(p->max_cands));
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // namespace ps
