// Harmonic summing by decimation (paper §2.3 and its GPU decimation listing).
//
// For every series, the normalised power P (M bins) gives the stage spectra
//   X_H[r] = sum_{h=1}^{H} sum_{j=0}^{h-1} P[h r + j],  r < floor(M / H),
// H = 2..numharm: the spectrum decimated by h (adjacent non-overlapping
// groups of h bins summed) puts the h-th harmonic of a signal at r into bin
// r, and the decimated spectra are added aligned at bin 0.  For noise
// P ~ Exp(1) (chi^2_2 / 2), so X_H is a sum of H(H+1)/2 unit exponentials
// (chi^2 with H(H+1) degrees of freedom).  The stage spectra are then
// searched by the same bank as P.
//
// One thread per (series, r): the running sum over h serves every stage
// (X_H = X_{H-1} + the H-group at H r), so each P value a stage needs is read
// once per stage; a thread stops at the first stage whose group runs past M
// (later stages are shorter still).  HBM-bound: ~4 B x (numharm - 1 + 1/2)
// read and 4 B x (1/2 + 1/3 + ...) written per bin of P.
#include <algorithm>

#include "common.cuh"

namespace ps {

namespace {

constexpr int kHarmMax = 8;

__global__ void __launch_bounds__(256) harmonic_sum_kernel(float *__restrict__ power,
                                                           const SeriesDev *__restrict__ series, int n_base,
                                                           int numharm) {
  const int b = blockIdx.y;
  const SeriesDev S = series[b];
  const float *p = power + S.p_off;
  int64_t out_off[kHarmMax + 1];
#pragma unroll
  for (int h = 2; h <= kHarmMax; ++h)
    out_off[h] = (h <= numharm) ? series[static_cast<int64_t>(n_base) * (h - 1) + b].p_off : 0;
  const int64_t r_end = S.m / 2;   // stage 2 is the longest
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < r_end;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float acc = p[r];
#pragma unroll
    for (int h = 2; h <= kHarmMax; ++h) {
      if (h > numharm || h * r + h > S.m) break;   // the h-group [h r, h r + h) must lie inside M
      const float *g = p + h * r;
      float grp = 0.0f;
      for (int j = 0; j < h; ++j) grp += g[j];
      acc += grp;
      power[out_off[h] + r] = acc;
    }
  }
}

}  // namespace

int launch_harmonic_sums(pulscan_plan p, float *d_power, cudaStream_t s) {
  if (p->numharm <= 1) return PULSCAN_OK;
  if (p->n_base > 65535) return fail(PULSCAN_ERR_UNSUPPORTED, "too many series for the harmonic launch");
  int64_t max_r = 0;
  for (int64_t i = 0; i < p->n_base; ++i) max_r = std::max<int64_t>(max_r, p->series[i].m / 2);
  const unsigned gx = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((max_r + 255) / 256, 2048)));
  harmonic_sum_kernel<<<dim3(gx, static_cast<unsigned>(p->n_base)), 256, 0, s>>>(
      d_power, p->d_series, static_cast<int>(p->n_base), p->numharm);
  PS_CUDA(cudaGetLastError());
  return PULSCAN_OK;
}

}  // namespace ps
