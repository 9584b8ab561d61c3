// Chi-square significance used by the plan (threshold table, host, FP64) and
// by the candidate finaliser (device, FP32: GB300's FP64 rate is 1/64 of FP32).
//
// Paper §2.2.3, Eq. 9: a width-w boxcar of normalised power is a sum of w
// chi^2(2) variables.  With P = (a^2 + b^2)/2 a width-w sum S has 2S ~
// chi^2(2w), so p = Q(w, S), the regularised upper incomplete gamma.  It is
// Bonferroni-corrected for the trial count and converted to a one-sided
// Gaussian-equivalent sigma.
//
// ln Q(a, x) follows the published method of Press et al., Numerical Recipes
// (3rd ed., §6.2): the power series for P(a, x) when x < a + 1, and Legendre's
// continued fraction for Q(a, x), evaluated by the modified Lentz method,
// otherwise; both in log form so deep tails stay finite.  sigma is the root of
// ln Phi_c(sigma) = ln p, found by Newton's method on
// ln Phi_c(s) = ln(erfcx(s / sqrt 2) / 2) - s^2 / 2 (derivative
// -sqrt(2/pi) / erfcx(s / sqrt 2)); ln Phi_c is concave, so after the first
// step the iterates approach the root monotonically from above.
#pragma once
#include <math.h>

namespace ps {

__host__ __device__ inline double log_q_gamma(double a, double x) {
  if (!(x > 0.0)) return 0.0;
  const double lpre = -x + a * log(x) - lgamma(a);  // ln(x^a e^-x / Gamma(a))
  if (x < a + 1.0) {
    // P(a, x) = x^a e^-x / Gamma(a) * sum_{n>=0} x^n / (a (a+1) ... (a+n))
    double ap = a, del = 1.0 / a, sum = del;
    for (int n = 0; n < 200000; ++n) {
      ap += 1.0;
      del *= x / ap;
      sum += del;
      if (fabs(del) < fabs(sum) * 1e-17) break;
    }
    const double lp = lpre + log(sum);
    return log1p(-exp(lp));
  }
  // Q(a, x) = x^a e^-x / Gamma(a) * 1 / (x + 1 - a - 1 (1 - a) / (x + 3 - a - ...))
  const double tiny = 1e-300;
  double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 200000; ++i) {
    const double an = -i * (i - a);
    b += 2.0;
    d = an * d + b;
    if (fabs(d) < tiny) d = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    const double del = d * c;
    h *= del;
    if (fabs(del - 1.0) < 4e-16) break;   // two ulps of 1: FP64 convergence
  }
  return lpre + log(h);
}

// g(a) = a ln a - a - ln Gamma(a): with lambda = x / a and delta = lambda - 1,
//   ln(x^a e^-x / Gamma(a)) = -a (delta - ln(1 + delta)) + g(a)
// exactly, and both terms are free of cancellation (g(a) is O(ln a)).  The
// host tabulates g per width in FP64 so the device can work in FP32.
inline double g_of(double a) { return a * log(a) - a - lgamma(a); }

#ifdef __CUDACC__
// delta - ln(1 + delta), >= 0; a power series near 0 avoids the cancellation.
__device__ inline float h_delta_f32(float d) {
  if (fabsf(d) < 0.25f) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 16; k >= 2; --k) acc = fmaf(acc, d, ((k & 1) ? -1.0f : 1.0f) / static_cast<float>(k));
    return acc * d * d;
  }
  return d - log1pf(d);
}

// ln Q(a, x) in FP32 from the cancellation-free prefactor above and the same
// series / continued fraction as log_q_gamma.  Absolute error ~1e-4 at
// ln Q ~ -500 (relative ~3e-7), far inside what an FP32 sigma resolves.
__device__ inline float log_q_f32(float a, float x, float g) {
  if (!(x > 0.0f)) return 0.0f;
  const float lpre = -a * h_delta_f32((x - a) / a) + g;
  if (x < a + 1.0f) {
    float ap = a, del = 1.0f / a, sum = del;
    for (int n = 0; n < 20000; ++n) {
      ap += 1.0f;
      del *= x / ap;
      sum += del;
      if (fabsf(del) < fabsf(sum) * 1e-8f) break;
    }
    return log1pf(-expf(lpre + logf(sum)));
  }
  const float tiny = 1e-30f;
  float b = x + 1.0f - a, c = 1.0f / tiny, d = 1.0f / b, h = d;
  for (int i = 1; i < 2000; ++i) {
    const float an = -static_cast<float>(i) * (static_cast<float>(i) - a);
    b += 2.0f;
    d = fmaf(an, d, b);
    if (fabsf(d) < tiny) d = tiny;
    c = b + an / c;
    if (fabsf(c) < tiny) c = tiny;
    d = 1.0f / d;
    const float del = d * c;
    h *= del;
    if (fabsf(del - 1.0f) < 2.4e-7f) break;
  }
  return lpre + logf(h);
}

// sigma with ln Phi_c(sigma) = lp <= ln(1/2), FP32 Newton on
// ln Phi_c(s) = ln(erfcx(s / sqrt 2) / 2) - s^2 / 2.
__device__ inline float sigma_from_log_p_f32(float lp) {
  const float t = -2.0f * lp;
  float s = (t > 2.0f) ? sqrtf(fmaxf(t - logf(t) - 1.8378770664f, 0.0f)) : 0.0f;
  float prev = INFINITY;
  for (int it = 0; it < 20; ++it) {
    const float e = erfcxf(s * 0.70710678f);
    const float f = logf(0.5f * e) - 0.5f * s * s - lp;
    const float step = f * e * 1.2533141f;
    if (it >= 3 && !(fabsf(step) < prev)) break;
    s += step;
    prev = fabsf(step);
    if (prev <= 1e-7f * fmaxf(1.0f, fabsf(s))) break;
  }
  return s;
}

// sigma with ln Phi_c(sigma) = lp, lp <= ln(1/2) (device: uses erfcx).
__device__ inline double sigma_from_log_p(double lp) {
  const double t = -2.0 * lp;
  double s = (t > 2.0) ? sqrt(fmax(t - log(t) - 1.8378770664093453, 0.0)) : 0.0;  // ln(2 pi)
  // stop at a relative step of 1e-12 (the result is stored in FP32), or once
  // the steps stop shrinking: then they are FP64 rounding noise of ln Phi_c
  double prev = INFINITY;
  for (int it = 0; it < 40; ++it) {
    const double e = erfcx(s * 0.70710678118654752);
    const double f = log(0.5 * e) - 0.5 * s * s - lp;
    const double step = f * e * 1.2533141373155003;  // sqrt(pi / 2)
    if (it >= 3 && !(fabs(step) < prev)) break;
    s += step;
    prev = fabs(step);
    if (prev <= 1e-12 * fmax(1.0, fabs(s))) break;
  }
  return s;
}
#endif

}  // namespace ps
