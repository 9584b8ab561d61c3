"""Chi-square significance, Bonferroni correction and Gaussian sigma, FP64.

Test infrastructure.  §2.2.3 (Eq. 9): a width-w boxcar of unit-variance
normalised power is a sum of w independent chi^2(2) variables, so with the
P = (a^2 + b^2)/2 reading, 2 S ~ chi^2(2 w) and the p-value of a sum S is the
chi^2(2w) survival at 2S, i.e. the regularised upper incomplete gamma
Q(w, S).  For integer w this has the closed form of a Poisson CDF,

    Q(w, S) = exp(-S) * sum_{j=0}^{w-1} S^j / j!,

which is evaluated here in log space term by term (logsumexp), so it stays
finite far beyond FP64 underflow.  The p-value is then Bonferroni-corrected
for the number of trials (§2.2.3: across widths and bins; reading:
n_trials = M x number of widths searched) and turned into a one-sided
Gaussian-equivalent sigma.  The sigma inversion is a plain bisection on
log Phi_c(sigma) = log_ndtr(-sigma).
"""
import numpy as np
from scipy.special import gammaln, log_ndtr


def log_q(w, s):
    """ln Q(w, S) for integer w >= 1 and S >= 0 (Poisson-sum closed form)."""
    w = int(w)
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    j = np.arange(w, dtype=np.float64)
    lg = gammaln(j + 1.0)
    out = np.zeros_like(s)
    pos = np.nonzero(s > 0.0)[0]          # Q(w, 0) = 1
    rows = max(1, (1 << 22) // w)
    for c in range(0, pos.shape[0], rows):
        idx = pos[c:c + rows]
        si = s[idx][:, None]
        t = j[None, :] * np.log(si) - lg[None, :] - si
        mt = t.max(axis=1, keepdims=True)
        out[idx] = (mt + np.log(np.sum(np.exp(t - mt), axis=1, keepdims=True)))[:, 0]
    return np.minimum(out, 0.0)


def log_sf_normal(sigma):
    """ln Phi_c(sigma), the one-sided Gaussian tail, accurate deep in the tail."""
    return log_ndtr(-np.asarray(sigma, dtype=np.float64))


def sigma_from_log_p(lp):
    """sigma with ln Phi_c(sigma) = lp (lp <= 0), by bisection to FP64 precision."""
    lp = np.atleast_1d(np.asarray(lp, dtype=np.float64))
    lo = np.full_like(lp, -40.0)
    hi = np.sqrt(np.maximum(-2.0 * lp, 0.0)) + 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        above = log_sf_normal(mid) > lp     # tail still too heavy: sigma is larger
        lo = np.where(above, mid, lo)
        hi = np.where(above, hi, mid)
    return 0.5 * (lo + hi)


def log_p_adjusted(w, s, n_trials):
    """Bonferroni-corrected ln p = min(0, ln Q(w, S) + ln n_trials)."""
    return np.minimum(0.0, log_q(w, s) + np.log(float(n_trials)))


def passes(w, s, n_trials, sigma_thr):
    """Emission rule: Gaussian-equivalent sigma >= sigma_thr."""
    return log_p_adjusted(w, s, n_trials) <= log_sf_normal(sigma_thr)


def sigma_of(w, s, n_trials):
    """Gaussian-equivalent sigma of a width-w sum S after Bonferroni."""
    return sigma_from_log_p(log_p_adjusted(w, s, n_trials))


def threshold_power(w, sigma_thr, n_trials):
    """T_w: the smallest S with sigma(S) >= sigma_thr, by bisection on S."""
    target = float(log_sf_normal(sigma_thr)) - np.log(float(n_trials))
    lo, hi = 0.0, float(w) + 50.0 + 50.0 * np.sqrt(w) - target * 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if log_q(w, mid)[0] > target:
            lo = mid
        else:
            hi = mid
    return hi
