"""Host analysis of the effective-mass series (App. B): statistical errors of
the m*/m partial sums, the truncation uncertainty from the last three
orders, the choice of the screening parameter over a scan, and the
linear-in-T extrapolation to zero temperature.

Readings where the paper gives the procedure in words only:

* statistical errors: the self-energy estimates of different roots are
  taken as independent, and their errors are propagated to the partial sums
  linearly, through the Jacobian of the post-process (`api.postprocess`,
  the C-ABI host routine) by central differences;
* truncation: the estimate is the highest-order partial sum, and its
  systematic uncertainty the largest deviation of the previous `last - 1`
  partial sums from it (the "variation across the last three orders");
* screening parameter: the value whose last three partial sums vary least
  (the fastest apparent convergence); the systematic uncertainty is the
  largest three-order variation among it and its neighbours in the scan;
* temperature: y(T) = y(0) (1 + alpha T/T_F) fitted by weighted least
  squares in T/T_F; y(0), alpha, their errors and chi^2 per degree of
  freedom are returned;
* iterations: independent estimates of one integral (VEGAS iterations, each
  on its own grid) are combined with inverse-variance weights, with chi^2
  per degree of freedom as the consistency check (Lepage 1978).
"""
import math

import numpy as np

from . import api


def _flatten(N, sigma, dsigma):
    keys_s = sorted(sigma)
    keys_d = sorted(dsigma)
    x = []
    for k in keys_s:
        x += [complex(sigma[k]).real, complex(sigma[k]).imag]
    for k in keys_d:
        x.append(complex(dsigma[k]).real)
    return np.array(x), keys_s, keys_d


def _unflatten(x, keys_s, keys_d):
    sigma, dsigma = {}, {}
    for i, k in enumerate(keys_s):
        sigma[k] = complex(x[2 * i], x[2 * i + 1])
    off = 2 * len(keys_s)
    for i, k in enumerate(keys_d):
        dsigma[k] = complex(x[off + i], 0.0)
    return sigma, dsigma


def meff_with_errors(N, sigma, sigma_err, dsigma, dsigma_err, kF, beta, Lam):
    """(partial sums meff [N+1], their statistical errors [N+1]).

    sigma, dsigma: {(n, m, l): complex estimate}; sigma_err: {(n, m, l):
    complex (error of Re, error of Im)}; dsigma_err: {(n, m, l): error of
    Re}.  Errors are propagated linearly through the post-process."""
    x, ks, kd = _flatten(N, sigma, dsigma)
    err = []
    for k in ks:
        e = complex(sigma_err.get(k, 0.0))
        err += [e.real, e.imag]
    for k in kd:
        err.append(float(complex(dsigma_err.get(k, 0.0)).real))
    err = np.array(err)

    def f(v):
        s, d = _unflatten(v, ks, kd)
        return api.postprocess(N, s, d, kF, beta, Lam)["meff"]
    base = f(x)
    var = np.zeros(N + 1)
    for i in range(x.size):
        if err[i] == 0.0:
            continue
        h = 1e-4 * (abs(x[i]) + err[i])          # the post-process is a polynomial in its inputs
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        var += ((f(xp) - f(xm)) / (2 * h) * err[i]) ** 2
    return base, np.sqrt(var)


def truncation_estimate(partial_sums, last=3):
    """(estimate, systematic uncertainty): the highest-order partial sum and
    the largest deviation of the previous last - 1 partial sums from it."""
    p = np.asarray(partial_sums, dtype=float)
    if p.size < last:
        raise ValueError("need at least %d orders" % last)
    tail = p[-last:]
    return float(p[-1]), float(np.max(np.abs(tail - p[-1])))


def choose_screening(scan, last=3):
    """scan: {Lambda: partial sums}.  Returns (Lambda*, estimate, systematic):
    Lambda* the value whose last `last` partial sums vary least; the
    systematic uncertainty the largest such variation among Lambda* and its
    neighbours in the scan."""
    lams = sorted(scan)
    spread = [float(np.ptp(np.asarray(scan[L], dtype=float)[-last:])) for L in lams]
    i = int(np.argmin(spread))
    est, _ = truncation_estimate(scan[lams[i]], last)
    near = [lams[j] for j in (i - 1, i, i + 1) if 0 <= j < len(lams)]
    sys = max(truncation_estimate(scan[L], last)[1] for L in near)
    return lams[i], est, sys


def extrapolate_linear_T(t, y, dy):
    """Weighted least squares y = y0 (1 + alpha t) over t = T/T_F.  Returns a
    dict with y0, dy0, alpha, dalpha, the covariance of (y0, slope) and
    chi2 per degree of freedom (nan with two points)."""
    t = np.asarray(t, dtype=float)
    y = np.asarray(y, dtype=float)
    w = 1.0 / np.asarray(dy, dtype=float) ** 2
    S, St, Stt = w.sum(), (w * t).sum(), (w * t * t).sum()
    Sy, Sty = (w * y).sum(), (w * t * y).sum()
    det = S * Stt - St * St
    if det <= 0:
        raise ValueError("need at least two distinct temperatures")
    c0 = (Stt * Sy - St * Sty) / det
    c1 = (S * Sty - St * Sy) / det
    cov = np.array([[Stt, -St], [-St, S]]) / det
    resid = y - (c0 + c1 * t)
    dof = t.size - 2
    chi2 = float((w * resid ** 2).sum() / dof) if dof > 0 else math.nan
    alpha = c1 / c0
    # alpha = c1 / c0: linear propagation with the covariance
    ga = np.array([-c1 / c0 ** 2, 1.0 / c0])
    dalpha = math.sqrt(float(ga @ cov @ ga))
    return {"y0": float(c0), "dy0": math.sqrt(cov[0, 0]), "alpha": float(alpha), "dalpha": dalpha,
            "slope": float(c1), "cov": cov, "chi2_dof": chi2}


def combine_iterations(means, variances):
    """Inverse-variance weighted combination of K independent estimates.

    means, variances: arrays [K, ...] (iterations first; the variance of each
    estimate, > 0).  Returns (mean, variance, chi2_per_dof) with
    mean = sum(I_k / s_k^2) / sum(1 / s_k^2), variance = 1 / sum(1 / s_k^2) and
    chi2_per_dof = sum((I_k - mean)^2 / s_k^2) / (K - 1) (NaN for K = 1), each
    of the shape of one estimate.
    """
    m = np.asarray(means, dtype=np.float64)
    v = np.asarray(variances, dtype=np.float64)
    if m.shape != v.shape or m.shape[0] < 1:
        raise ValueError("means and variances need the same shape, iterations first")
    if not np.all(v > 0.0):
        raise ValueError("every variance must be positive")
    w = 1.0 / v
    wsum = w.sum(axis=0)
    mean = (w * m).sum(axis=0) / wsum
    K = m.shape[0]
    chi2 = ((m - mean) ** 2 * w).sum(axis=0) / (K - 1) if K > 1 else np.full(mean.shape, np.nan)
    return mean, 1.0 / wsum, chi2
