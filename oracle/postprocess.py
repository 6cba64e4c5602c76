"""Renormalization post-processing and the effective mass (oracle, FP64).

Sec. VI.A: the self-energy is a triple series (Eq. sigma_xi_dmu_dlambda)
Sigma = sum xi^n dmu^m/m! dlam^l/l! Sigma^(n,m,l) with dlam = -xi Lambda
(Eq. interaction_ct, bare interaction at Lambda = 0) and dmu = sum_{i>=1} xi^i dmu_i
(Sec. III.B).  Reading of the garbled condition (Eq. counterterm): the Fermi
surface stays at k_F, i.e. dmu(xi) = Re Sigma(xi)|_(k_F, i omega_0) order by
order in xi; the xi^N coefficient involves only dmu_i with i < N.
a(xi), b(xi) re-expand the same way (Eqs. dsigma_depsilon_series,
deltam_partitions, deltas_partitions) with
  a^(n,m,l) = (1 / (2 k_F)) d Re Sigma^(n,m,l)(k, i w0) / dk at k_F   (m = 1/2),
  b^(n,m,l) = Im Sigma^(n,m,l)(k_F, i w0) / w0,   w0 = pi / beta,
and m*/m = (1 - b) / (1 + a) expanded as a power series in xi and summed to
xi^N (Eq. eff_mass_ratio with Z = 1 / (1 - b)).

Pinned: at order 1 the result reduces to the Hartree-Fock mass
1 / (1 + Sigma_x'(k_F) / (2 k_F)) truncated at first order (tests), and the
series algebra is checked against direct substitution at small xi.
"""
import math

import numpy as np


def _mul(a, b, N):
    out = np.zeros(N + 1)
    for i in range(N + 1):
        for j in range(N + 1 - i):
            out[i + j] += a[i] * b[j]
    return out


def _pow(a, m, N):
    out = np.zeros(N + 1)
    out[0] = 1.0
    for _ in range(m):
        out = _mul(out, a, N)
    return out


def _substitute(coef, dmu, Lam, N):
    """sum_{n,m,l} xi^(n+l) dmu(xi)^m/m! (-Lam)^l/l! coef[(n,m,l)] as a xi-series."""
    out = np.zeros(N + 1)
    for (n, m, l), c in coef.items():
        if n + l > N:
            continue
        sh = np.zeros(N + 1)
        sh[n + l] = c * (-Lam) ** l / math.factorial(l) / math.factorial(m)
        out += _mul(sh, _pow(dmu, m, N), N)
    return out


def renormalize(sigma, dsigma_dk, kF, beta, Lam, N):
    """sigma, dsigma_dk: dict (n,m,l) -> complex estimate at (k_F, i w0).

    Returns dict with dmu [N+1], a [N+1], b [N+1] (xi-series coefficients),
    meff [N+1] (partial sums of the xi-series of (1-b)/(1+a), index = order)
    and meff_ratio [N+1] ((1 - sum b) / (1 + sum a) of the truncated sums).
    """
    w0 = math.pi / beta
    re = {k: complex(v).real for k, v in sigma.items()}
    dmu = np.zeros(N + 1)
    for order in range(1, N + 1):
        s = _substitute(re, dmu, Lam, order)
        dmu[order] = s[order]
    acoef = {k: complex(v).real / (2.0 * kF) for k, v in dsigma_dk.items()}
    bcoef = {k: complex(v).imag / w0 for k, v in sigma.items()}
    a = _substitute(acoef, dmu, Lam, N)
    b = _substitute(bcoef, dmu, Lam, N)
    # (1 - b) / (1 + a) as a series: c (1 + a) = 1 - b
    onea = a.copy()
    onea[0] += 1.0
    oneb = -b
    oneb[0] += 1.0
    c = np.zeros(N + 1)
    for i in range(N + 1):
        c[i] = (oneb[i] - sum(c[j] * onea[i - j] for j in range(i))) / onea[0]
    meff = np.cumsum(c)
    ratio = np.array([(1.0 - b[:i + 1].sum()) / (1.0 + a[:i + 1].sum()) for i in range(N + 1)])
    return {"dmu": dmu, "a": a, "b": b, "meff": meff, "meff_ratio": ratio}
