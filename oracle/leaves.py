"""Bare propagator and interaction leaves with their derivatives (oracle).

G0 (Eq. propagator, standard Matsubara sign): for tau in (-beta, beta),
    tau > 0 :  G0(eps, tau) = -exp(-eps tau) (1 - f(eps))
    tau <= 0:  G0(eps, tau) = +exp(-eps tau) f(eps)        (tau = 0 means 0^-)
with f(eps) = 1 / (exp(beta eps) + 1) and eps = k^2 - mu.

Chemical-potential counterterm leaves (Eq. green_ct, re-expansion of g(mu)):
d^m G0 / d mu^m = (-1)^m d^m G0 / d eps^m, expanded by Leibniz over
exp(-eps tau) and the Fermi factor; the j-th derivative of the logistic
function s(x) = 1/(1+exp(-x)) is P_j(s) with P_0 = s, P_{j+1} = P_j'(s) s (1-s).

Interaction counterterm leaves (Eq. interaction_ct, V_q = 8 pi / (q^2 + Lambda)):
d^l V / d Lambda^l = 8 pi (-1)^l l! / (q^2 + Lambda)^(l+1).

Pinned in tests/test_oracle_leaves.py against mpmath high-precision numerical
derivatives of the undifferentiated definitions.
"""
import math

import numpy as np

_R_CACHE = {}


def logistic_derivative_terms(j):
    """For i <= j: d^i s / dx^i = s * sum_(a,b) coef * s^a (1-s)^b for the logistic s.

    Polynomials are kept in the two variables s and c = 1 - s (ds/dx = s c,
    dc/dx = -s c), so that both limits s -> 0 and s -> 1 are evaluated
    without cancellation.
    """
    if j in _R_CACHE:
        return _R_CACHE[j]
    P = [{(1, 0): 1}]
    for _ in range(j):
        nxt = {}
        for (a, b), c in P[-1].items():
            if a:
                nxt[(a, b + 1)] = nxt.get((a, b + 1), 0) + a * c
            if b:
                nxt[(a + 1, b)] = nxt.get((a + 1, b), 0) - b * c
        P.append({k: v for k, v in nxt.items() if v != 0})
    R = [{(a - 1, b): c for (a, b), c in p.items()} for p in P]
    _R_CACHE[j] = R
    return R


def _eval_terms(terms, s, c):
    out = 0.0
    for (a, b), coef in terms.items():
        out = out + coef * s ** a * c ** b
    return out


def G0_deriv(eps, tau, beta, m):
    """d^m G0(eps, tau) / d mu^m in FP64 (arrays broadcast; tau == 0 is 0^-).

    Evaluated as sign * exp(-eps tau*) * phi(eps) with the Fermi factor phi that
    is >= 1/2 (phi = 1 - f for eps >= 0, phi = f for eps < 0) and tau* the
    matching time (tau shifted by -/+beta using f e^(beta eps) = 1 - f), so that
    the exponent is never positive and the Leibniz sum does not cancel.
    """
    eps = np.asarray(eps, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    eps, tau = np.broadcast_arrays(eps, tau)
    pos = tau > 0
    occ = eps < 0
    # tau*: eps >= 0 -> tau mod beta in (0, beta];  eps < 0 -> in (-beta, 0]
    tstar = np.where(occ, np.where(pos, tau - beta, tau), np.where(pos, tau, tau + beta))
    x = np.where(occ, -beta * eps, beta * eps)           # phi = s(x), x >= 0
    log_s = -np.logaddexp(0.0, -x)
    s = np.exp(log_s)
    c = np.exp(-np.logaddexp(0.0, x))                    # 1 - s without cancellation
    base = np.exp(-eps * tstar + log_s)
    dxde = np.where(occ, -beta, beta)
    R = logistic_derivative_terms(m)
    total = np.zeros(eps.shape)
    for i in range(m + 1):
        total = total + math.comb(m, i) * (-tstar) ** (m - i) * dxde ** i * _eval_terms(R[i], s, c)
    sign = np.where(pos, -1.0, 1.0)
    return (-1.0) ** m * sign * base * total


def V_deriv(q2, Lam, l):
    """d^l V / d Lambda^l with V = 8 pi / (q^2 + Lambda)."""
    q2 = np.asarray(q2, dtype=np.float64)
    return 8.0 * math.pi * (-1.0) ** l * math.factorial(l) / (q2 + Lam) ** (l + 1)
