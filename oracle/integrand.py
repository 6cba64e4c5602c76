"""Per-sample integrand roots Sigma^(n,m,l) of the self-energy (oracle).

What is computed (Eqs. sigma_integration and sigma_xi_dmu_dlambda, Sec. VI.A):
for a hypercube point x, external momentum k (along z) and root (n, m, l, dk),

  W(x) = sum_t  s_t * d^m_mu d^l_Lambda (d_k)^dk [ prod_G G0 prod_V V ] * J(x) * exp(i pi x_out)

summed over the order-n topologies t of ``diagrams``, with s_t = (-1)^(n+F) 2^F,
J the Jacobian of the map below and x_out the hypercube coordinate of the
out-vertex's time (omega_0 tau_out = pi x_out for the lowest Matsubara
frequency omega_0 = pi / beta; tau_out = 0 when the out-vertex sits on line 0).
The Monte Carlo average of W over uniform x estimates Sigma^(n,m,l)(k, i omega_0).
Derivatives are distributed over the lines by Leibniz' rule; the k-derivative
acts through eps_p and q^2 of lines that carry k_ext (d eps / dk = 2 c p_z).

Hypercube layout for order n (D = 4n - 1): k_1 <- x[0:3]; for j = 2..n:
k_j <- x[4j-5 : 4j-2] and the time of interaction line j-1 <- beta * x[4j-2].
Loop momentum from (a, b, c): r = K_c a, cos(theta) = 2b - 1, phi = 2 pi c,
d^3k / (2 pi)^3 = K_c r^2 / (2 pi^2) da db dc.  Roots with n below the graph's
order use the leading 4n - 1 coordinates.

Reduction: mean and variance of W over samples with exactly rounded sums
(math.fsum), and the Kish effective sample size of the weighted values.
"""
import itertools
import math

import numpy as np

from . import diagrams as dg
from .leaves import G0_deriv, V_deriv


def dim_of_order(n):
    return 4 * n - 1


def time_coord(line):
    """Hypercube coordinate holding the time of interaction line `line` >= 1."""
    return 4 * line + 2


def map_hypercube(x, n, P):
    """x [D>=4n-1, N] -> (kvec [n+1, 3, N] with kvec[0] = k_ext, tau [n, N], jac [N])."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[1]
    kvec = np.zeros((n + 1, 3, N))
    kvec[0, 2, :] = P.kext
    jac = np.ones(N)
    for j in range(1, n + 1):
        c0 = 0 if j == 1 else 4 * j - 5
        a, b, c = x[c0], x[c0 + 1], x[c0 + 2]
        r = P.kc * a
        cth = 2.0 * b - 1.0
        sth = 2.0 * np.sqrt(b * (1.0 - b))
        phi = 2.0 * math.pi * c
        kvec[j, 0] = r * sth * np.cos(phi)
        kvec[j, 1] = r * sth * np.sin(phi)
        kvec[j, 2] = r * cth
        jac = jac * P.kc * r * r / (2.0 * math.pi ** 2)
    tau = np.zeros((n, N))
    for i in range(1, n):
        tau[i] = P.beta * x[time_coord(i)]
        jac = jac * P.beta
    return kvec, tau, jac


def _compositions(total, parts):
    """All tuples of `parts` non-negative ints summing to `total`."""
    if parts == 0:
        if total == 0:
            yield ()
        return
    for c in itertools.combinations(range(total + parts - 1), parts - 1):
        prev = -1
        out = []
        for b in c:
            out.append(b - prev - 1)
            prev = b
        out.append(total + parts - 1 - prev - 1)
        yield tuple(out)


def _multinomial(total, parts):
    r = math.factorial(total)
    for p in parts:
        r //= math.factorial(p)
    return r


def diagram_value(d, kvec, tau, P, m, l, dk, return_abs=False):
    """d^m_mu d^l_Lambda d_k^dk of s_t prod G prod V for one routed diagram [N] (real)."""
    nG = 2 * d.n - 1
    nV = d.n
    # line momenta
    pG = np.einsum("ej,jcn->ecn", d.g_mom.astype(np.float64), kvec)
    pV = np.einsum("ej,jcn->ecn", d.v_mom.astype(np.float64), kvec)
    epsG = np.sum(pG * pG, axis=1) - P.mu
    q2V = np.sum(pV * pV, axis=1)
    tauG = tau[d.g_tau[:, 0]] - tau[d.g_tau[:, 1]]
    cG = d.g_mom[:, 0]
    cV = d.v_mom[:, 0]
    Gd = [[G0_deriv(epsG[e], tauG[e], P.beta, j) for j in range(m + dk + 1)] for e in range(nG)]
    Vd = [[V_deriv(q2V[v], P.Lambda, j) for j in range(l + dk + 1)] for v in range(nV)]
    total = 0.0
    l1 = 0.0
    for mg in _compositions(m, nG):
        cg = _multinomial(m, mg)
        for lv in _compositions(l, nV):
            cv = _multinomial(l, lv)
            if dk == 0:
                t = np.ones_like(epsG[0])
                for e in range(nG):
                    t = t * Gd[e][mg[e]]
                for v in range(nV):
                    t = t * Vd[v][lv[v]]
                total = total + cg * cv * t
                l1 = l1 + abs(cg * cv) * np.abs(t)
            else:
                for e in range(nG):
                    if cG[e] == 0:
                        continue
                    t = -2.0 * cG[e] * pG[e, 2] * Gd[e][mg[e] + 1]
                    for e2 in range(nG):
                        if e2 != e:
                            t = t * Gd[e2][mg[e2]]
                    for v in range(nV):
                        t = t * Vd[v][lv[v]]
                    total = total + cg * cv * t
                    l1 = l1 + abs(cg * cv) * np.abs(t)
                for v in range(nV):
                    if cV[v] == 0:
                        continue
                    t = 2.0 * cV[v] * pV[v, 2] * Vd[v][lv[v] + 1]
                    for e in range(nG):
                        t = t * Gd[e][mg[e]]
                    for v2 in range(nV):
                        if v2 != v:
                            t = t * Vd[v2][lv[v2]]
                    total = total + cg * cv * t
                    l1 = l1 + abs(cg * cv) * np.abs(t)
    if return_abs:
        return d.sign * total, l1
    return d.sign * total


def eval_roots(x, roots, P, with_l1=False):
    """Integrand roots at hypercube points x [D, N] -> complex [R, N] (and L1 magnitudes).

    roots: list of (n, m, l, dk).  Includes Jacobian and exp(i pi x_out).
    """
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[1]
    out = np.zeros((len(roots), N), dtype=np.complex128)
    mag = np.zeros((len(roots), N))
    by_n = {}
    for r, (n, m, l, dk) in enumerate(roots):
        if n not in by_n:
            by_n[n] = (dg.routed_self_energy(n), map_hypercube(x, n, P))
        diags, (kvec, tau, jac) = by_n[n]
        acc = np.zeros(N, dtype=np.complex128)
        acc_l1 = np.zeros(N)
        for d in diags:
            val, l1 = diagram_value(d, kvec, tau, P, m, l, dk, return_abs=True)
            out_line = d.out_vertex // 2
            if out_line == 0:
                phase = 1.0
            else:
                phase = np.exp(1j * math.pi * x[time_coord(out_line)])
            acc = acc + val * phase
            acc_l1 = acc_l1 + np.abs(d.sign) * l1
        out[r] = acc * jac
        mag[r] = acc_l1 * np.abs(jac)
    if with_l1:
        return out, mag
    return out


def graph_roots(order, with_dk=False):
    """Root list of an order-N graph: all (n, m, l) with n + m + l = N (this ordering)."""
    roots = []
    for dk in ((0, 1) if with_dk else (0,)):
        for n in range(order, 0, -1):
            for m in range(order - n + 1):
                roots.append((n, m, order - n - m, dk))
    return roots


def mean_var(values):
    """(mean, variance of the mean) of a real sample array with exactly rounded sums."""
    v = np.asarray(values, dtype=np.float64)
    N = v.size
    s1 = math.fsum(v.tolist())
    mean = s1 / N
    s2 = math.fsum(((v - mean) ** 2).tolist())
    var = s2 / (N - 1) / N if N > 1 else 0.0
    return mean, var


def kish_ess(values):
    """Kish effective sample size (sum |v|)^2 / sum v^2 of weighted values v
    (w f per sample), with exactly rounded sums; 0 when every value is 0."""
    v = np.abs(np.asarray(values, dtype=np.float64)).ravel()
    s2 = math.fsum((v * v).tolist())
    if s2 == 0.0:
        return 0.0
    s1 = math.fsum(v.tolist())
    return s1 * s1 / s2
