"""Pin the oracle's integrand (map, leaves, diagrams, weighting) to closed forms,
1D/2D quadrature and finite differences."""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy import integrate
from scipy.special import expit

import workloads
from oracle import conventions, diagrams as dg, integrand as ig, philox
from oracle.leaves import G0_deriv

FOCK = workloads.FOCK_ORDER1


def _params(kext_over_kF, lam=0.5, T=0.04):
    return conventions.ueg_params(1.0, T, lam, kext_over_kF)


def fock_quad(P, k, dmu=0, dlam=0):
    """Sigma_x(k) = -(1/(pi k)) int_0^Kc q f(q^2-mu) ln(((k+q)^2+L)/((k-q)^2+L)) dq
    (angular integration of -int d^3q/(2pi)^3 V(k-q) f), with mu/Lambda derivatives."""
    b = P.beta

    def fder(e):
        f = expit(-b * e)
        if dmu == 0:
            return f
        if dmu == 1:      # d/dmu f(q^2 - mu) = beta f (1-f)
            return b * f * (1 - f)
        if dmu == 2:
            return b * b * f * (1 - f) * (1 - 2 * f)
        raise ValueError

    def logterm(q):
        A = (k + q) ** 2 + P.Lambda
        B = (k - q) ** 2 + P.Lambda
        if dlam == 0:
            return math.log(A / B)
        if dlam == 1:
            return 1 / A - 1 / B
        raise ValueError

    if k == 0.0:
        # removable singularity: ln(A/B)/k -> 4q/(q^2+L) (and its Lambda derivative)
        def f0(q):
            lt = 4 * q / (q * q + P.Lambda) if dlam == 0 else -4 * q / (q * q + P.Lambda) ** 2
            return q * fder(q * q - P.mu) * lt
        val, _ = integrate.quad(f0, 0, P.kc, limit=500, epsabs=1e-14, epsrel=1e-13, points=[P.kF])
        return -val / math.pi
    val, _ = integrate.quad(lambda q: q * fder(q * q - P.mu) * logterm(q), 0, P.kc, limit=500,
                            epsabs=1e-14, epsrel=1e-13, points=[P.kF, k])
    return -val / (math.pi * k)


def test_fock_quadrature_coulomb_limit():
    # T = 0, Lambda -> 0: Sigma_x = -(4 k_F / pi) [1/2 + (1-x^2)/(4x) ln|(1+x)/(1-x)|]
    P = conventions.ueg_params(1.0, 1e-5, 1e-7, 0.5)
    x = 0.5
    closed = -(4 * P.kF / math.pi) * (0.5 + (1 - x * x) / (4 * x) * math.log((1 + x) / (1 - x)))
    assert abs(fock_quad(P, 0.5 * P.kF) - closed) < 2e-6


def _mc(roots, P, n_samples, seed, dim):
    x = philox.uniforms(seed, 0, 0, np.arange(n_samples), dim)
    return ig.eval_roots(x, roots, P)


@pytest.mark.parametrize("j", [0, 2, 4, 7])
def test_fock_mc_vs_quadrature(j):
    kk = FOCK["kext_over_kF"][j]
    P = _params(kk)
    W = _mc([(1, 0, 0, 0)], P, 1 << 17, FOCK["seed"], 3)[0]
    assert np.all(W.imag == 0)
    m, v = ig.mean_var(W.real)
    ref = fock_quad(P, P.kext)
    assert abs(m - ref) < 3.0 * math.sqrt(v), (m, math.sqrt(v), ref)


@pytest.mark.parametrize("root,kw", [((1, 1, 0, 0), dict(dmu=1)), ((1, 0, 1, 0), dict(dlam=1)),
                                     ((1, 2, 0, 0), dict(dmu=2)), ((1, 1, 1, 0), dict(dmu=1, dlam=1))])
def test_fock_counterterm_roots_vs_quadrature(root, kw):
    P = _params(1.0)
    W = _mc([root], P, 1 << 17, 11, 3)[0]
    m, v = ig.mean_var(W.real)
    ref = fock_quad(P, P.kext, **kw)
    assert abs(m - ref) < 3.0 * math.sqrt(v), (m, math.sqrt(v), ref)


def test_fock_k_derivative_vs_quadrature():
    P = _params(1.0)
    W = _mc([(1, 0, 0, 1)], P, 1 << 17, 12, 3)[0]
    m, v = ig.mean_var(W.real)
    h = 1e-3
    k = P.kext
    ref = (8 * (fock_quad(P, k + h) - fock_quad(P, k - h))
           - (fock_quad(P, k + 2 * h) - fock_quad(P, k - 2 * h))) / (12 * h)
    assert abs(m - ref) < 3.0 * math.sqrt(v), (m, math.sqrt(v), ref)


def test_free_density():
    # n(mu) = 2 int d^3k/(2pi)^3 G0(k, 0^-) = -Li_{3/2}(-e^{beta mu}) / (4 pi^{3/2} beta^{3/2})
    P = _params(1.0)
    x = philox.uniforms(21, 0, 0, np.arange(1 << 17), 3)
    kvec, tau, jac = ig.map_hypercube(x, 1, P)
    eps = np.sum(kvec[1] ** 2, axis=0) - P.mu
    W = 2.0 * G0_deriv(eps, np.zeros_like(eps), P.beta, 0) * jac
    m, v = ig.mean_var(W)
    mp.mp.dps = 30
    ref = float(mp.re(-mp.polylog(1.5, -mp.exp(P.beta * P.mu)) / (4 * mp.pi ** 1.5 * mp.mpf(P.beta) ** 1.5)))
    assert abs(m - ref) < 3.0 * math.sqrt(v), (m, math.sqrt(v), ref)
    # the T -> 0 limit of the same formula is the r_s density 3 / (4 pi r_s^3)
    P0 = conventions.ueg_params(1.0, 1e-4, 0.5, 0.0)
    n0 = float(mp.re(-mp.polylog(1.5, -mp.exp(P0.beta * P0.mu)) / (4 * mp.pi ** 1.5 * mp.mpf(P0.beta) ** 1.5)))
    assert abs(n0 - 3 / (4 * math.pi)) < 1e-6


def test_static_lindhard_bubble():
    # Pi0(q) = 2 int d^3p/(2pi)^3 int_0^beta G0(p,tau) G0(p+q,-tau) dtau
    #        = -(1/(2 pi^2 q)) int_0^inf p f(p^2-mu) ln|(2p+q)/(2p-q)| dp
    P = _params(0.0)
    q = 0.7 * P.kF
    x = philox.uniforms(22, 0, 0, np.arange(1 << 17), 4)
    kvec, _, jac = ig.map_hypercube(x[:3], 1, P)
    p = kvec[1]
    tau = P.beta * x[3]
    e1 = np.sum(p * p, axis=0) - P.mu
    pq = p.copy()
    pq[2] += q
    e2 = np.sum(pq * pq, axis=0) - P.mu
    W = 2.0 * G0_deriv(e1, tau, P.beta, 0) * G0_deriv(e2, -tau, P.beta, 0) * jac * P.beta
    m, v = ig.mean_var(W)
    f = lambda pp: pp * expit(-P.beta * (pp * pp - P.mu)) * math.log(abs((2 * pp + q) / (2 * pp - q)))
    val, _ = integrate.quad(f, 0, P.kc, points=[q / 2, P.kF], limit=500, epsabs=1e-13)
    # second half of the cut: momenta p+q beyond Kc are kept by the integrand,
    # p itself is limited to Kc; the Fermi factor makes the difference negligible
    ref = -val / (2 * math.pi ** 2 * q)
    assert abs(m - ref) < 3.0 * math.sqrt(v), (m, math.sqrt(v), ref)


def test_rainbow_diagram_vs_2d_quadrature():
    # Fock self-energy inserted in the Fock line: Sigma_rb(k) = -int_q V(k-q) f'(eps_q) Sigma_x(q)
    P = _params(1.0)
    tops = dg.self_energy_topologies(2)
    rb = [dg.route(t) for t in tops if dg.route(t).out_vertex == 1 and t.F == 0]
    # the rainbow: open path 0 -> line1 -> line1 -> 1, outer interaction line joins in and out
    rb = [d for d in rb if tuple(d.g_tau[1]) == (1, 1)]
    assert len(rb) == 1
    d = rb[0]
    x = philox.uniforms(23, 0, 0, np.arange(1 << 17), 7)
    kvec, tau, jac = ig.map_hypercube(x, 2, P)
    W = ig.diagram_value(d, kvec, tau, P, 0, 0, 0) * jac
    m, v = ig.mean_var(W)
    b = P.beta
    qs = np.linspace(0, P.kc, 2001)
    sx = np.array([fock_quad(P, qq) if qq > 0 else fock_quad(P, 0.0) for qq in qs])

    def integrand(qq):
        fq = expit(-b * (qq * qq - P.mu))
        fprime = -b * fq * (1 - fq)
        s = np.interp(qq, qs, sx)
        k = P.kext
        return qq * fprime * s * math.log(((k + qq) ** 2 + P.Lambda) / ((k - qq) ** 2 + P.Lambda))
    val, _ = integrate.quad(integrand, 0, P.kc, points=[P.kF], limit=500)
    ref = -val / (math.pi * P.kext)   # -int V f' Sx with the Fock angular kernel
    assert abs(m - ref) < 3.0 * math.sqrt(v) + 1e-4 * abs(ref), (m, math.sqrt(v), ref)   # + the quadrature's tolerance


def test_second_order_quasiparticle_weight_below_one():
    # Z = 1/(1-b) < 1 needs Im Sigma^(2)(k_F, i w0) < 0
    P = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    W = _mc([(2, 0, 0, 0)], P, 1 << 16, 24, 7)[0]
    m, v = ig.mean_var(W.imag)
    assert m + 3 * math.sqrt(v) < 0


@pytest.mark.parametrize("n", [1, 2, 3])
def test_counterterm_roots_match_finite_differences(n):
    # counterterm derivatives equal finite differences in mu and Lambda
    P = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    x = workloads.uniform_points(31 + n, 4 * n - 1, 16)
    h = 1e-3

    def W(Pp, root):
        return ig.eval_roots(x, [root], Pp)[0]

    def rich(fun, h):
        return (8 * (fun(h) - fun(-h)) - (fun(2 * h) - fun(-2 * h))) / (12 * h)

    import dataclasses
    base = (n, 0, 0, 0)
    for root, shift in [((n, 1, 0, 0), "mu"), ((n, 0, 1, 0), "Lambda"), ((n, 0, 0, 1), "kext")]:
        got = W(P, root)
        fd = rich(lambda d: W(dataclasses.replace(P, **{shift: getattr(P, shift) + d}), base), h)
        scale = np.maximum(np.abs(got), 1e-3 * np.max(np.abs(got)))
        assert np.all(np.abs(got - fd) <= 1e-6 * scale), (root, np.max(np.abs(got - fd) / scale))
    # second mu derivative from the first
    got = W(P, (n, 2, 0, 0))
    fd = rich(lambda d: W(dataclasses.replace(P, mu=P.mu + d), (n, 1, 0, 0)), h)
    scale = np.maximum(np.abs(got), 1e-3 * np.max(np.abs(got)))
    assert np.all(np.abs(got - fd) <= 1e-6 * scale)


def test_kish_effective_sample_size():
    # N equal weights count fully, one nonzero weight counts once, signs do not matter
    assert ig.kish_ess(np.full(1000, 0.37)) == pytest.approx(1000.0, rel=1e-14)
    assert ig.kish_ess(np.r_[np.zeros(99), 5.0]) == pytest.approx(1.0, rel=1e-14)
    assert ig.kish_ess(np.tile([1.0, -1.0], 50)) == pytest.approx(100.0, rel=1e-14)
    assert ig.kish_ess(np.zeros(10)) == 0.0
    # two populations: (a n1 + b n2)^2 / (a^2 n1 + b^2 n2)
    a, b, n1, n2 = 1.0, 10.0, 900, 100
    v = np.r_[np.full(n1, a), np.full(n2, b)]
    assert ig.kish_ess(v) == pytest.approx((a * n1 + b * n2) ** 2 / (a * a * n1 + b * b * n2), rel=1e-14)
