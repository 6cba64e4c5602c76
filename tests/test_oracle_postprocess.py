"""Pins for the renormalisation post-processing (Sec. VI.A; Eqs. counterterm,
sigma_xi_dmu_dlambda, eff_mass_ratio) against sympy series algebra."""
import math

import sympy as sp

from oracle import postprocess


def test_order_one_is_hartree_fock():
    kF, beta, Lam = 1.9, 6.8, 0.9
    s = {(1, 0, 0): complex(-0.63, 0.0)}
    ds = {(1, 0, 0): complex(0.377, 0.0)}
    r = postprocess.renormalize(s, ds, kF, beta, Lam, 1)
    a1 = 0.377 / (2 * kF)
    assert math.isclose(r["dmu"][1], -0.63)
    assert math.isclose(r["a"][1], a1)
    assert r["b"][1] == 0.0
    assert math.isclose(r["meff"][1], 1 - a1)
    assert math.isclose(r["meff_ratio"][1], 1 / (1 + a1))


def test_series_against_sympy():
    # toy self-energy with known mu and Lambda dependence:
    #   Sigma^(n)(mu, Lam) = c_n exp(g_n mu) / (1 + h_n Lam)   (complex c_n)
    # then Sigma^(n,m,l) are its derivatives at (mu_R, Lam_R); the exact
    # renormalised series follows from solving dmu = Re Sigma(xi; mu_R + dmu,
    # Lam_R - xi Lam_R) order by order with sympy.
    N = 4
    xi, d = sp.symbols("xi d")
    mu_R, L_R = sp.Rational(3, 2), sp.Rational(7, 10)
    cs = [None, (-0.6, 0.0), (-0.2, -0.05), (0.07, -0.02), (-0.03, 0.01)]
    gs = [None, 0.3, -0.5, 0.8, 0.2]
    hs = [None, 0.4, 0.1, -0.3, 0.6]
    dk = [None, 0.2, -0.1, 0.05, 0.03]       # d/dk factor per order (toy)
    mu, Lm = sp.symbols("mu Lm")
    funcs = {n: sp.exp(gs[n] * mu) / (1 + hs[n] * Lm) for n in range(1, N + 1)}
    sig, dsig = {}, {}
    for n in range(1, N + 1):
        for m in range(N - n + 1):
            for l in range(N - n - m + 1):
                der = sp.diff(funcs[n], mu, m, Lm, l).subs({mu: mu_R, Lm: L_R})
                val = float(der)
                sig[(n, m, l)] = complex(cs[n][0] * val, cs[n][1] * val)
                dsig[(n, m, l)] = complex(dk[n] * val, 0.0)
    kF, beta = 1.3, 5.0
    w0 = math.pi / beta
    r = postprocess.renormalize(sig, dsig, kF, beta, float(L_R), N)
    # sympy: dmu(xi) as a polynomial with unknown coefficients
    dm = sp.symbols("dm1:%d" % (N + 1))
    dmu = sum(dm[i] * xi ** (i + 1) for i in range(N))
    ReS = sum(xi ** n * cs[n][0] * funcs[n].subs({mu: mu_R + dmu, Lm: L_R - xi * L_R}) for n in range(1, N + 1))
    ser = sp.series(ReS - dmu, xi, 0, N + 1).removeO()
    sol = {}
    for k in range(1, N + 1):
        eq = sp.expand(ser.coeff(xi, k)).subs(sol)
        sol[dm[k - 1]] = sp.solve(eq, dm[k - 1])[0]
    for k in range(1, N + 1):
        assert abs(float(sol[dm[k - 1]]) - r["dmu"][k]) < 1e-10
    dmu_s = dmu.subs(sol)
    a = sum(xi ** n * dk[n] / (2 * kF) * funcs[n].subs({mu: mu_R + dmu_s, Lm: L_R - xi * L_R}) for n in range(1, N + 1))
    b = sum(xi ** n * cs[n][1] / w0 * funcs[n].subs({mu: mu_R + dmu_s, Lm: L_R - xi * L_R}) for n in range(1, N + 1))
    acoef = sp.expand(sp.series(a, xi, 0, N + 1).removeO())
    bcoef = sp.expand(sp.series(b, xi, 0, N + 1).removeO())
    meff = sp.expand(sp.series((1 - bcoef) / (1 + acoef), xi, 0, N + 1).removeO())
    for k in range(1, N + 1):
        assert abs(float(acoef.coeff(xi, k)) - r["a"][k]) < 1e-10
        partial = sum(float(meff.coeff(xi, j)) for j in range(k + 1))
        assert abs(partial - r["meff"][k]) < 1e-10
