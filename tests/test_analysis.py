"""Host analysis of the effective-mass series (App. B): error propagation
through the post-process (closed form at order 1, Monte Carlo resampling at
order 3), the three-order truncation estimate, the screening-parameter
choice, and the weighted linear-T extrapolation (exact lines, the textbook
least-squares errors, and coverage on seeded noisy data)."""
import math

import numpy as np
import pytest

from paper_2403_18840_gb300 import analysis as A
from paper_2403_18840_gb300 import api


def test_order_one_errors_closed_form():
    kF, beta, Lam = 1.9, 6.8, 0.9
    s = {(1, 0, 0): complex(-0.63, 0.11)}
    ds = {(1, 0, 0): complex(0.377, 0.0)}
    se = {(1, 0, 0): complex(0.01, 0.004)}
    dse = {(1, 0, 0): 0.02}
    m, dm = A.meff_with_errors(1, s, se, ds, dse, kF, beta, Lam)
    w0 = math.pi / beta
    assert math.isclose(m[1], 1 - 0.377 / (2 * kF) - 0.11 / w0, rel_tol=1e-12)
    want = math.hypot(0.02 / (2 * kF), 0.004 / w0)
    assert math.isclose(dm[1], want, rel_tol=1e-6)
    assert dm[0] == 0.0


def _toy_inputs(N, seed):
    rng = np.random.default_rng(seed)
    sig, dsig, se, dse = {}, {}, {}, {}
    for n in range(1, N + 1):
        for m in range(N - n + 1):
            for l in range(N - n - m + 1):
                sig[(n, m, l)] = complex(rng.normal(0, 0.5), rng.normal(0, 0.1))
                dsig[(n, m, l)] = complex(rng.normal(0, 0.3), 0.0)
                se[(n, m, l)] = complex(0.01 * abs(sig[(n, m, l)].real) + 1e-3, 0.01 * abs(sig[(n, m, l)].imag) + 1e-3)
                dse[(n, m, l)] = 0.01 * abs(dsig[(n, m, l)].real) + 1e-3
    return sig, dsig, se, dse


def test_error_propagation_matches_resampling():
    N, kF, beta, Lam = 3, 1.3, 5.0, 0.7
    sig, dsig, se, dse = _toy_inputs(N, 3)
    m, dm = A.meff_with_errors(N, sig, se, dsig, dse, kF, beta, Lam)
    rng = np.random.default_rng(4)
    draws = []
    for _ in range(3000):
        s = {k: complex(v.real + rng.normal() * se[k].real, v.imag + rng.normal() * se[k].imag) for k, v in sig.items()}
        d = {k: complex(v.real + rng.normal() * dse[k], 0.0) for k, v in dsig.items()}
        draws.append(api.postprocess(N, s, d, kF, beta, Lam)["meff"])
    sd = np.std(np.array(draws), axis=0)
    # 3000 draws: the sample standard deviation is within ~4 % (3 sigma ~ 4 %)
    assert np.allclose(dm[1:], sd[1:], rtol=0.08)


def test_truncation_estimate():
    est, sys = A.truncation_estimate([1.0, 0.9, 0.95, 0.97, 0.975, 0.979])
    assert est == 0.979 and math.isclose(sys, 0.009)
    with pytest.raises(ValueError):
        A.truncation_estimate([1.0, 0.9])


def test_choose_screening_prefers_fast_convergence():
    # partial sums converging to 0.98 with ratios r(Lambda): fastest at 1.5
    scan = {}
    for L, r in ((1.0, 0.6), (1.25, 0.4), (1.5, 0.1), (1.75, 0.3), (2.0, 0.5)):
        scan[L] = [0.98 + 0.1 * r ** k for k in range(7)]
    L, est, sys = A.choose_screening(scan)
    assert L == 1.5
    assert math.isclose(est, 0.98 + 0.1 * 0.1 ** 6)
    # the neighbours' three-order variation (ratio 0.4 at 1.25) sets the uncertainty
    assert math.isclose(sys, 0.1 * (0.4 ** 4 - 0.4 ** 6))


def test_extrapolation_exact_line_and_textbook_errors():
    t = np.array([1 / 40, 1 / 30, 1 / 20, 1 / 10])
    y = 0.98 * (1 + 0.3 * t)
    r = A.extrapolate_linear_T(t, y, np.full(4, 1e-3))
    assert math.isclose(r["y0"], 0.98, rel_tol=1e-12) and math.isclose(r["alpha"], 0.3, rel_tol=1e-10)
    assert r["chi2_dof"] < 1e-20
    # equal weights: var(intercept) = s^2 sum t^2 / (n sum t^2 - (sum t)^2)
    n = t.size
    want = 1e-3 * math.sqrt((t * t).sum() / (n * (t * t).sum() - t.sum() ** 2))
    assert math.isclose(r["dy0"], want, rel_tol=1e-12)


def test_extrapolation_coverage_on_noisy_data():
    rng = np.random.default_rng(9)
    t = np.linspace(0.02, 0.1, 6)
    dy = np.full(t.size, 2e-3)
    pulls = []
    for _ in range(400):
        y = 0.95 * (1 - 0.5 * t) + rng.normal(0, 2e-3, t.size)
        r = A.extrapolate_linear_T(t, y, dy)
        pulls.append((r["y0"] - 0.95) / r["dy0"])
    pulls = np.array(pulls)
    assert abs(pulls.mean()) < 0.2 and 0.85 < pulls.std() < 1.15


def test_combine_iterations():
    # hand example: weights 1 and 1/4
    m, v, c = A.combine_iterations([1.0, 2.0], [1.0, 4.0])
    assert abs(m - 1.2) < 1e-15 and abs(v - 0.8) < 1e-15 and abs(c - 0.2) < 1e-15
    # equal variances: the plain mean, s^2 / K, and chi^2 = sample variance / s^2
    x = np.array([0.3, -0.1, 0.7, 0.2])
    m, v, c = A.combine_iterations(x, np.full(4, 0.5))
    assert abs(m - x.mean()) < 1e-15 and abs(v - 0.5 / 4) < 1e-15
    assert abs(c - x.var(ddof=1) / 0.5) < 1e-14
    # independent draws with different errors around one value: unbiased,
    # unit pull scale and chi^2 per degree of freedom near 1
    rng = np.random.default_rng(4)
    sig = rng.uniform(0.5, 3.0, (200, 1000))
    draws = 2.0 + sig * rng.standard_normal(sig.shape)
    m, v, c = A.combine_iterations(draws, sig ** 2)
    pull = (m - 2.0) / np.sqrt(v)
    assert abs(pull.mean()) < 0.15 and abs(pull.std() - 1.0) < 0.08
    assert abs(c.mean() - 1.0) < 0.02
    with pytest.raises(ValueError):
        A.combine_iterations([1.0, 2.0], [1.0, 0.0])


def test_kish_fraction_matches_the_oracle():
    """The host side of the bench's Kish effective sample size fraction
    (driver.kish_fraction) against the oracle's Kish ESS divided by the
    sample count, on heavy-tailed signed weights and the degenerate cases."""
    import torch
    from oracle import integrand as oig
    from paper_2403_18840_gb300 import driver
    rng = np.random.default_rng(8)
    v = rng.standard_cauchy(50000) * rng.choice([-1.0, 1.0], 50000)
    assert driver.kish_fraction(torch.tensor(v, dtype=torch.float32)) == pytest.approx(
        oig.kish_ess(v.astype(np.float32)) / v.size, rel=1e-12)
    assert driver.kish_fraction(torch.full((64,), 2.5)) == pytest.approx(1.0, rel=1e-15)
    assert driver.kish_fraction(torch.zeros(16)) == 0.0


def test_production_protocol_recovers_a_known_model():
    """The App. B protocol (production_run.protocol) on synthetic partial sums
    with a known answer: m*/m(T) = m0 (1 + alpha T / T_F), partial sums
    S_N = m*/m(T) + c q(lambda)^N that converge fastest at lambda_best (the
    variation of the last three sums there well above the noise), and
    Gaussian noise of known size on every sum.  The protocol must pick
    lambda_best at every temperature and recover m0 and alpha within three
    of its own error bars."""
    from paper_2403_18840_gb300 import production_run as PR
    m0, alpha, lam_best, c = 0.955, 1.8, 1.375, 1.0
    lams, temps = [1.0, 1.25, 1.375, 1.5, 1.75], [1.0 / 40.0, 1.0 / 30.0, 1.0 / 25.0, 1.0 / 20.0]
    rng = np.random.default_rng(31)

    def runner(lam, T):
        q = 0.1 + abs(lam - lam_best)                 # the series' convergence ratio
        sig = np.array([1e-5, 2e-5, 5e-5, 1e-4, 2e-4, 4e-4])
        exact = m0 * (1.0 + alpha * T) + c * q ** np.arange(1, 7)
        return {"meff": exact + rng.normal(0.0, 1.0, 6) * sig, "meff_err": sig}

    res = PR.protocol(runner, lams, temps)
    assert [p["lam_over_kF"] for p in res["per_T"]] == [lam_best] * len(temps)
    T0 = res["T0"]
    assert abs(T0["meff_T0"] - m0) < 3.0 * T0["err_T0"], T0
    assert abs(T0["alpha"] - alpha) < 3.0 * T0["dalpha"], T0
    assert T0["err_T0"] < 2e-2
    # one temperature: a choice but no extrapolation
    one = PR.protocol(runner, lams, temps[:1])
    assert one["T0"] is None and one["per_T"][0]["lam_over_kF"] == lam_best
