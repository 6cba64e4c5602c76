"""NF-MCMC / VEGAS-MCMC (Sec. V, Eqs. target_distr and nf_mcmc_estimator) on
the GPU: the chain kernel takes the oracle's decisions on the same proposal
weights and uniforms (ragged chain count, several weight rows, two calls in a
row; the oracle reports near ties, where reordered arithmetic may decide
otherwise) and its sums and estimates agree to rounding, and the whole path (proposals from the VEGAS map or the
flow, integrand weights, chains, estimator) recovers the Fock self-energy's
closed form."""
import math

import numpy as np
import pytest

import workloads
from oracle import conventions, mcmc as omcmc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_2403_18840_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def _weights(seed, n_out, n):
    """Signed heavy-tailed FP32 weights, some exactly zero (points outside the cutoff)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_cauchy((n_out, n)) * rng.choice([1e-3, 1.0, 30.0], size=(n_out, n))
    w[:, rng.random(n) < 0.05] = 0.0
    return w.astype(np.float32)


def _agree(sums, state, rs, rst, ties, n_out):
    """Every chain without a near tie took the oracle's decisions: the same
    accepted count and final state; its sums of f/pi and q/pi agree to rounding
    (the kernel tests u g_t < g' and multiplies by 1/g)."""
    ok = ~ties
    assert ok.mean() >= 0.999
    acc, racc = sums[n_out + 1], rs[n_out + 1]
    assert np.array_equal(acc[ok], racc[ok])
    assert np.array_equal(state[:n_out, ok], rst[:n_out, ok])
    assert np.allclose(state[n_out, ok], rst[n_out, ok], rtol=1e-15, atol=0)
    scale = np.abs(rs[:n_out + 1, ok]).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(sums[:n_out + 1, ok] - rs[:n_out + 1, ok]) / scale) <= 1e-12
    return float(np.mean(acc == racc))


def test_chains_match_oracle(api):
    C, S, n_out, n_sel, alpha = 3000, 37, 4, 2, 0.35
    w1, w2 = _weights(1, n_out, C * S), _weights(2, n_out, C * S)
    ch = api.Chains(n_out, C, n_sel=n_sel, alpha=alpha)
    ch.run(torch.tensor(w1, device="cuda"), S, 17, 0, n_therm=5)
    sums1, st1 = ch.sums.cpu().numpy(), ch.state.cpu().numpy()
    out2 = ch.run(torch.tensor(w2, device="cuda"), S, 17, 1).cpu().numpy()
    sums2, st2 = ch.sums.cpu().numpy(), ch.state.cpu().numpy()
    ties = np.zeros(C, dtype=bool)
    rs1, rst1 = omcmc.run_chains(w1, n_sel, alpha, C, S, 17, 0, n_therm=5, near_ties=ties)
    m1 = _agree(sums1, st1, rs1, rst1, ties, n_out)
    rs2, rst2 = omcmc.run_chains(w2, n_sel, alpha, C, S, 17, 1, state=rst1, near_ties=ties)
    m2 = _agree(sums2, st2, rs2, rst2, ties, n_out)
    print("chains with the oracle's decisions: %.5f, %.5f (near ties: %d)" % (m1, m2, int(ties.sum())))
    I, var = omcmc.estimate(rs2, n_out)
    assert np.allclose(out2[:n_out, 0], I, rtol=1e-12, atol=0)
    assert np.allclose(out2[:n_out, 1], var, rtol=1e-10, atol=0)
    assert out2[n_out, 0] == rs2[n_out + 1].sum() / (C * S)
    assert 0.05 < out2[n_out, 0] < 0.95


def test_alpha_one_is_importance_sampling(api):
    C, S = 1000, 8
    w = _weights(3, 2, C * S)
    ch = api.Chains(2, C, n_sel=1, alpha=1.0)
    out = ch.run(torch.tensor(w, device="cuda"), S, 1, 0).cpu().numpy()
    assert out[2, 0] == 1.0
    assert np.allclose(out[:2, 0], w.astype(np.float64).mean(axis=1), rtol=1e-12)


@pytest.mark.parametrize("kw", [dict(alpha=0.0), dict(alpha=1.5), dict(n_out=33), dict(n_sel=3)])
def test_invalid_arguments_are_rejected(api, kw):
    a = dict(n_out=2, n_sel=1, alpha=0.5)
    a.update(kw)
    ch = api.Chains(a["n_out"], 64, n_sel=a["n_sel"], alpha=a["alpha"])
    w = torch.zeros((a["n_out"], 64 * 2), dtype=torch.float32, device="cuda")
    with pytest.raises(api.L.FdError):
        ch.run(w, 2, 0, 0)
    with pytest.raises(api.L.FdError):                       # too few columns for chains x steps
        api.Chains(2, 64).run(torch.zeros((2, 64), dtype=torch.float32, device="cuda"), 2, 0, 0)


def _fock_quad(P, k):
    from scipy import integrate
    from scipy.special import expit
    f = lambda q: q * expit(-P.beta * (q * q - P.mu)) * math.log(((k + q) ** 2 + P.Lambda) / ((k - q) ** 2 + P.Lambda))
    v, _ = integrate.quad(f, 0, P.kc, limit=500, epsabs=1e-14, epsrel=1e-13, points=[P.kF, k])
    return -v / (math.pi * k)


@pytest.mark.parametrize("sampler", ["vegas", "flow", "spline"])
def test_mcmc_recovers_the_fock_closed_form(api, sampler):
    from paper_2403_18840_gb300 import driver
    cfg = workloads.FOCK_ORDER1
    G = api.Graph(1)
    p = api.ueg_params(1, cfg["rs"], cfg["T_over_TF"], cfg["lam_over_kF"], 1.0)
    V = api.Vegas(G.dim, 256)
    driver.adapt_vegas(G, p, V, 1 << 18, 6, seed=3)
    flow = None                                              # untrained flows: any q is valid
    if sampler == "flow":
        flow = api.Flow(G.dim, n_layers=4, hidden=128, seed=5)
    elif sampler == "spline":
        flow = api.SplineFlow(G.dim, 4)
        flow.set_params(workloads.small_params(5, flow.n_params))
    C, S = 1 << 15, 32
    ch, plan, out = driver.mcmc(G, p, V, flow, C, S, 0.5, seed=9, it=100, n_therm=4)
    out = out.cpu().numpy()
    P = conventions.ueg_params(cfg["rs"], cfg["T_over_TF"], cfg["lam_over_kF"], 1.0)
    ref = _fock_quad(P, P.kext)
    print(sampler, "MCMC Fock", out[0], "ref", ref, "accepted", out[2, 0])
    # six estimates over the three samplers and two calls: 3.5 sigma each keeps the
    # two-sided 3-sigma p-value 0.0027 overall (measured |z| 0.44 - 0.97 on the first calls)
    assert abs(out[0, 0] - ref) < 3.5 * math.sqrt(out[0, 1]), (out[0], ref)
    assert out[1, 0] == 0.0                                  # the Fock self-energy is static: Im = 0
    assert 0.02 < out[2, 0] <= 1.0
    # continuing the same chains: a second call, estimate again consistent
    _, _, out2 = driver.mcmc(G, p, V, flow, C, S, 0.5, seed=9, it=101, chains=ch, plan=plan)
    out2 = out2.cpu().numpy()
    print(sampler, "MCMC Fock, continued", out2[0], "ref", ref)
    assert abs(out2[0, 0] - ref) < 3.5 * math.sqrt(out2[0, 1]), (out2[0], ref)


def test_long_chains_agree_with_importance_sampling_order3(api):
    # the sampler comparison's bias check: at order 3 the VEGAS-MCMC estimate
    # of long chains (2^12 x 2^12, one call thermalising) against 2^30 samples
    # of VEGAS importance sampling on the same frozen grid (short chains,
    # 2^16 x 256, missed this reference by ~7 of their error bars)
    from paper_2403_18840_gb300 import driver
    order = 3
    G = api.Graph(order, roots=[(order, 0, 0, 0)], budget=8192)
    G.jit()
    p = api.ueg_params(order, 1.0, 1.0 / 32.0, 1.0, 1.0)
    V = api.Vegas(G.dim, 1024)
    driver.adapt_vegas(G, p, V, 1 << 22, 12, seed=41)
    plan = api.EvalPlan([G], [p], [0], 1 << 22, maps=[V])
    means = np.array([plan.run(500, k)[0, 0, 0, 0].item() for k in range(256)])
    ref, ref_err = means.mean(), means.std(ddof=1) / math.sqrt(means.size)
    C = S = 1 << 12
    ch, plan2, _ = driver.mcmc(G, p, V, None, C, S, 0.5, seed=7, it=600, n_therm=S)
    _, _, out = driver.mcmc(G, p, V, None, C, S, 0.5, seed=7, it=601, chains=ch, plan=plan2)
    out = out.cpu().numpy()
    print("order 3: VEGAS IS %.6f +- %.6f, VEGAS-MCMC %.6f +- %.6f" % (ref, ref_err, out[0, 0], math.sqrt(out[0, 1])))
    assert abs(out[0, 0] - ref) < 3.0 * math.sqrt(out[0, 1] + ref_err ** 2)   # measured 1.2 sigma
