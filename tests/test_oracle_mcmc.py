"""Pins of the MCMC oracle (Sec. V, Eqs. target_distr and nf_mcmc_estimator).

* alpha = 1: pi = q, every proposal is accepted and the estimator is the plain
  importance-sampling mean of the weights.
* A discrete toy (finite state set, proposal probabilities q_j): the
  distribution of the chains' states after k steps equals q P^(k-1), with the
  Metropolis-Hastings transition matrix P built here from its definition; the
  chains' stationary distribution is pi_j / sum pi.
* The estimator recovers integrals with a closed form (signed integrands), and
  its delta-method error bar matches the scatter over independent replicas.
"""
import numpy as np
import pytest

from oracle import mcmc, philox

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _discrete(seed, C, S, q, f):
    """Weights [1, C*S] of proposals drawn from the discrete q, and their state ids."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(q), size=C * S, p=q)
    return (f[idx] / q[idx])[None, :], idx


def _mh_matrix(q, f, alpha, inverted=False):
    """P[i, j]: independence MH transition probabilities written from the
    definition (inverted: the acceptance ratio turned upside down)."""
    g = alpha + (1 - alpha) * np.abs(f / q)
    m = len(q)
    P = np.zeros((m, m))
    for i in range(m):
        for j in range(m):
            if i != j:
                P[i, j] = q[j] * min(1.0, (g[i] / g[j]) if inverted else (g[j] / g[i]))
        P[i, i] = 1.0 - P[i].sum()
    return P


def test_uniform_stream_is_philox_with_the_tagged_counter():
    u = mcmc.chain_uniforms(9, 4, 5, 6)
    for c in range(5):
        for k in range(6):
            w = philox.philox4x32_10(c, 0, 4, mcmc.TAG | (k >> 2), 9, 0)[k & 3]
            assert u[k, c] == philox.words_to_uniform(w)
    assert np.all((u > 0) & (u < 1))


def test_alpha_one_is_importance_sampling():
    rng = np.random.default_rng(1)
    C, S = 64, 9
    w = rng.standard_cauchy((3, C * S)).astype(np.float32)
    sums, state = mcmc.run_chains(w, 2, 1.0, C, S, 5, 0)
    assert np.all(sums[4] == S)                                   # every proposal accepted
    assert np.array_equal(sums[3], np.full(C, float(S)))         # q/pi = 1
    wc = w.astype(np.float64).reshape(3, S, C)
    assert np.allclose(sums[:3], wc.sum(axis=1), rtol=1e-13, atol=0)
    I, _ = mcmc.estimate(sums, 3)
    assert np.allclose(I, w.astype(np.float64).mean(axis=1), rtol=1e-12)
    assert np.array_equal(state[:3], wc[:, -1, :])


@pytest.mark.parametrize("alpha", [0.2, 0.7])
def test_discrete_state_distribution_follows_the_mh_kernel(alpha):
    q = np.array([0.5, 0.3, 0.15, 0.05])
    f = np.array([0.05, -0.6, 0.9, 0.4])          # signed; |f| peaks where q is small
    C, S = 1 << 17, 4
    w, idx = _discrete(3, C, S, q, f)
    _, state = mcmc.run_chains(w, 1, alpha, C, S, 11, 2)
    wq = f / q
    final = np.array([np.flatnonzero(np.isclose(wq, x))[0] for x in state[0]])
    emp = np.bincount(final, minlength=4) / C
    exact = q @ np.linalg.matrix_power(_mh_matrix(q, f, alpha), S - 1)
    sig = np.sqrt(exact * (1 - exact) / C)
    assert np.all(np.abs(emp - exact) <= 5 * sig), (emp, exact)
    # the pin has the power to see a wrong rule: the inverted ratio's law is far off
    wrong = q @ np.linalg.matrix_power(_mh_matrix(q, f, alpha, inverted=True), S - 1)
    assert np.max(np.abs(emp - wrong) / sig) > 20


def test_discrete_stationary_law_and_estimator():
    q = np.array([0.5, 0.3, 0.15, 0.05])
    f = np.array([0.05, -0.6, 0.9, 0.4])
    alpha = 0.3
    C, S, therm = 1 << 14, 64, 16
    w, _ = _discrete(4, C, S, q, f)
    sums, state = mcmc.run_chains(w, 1, alpha, C, S, 12, 0, n_therm=therm)
    wq = f / q
    final = np.array([np.flatnonzero(np.isclose(wq, x))[0] for x in state[0]])
    pi = alpha * q + (1 - alpha) * np.abs(f)
    pi = pi / pi.sum()
    emp = np.bincount(final, minlength=4) / C
    # four states at once: 3.2 sigma each keeps the two-sided 3-sigma p-value 0.0027 overall
    assert np.all(np.abs(emp - pi) <= 3.2 * np.sqrt(pi * (1 - pi) / C))
    I, var = mcmc.estimate(sums, 1)
    assert abs(I[0] - f.sum()) <= 3 * np.sqrt(var[0]), (I, f.sum(), np.sqrt(var))


def test_continuous_closed_form_and_error_bar():
    # f(x) = sin(2 pi x) + 0.3 on (0, 1), q uniform: the integral is 0.3
    alpha, C, S = 0.3, 4096, 32
    est, errs = [], []
    for rep in range(24):
        rng = np.random.default_rng(100 + rep)
        x = rng.random(C * S)
        w = (np.sin(2 * np.pi * x) + 0.3)[None, :]
        sums, _ = mcmc.run_chains(w, 1, alpha, C, S, 7, rep, n_therm=4)
        I, var = mcmc.estimate(sums, 1)
        est.append(I[0])
        errs.append(np.sqrt(var[0]))
    est, errs = np.array(est), np.array(errs)
    # 24 replicas at once: 3.9 sigma each keeps the two-sided 3-sigma p-value 0.0027 overall
    assert np.all(np.abs(est - 0.3) <= 3.9 * errs)
    ratio = est.std(ddof=1) / errs.mean()          # the error bar describes the scatter
    assert 0.6 < ratio < 1.5, ratio


def test_continuing_chains_equals_one_long_call():
    rng = np.random.default_rng(2)
    C = 32
    w = rng.standard_normal((2, C * 10)).astype(np.float32)
    u_all = np.concatenate([mcmc.chain_uniforms(3, 0, C, 6), mcmc.chain_uniforms(3, 1, C, 4)])
    s1, st = mcmc.run_chains(w[:, :6 * C], 1, 0.4, C, 6, 3, 0)
    s2, st2 = mcmc.run_chains(w[:, 6 * C:], 1, 0.4, C, 4, 3, 1, state=st)
    # a reference loop with the concatenated uniforms
    cur, g = np.zeros((2, C)), np.zeros(C)
    A, B = np.zeros((2, C)), np.zeros(C)
    for k in range(10):
        wp = w[:, k * C:(k + 1) * C].astype(np.float64)
        gp = 0.4 + 0.6 * np.abs(wp[0])
        acc = np.array([g[c] == 0 or u_all[k, c] < gp[c] / g[c] for c in range(C)])
        cur[:, acc], g[acc] = wp[:, acc], gp[acc]
        A += cur / g
        B += 1 / g
    assert np.allclose(s1[:2] + s2[:2], A, rtol=1e-12) and np.allclose(s1[2] + s2[2], B, rtol=1e-12)
    assert np.array_equal(st2[2], g)


def test_alpha_must_be_positive():
    with pytest.raises(AssertionError):
        mcmc.run_chains(np.ones((1, 4)), 1, 0.0, 4, 1, 0, 0)
