"""Independence Metropolis-Hastings chains over importance-weighted proposals
(oracle; test infrastructure, never imported by the product path).

Sec. V (NF-MCMC) samples configurations from the target

    pi(x) = alpha q(x) + (1 - alpha) p(x),   p(x) = |f(x)|        (Eq. target_distr)

with proposals drawn from q independently of the chain's state, accepts a
proposal x with probability

    R = min{1, pi(x) q(x_t) / (pi(x_t) q(x))}                     (Metropolis-Hastings step)

and estimates the integral from the visited states x_i as

    I = sum_i f(x_i)/pi(x_i) / sum_i q(x_i)/pi(x_i).              (Eq. nf_mcmc_estimator)

All three depend on a configuration only through its importance weight
w = f(x)/q(x): with g = pi/q = alpha + (1 - alpha) |w|_p, R = g(x)/g(x_t),
f/pi = w/g and q/pi = 1/g.  Here w has n_out components (e.g. the real and
imaginary parts of several roots); |w|_p is the sum of the magnitudes of the
first n_sel components (the integrand whose magnitude the chain follows); the
estimator is applied to every component.  The paper's VEGAS-MCMC and NF-MCMC
differ only in q (the VEGAS map's density, or the flow's).

Reading where the paper is silent: alpha must be > 0 (with alpha = 0 a state
with f = 0 has pi = 0 and q/pi is undefined); a chain without a state accepts
its first proposal; every state after the first n_therm steps of a call is
measured (the error bar, from independent chains, includes the
autocorrelation).

Acceptance uniforms: Philox4x32-10 (oracle.philox) with counter
(chain_lo, chain_hi, iteration, TAG | (step >> 2)), word step & 3, key
(seed_lo, seed_hi), u = ((word >> 9) + 0.5) 2^-23: a stream disjoint from the
sample streams (whose last counter word is < 2^16).

The arithmetic is FP64 and follows the equations as written: a proposal is
accepted when u < R = g'/g_t, and the estimator sums f/pi = w/g and q/pi = 1/g.
An implementation may reorder this arithmetic (test u g_t < g', multiply by
1/g); it then takes the same decisions except where u lies within a few
rounding steps of g'/g_t (near_ties reports those steps), and its sums agree
to rounding.
"""
import numpy as np

from . import philox

TAG = 0x40000000


def chain_uniforms(seed, iteration, n_chains, n_steps):
    """Acceptance uniforms [n_steps, n_chains] (FP64, exact)."""
    c = np.arange(n_chains, dtype=np.uint64)
    lo, hi = c & np.uint64(0xFFFFFFFF), c >> np.uint64(32)
    k0, k1 = int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF
    out = np.empty((n_steps, n_chains))
    for b in range((n_steps + 3) // 4):
        words = philox.philox4x32_10(lo, hi, int(iteration) & 0xFFFFFFFF, TAG | b, k0, k1)
        for j in range(4):
            k = 4 * b + j
            if k < n_steps:
                out[k] = philox.words_to_uniform(words[j])
    return out


def g_of(w, n_sel, alpha):
    """pi/q = alpha + (1 - alpha) |w|_p for weights w [n_out, ...] (FP64)."""
    s = np.zeros(np.shape(w)[1:])
    for o in range(n_sel):
        s = s + np.abs(np.asarray(w[o], dtype=np.float64))
    return alpha + (1.0 - alpha) * s


def run_chains(w, n_sel, alpha, n_chains, n_steps, seed, iteration, n_therm=0, state=None, near_ties=None):
    """Advance n_chains chains by n_steps steps.

    w: proposal weights [n_out, n_chains * n_steps]; proposal k of chain c in
    column k * n_chains + c.  state: [n_out + 1, n_chains] (current weights, then
    g; g = 0: no state yet) or None.  Returns (sums, state): sums [n_out + 2,
    n_chains] holds, per chain, the sums over the measured steps of w_o/g and of
    1/g, then the number of accepted proposals.  near_ties: an optional boolean
    array [n_chains], set for chains with a step where u is within 8 rounding
    steps of g'/g_t (a decision that reordered arithmetic may take otherwise).
    """
    assert 0.0 < alpha <= 1.0
    w = np.asarray(w)
    n_out = w.shape[0]
    C = n_chains
    if state is None:
        state = np.zeros((n_out + 1, C))
    cur = np.array(state[:n_out], dtype=np.float64)
    g = np.array(state[n_out], dtype=np.float64)
    u = chain_uniforms(seed, iteration, C, n_steps)
    sums = np.zeros((n_out + 2, C))
    for k in range(n_steps):
        wp = w[:, k * C:(k + 1) * C].astype(np.float64)
        gp = g_of(wp, n_sel, alpha)
        # R = pi(x') q(x_t) / (pi(x_t) q(x')) = gp / g (g > 0 once the chain has a
        # state, since alpha > 0); a chain without a state accepts
        has = g > 0.0
        R = gp / np.where(has, g, 1.0)
        acc = ~has | (u[k] < R)
        if near_ties is not None:
            near_ties |= has & (np.abs(u[k] - R) <= 8.0 * np.finfo(np.float64).eps * np.maximum(R, u[k]))
        cur = np.where(acc[None, :], wp, cur)
        g = np.where(acc, gp, g)
        sums[n_out + 1] += acc
        if k >= n_therm:
            sums[:n_out] += cur / g[None, :]             # f/pi = (f/q) / (pi/q)
            sums[n_out] += 1.0 / g                       # q/pi
    return sums, np.concatenate([cur, g[None, :]])


def estimate(sums, n_out):
    """Per component: (I, variance of I) from the chains' sums (Eq. nf_mcmc_estimator).

    I = sum_c A_c / sum_c B_c; the chains are independent, so the variance
    follows from the spread of A_c - I B_c over the chains (delta method)."""
    A, B = sums[:n_out], sums[n_out]
    C = B.size
    I = A.sum(axis=1) / B.sum()
    r = A - I[:, None] * B[None, :]
    var = (r * r).sum(axis=1) / (C * (C - 1.0)) / (B.mean() ** 2)
    return I, var
