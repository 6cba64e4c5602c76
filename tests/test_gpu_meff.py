"""End to end to the effective mass (Sec. VI.A): GPU estimates of
Sigma^(n,m,l)(k_F, i w0) and d Sigma / dk for all n + m + l <= 4 from the
compiled graphs (integrand kernel, tile partials, fixed-order accumulation),
renormalised by the library's host post-process, against the oracle's
estimates on the same Philox points renormalised by the oracle's
post-process.  The two sides see the same samples, so they may differ only
by the per-sample FP32 error (<= 2e-5 of the oracle's L1 magnitude per
sample, tests/parity.py); the bound on m*/m follows by propagating that error through the
post-process with its central-difference derivatives."""
import numpy as np
import pytest

import oracle_pool
import parity

from oracle import conventions, postprocess as opp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 4
RS, T, LAM = 1.0, 1.0 / 25.0, 1.0


def _estimates(api, n, seed, jit):
    P = conventions.ueg_params(RS, T, LAM, 1.0)
    sig_g, dsig_g, sig_o, dsig_o, tol_s, tol_d = {}, {}, {}, {}, {}, {}
    for order in range(1, N + 1):
        G = api.Graph(order, with_dk=True, budget=8192 if jit else None)
        if jit:
            G.jit()
        plan = api.EvalPlan([G], [api.ueg_params(order, RS, T, LAM, 1.0)], [0], n)
        st = plan.run(seed, order).cpu().numpy()[0]                  # [R][2][2]
        ref, mag = oracle_pool.eval_roots(order, G.roots, seed, n, prm=(RS, T, LAM, 1.0), iteration=order)
        for r, (nn, m, l, dk) in enumerate(G.roots):
            g = complex(st[r, 0, 0], st[r, 1, 0])
            o = complex(ref[r].real.mean(), ref[r].imag.mean())
            t = parity.MAX_REL * mag[r].mean()
            if dk:
                dsig_g[(nn, m, l)], dsig_o[(nn, m, l)], tol_d[(nn, m, l)] = g, o, t
            else:
                sig_g[(nn, m, l)], sig_o[(nn, m, l)], tol_s[(nn, m, l)] = g, o, t
    return sig_g, dsig_g, sig_o, dsig_o, tol_s, tol_d


def _bound(sig, dsig, tol_s, tol_d, kF, beta, Lam):
    """sum_i |d meff / d input_i| tol_i (central differences of the oracle post-process)."""
    base = opp.renormalize(sig, dsig, kF, beta, Lam, N)["meff"]
    bound = np.zeros_like(base)
    for which, d, tol in (("s", sig, tol_s), ("d", dsig, tol_d)):
        for k in d:
            for comp in ((1.0, 0.0), (0.0, 1.0)):
                h = max(abs(d[k]), 1e-3) * 1e-6
                step = complex(*comp) * h
                dp, dm = dict(d), dict(d)
                dp[k] = d[k] + step
                dm[k] = d[k] - step
                args_p = (dp, dsig) if which == "s" else (sig, dp)
                args_m = (dm, dsig) if which == "s" else (sig, dm)
                mp = opp.renormalize(*args_p, kF, beta, Lam, N)["meff"]
                mm = opp.renormalize(*args_m, kF, beta, Lam, N)["meff"]
                bound += np.abs((mp - mm) / (2 * h)) * tol[k]
    return base, bound


@pytest.mark.parametrize("jit", [False, True])
def test_meff_matches_oracle_on_the_same_points(jit):
    from paper_2403_18840_gb300 import api
    n = 1 << 13
    sig_g, dsig_g, sig_o, dsig_o, tol_s, tol_d = _estimates(api, n, 77, jit)
    P = conventions.ueg_params(RS, T, LAM, 1.0)
    for k in sig_o:
        assert abs(sig_g[k] - sig_o[k]) <= 2 * tol_s[k] + 1e-12, k
    for k in dsig_o:
        assert abs(dsig_g[k] - dsig_o[k]) <= 2 * tol_d[k] + 1e-12, k
    got = api.postprocess(N, sig_g, dsig_g, P.kF, P.beta, P.Lambda)
    ref, bound = _bound(sig_o, dsig_o, tol_s, tol_d, P.kF, P.beta, P.Lambda)
    print("m*/m partial sums gpu", got["meff"], "oracle", ref, "bound", bound)
    assert np.all(np.abs(got["meff"] - ref) <= bound + 1e-12)
    # the first-order mass is the Hartree-Fock one: below 1 for the screened exchange
    assert 0.5 < ref[1] < 1.0
