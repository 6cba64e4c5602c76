"""Pin the oracle's counterterm leaves against mpmath high-precision derivatives
of the undifferentiated definitions (Eqs. propagator, green_ct, interaction_ct)."""

import mpmath as mp
import numpy as np
import pytest

from oracle.leaves import G0_deriv, V_deriv

mp.mp.dps = 50


def _G0_mp(eps, tau, beta):
    # definition: tau > 0: -exp(-eps tau)(1 - f); tau <= 0: exp(-eps tau) f
    f = 1 / (mp.exp(beta * eps) + 1)
    if tau > 0:
        return -mp.exp(-eps * tau) * (1 - f)
    return mp.exp(-eps * tau) * f


CASES = [(-3.0, 2.0), (-0.3, 5.5), (0.01, 0.7), (0.8, -1.2), (4.0, -6.0),
         (-2.0, -0.01), (1e-3, 0.0), (-1.5, 0.0), (25.0, 0.5), (-3.6, 6.7), (30.0, -6.0)]


@pytest.mark.parametrize("eps,tau", CASES)
@pytest.mark.parametrize("m", [0, 1, 2, 3, 4, 5])
def test_G0_mu_derivatives(eps, tau, m):
    beta = 6.787633974565
    # d/dmu = -d/deps at fixed momentum
    ref = mp.diff(lambda mu: _G0_mp(mp.mpf(eps) - mu, mp.mpf(tau), mp.mpf(beta)), 0, m)
    got = float(G0_deriv(np.array(eps), np.array(tau), beta, m))
    scale = max(abs(float(ref)), 1e-300)
    # exact derivatives of the definition; the stable evaluation keeps FP64
    # close to round-off in every regime
    assert abs(got - float(ref)) <= 1e-11 * scale + 1e-300, (got, float(ref))


def test_G0_no_overflow_far_from_fermi_surface():
    beta = 6.787633974565
    eps = np.array([4700.0, -3.68, 4700.0, -3.68])
    tau = np.array([-6.7, 6.7, 6.7, -6.7])
    for m in range(6):
        v = G0_deriv(eps, tau, beta, m)
        assert np.all(np.isfinite(v))


@pytest.mark.parametrize("q2", [0.0, 0.3, 4.0, 130.0])
@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 5])
def test_V_lambda_derivatives(q2, l):
    lam = 3.683168552353
    ref = mp.diff(lambda L: 8 * mp.pi / (mp.mpf(q2) + L), mp.mpf(lam), l)
    got = float(V_deriv(np.array(q2), lam, l))
    assert abs(got - float(ref)) <= 1e-12 * abs(float(ref))
