"""Per-sample parity criterion shared by the GPU tests (test infrastructure).

|f_gpu - f_oracle| (Re and Im summed) against the oracle's L1 magnitude M(x)
(the sum of |term| over diagrams and derivative distributions, Eq.
sigma_integration with Eq. sigma_xi_dmu_dlambda): every sample within
MAX_REL M(x), at least FRAC_MIN of them within FRAC_REL M(x); an absolute
1e-30 absorbs FP32 underflow of values below ~1e-38.

Where the bounds come from: after the double-float map and eps (exact up to
its FP32 rounding) the kernels' error is the FP32 arithmetic of the leaf
families and the contraction, a few 1e-6 of M; the single G line of the
order-1 diagram runs in FP64.  A CPU build of the same device code stays
below 1e-5 M at 2^16 samples per order (tests/test_integrand_host.py).
"""
import numpy as np

MAX_REL = 2e-5
FRAC_REL = 1e-5
FRAC_MIN = 0.999


def rel_error(f, ref, mag):
    """f [R, 2, n] (Re, Im), ref complex [R, n], mag [R, n] -> err / M [R, n]."""
    err = np.abs(f[:, 0] - ref.real) + np.abs(f[:, 1] - ref.imag)
    err = np.maximum(err - 1e-30, 0.0)
    return err / np.maximum(mag, 1e-30)


def check(rel, label):
    frac = float(np.mean(rel <= FRAC_REL))
    print("%s: max err/M %.3e, frac <= %.0e: %.5f (%d values)" % (label, rel.max(), FRAC_REL, frac, rel.size))
    assert rel.max() <= MAX_REL, (label, float(rel.max()))
    assert frac >= FRAC_MIN, (label, frac)


def bound(mag):
    """Per-value bound for tests that compare element-wise without fractions."""
    return MAX_REL * mag + 1e-30
