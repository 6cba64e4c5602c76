"""Order 6 (the effective-mass configuration, D = 23): per-sample parity of the
compiled graph against the FP64 oracle, through the specialised kernel and the
tape interpreter.  The oracle enumerates the 31130 self-energy topologies by
brute force over 12! contractions (about a minute) and evaluates them diagram
by diagram, so the sample counts are small; the roots are the undifferentiated
Sigma^(6) and one counterterm root.  On uniform points most order-6 samples
are negligible (below 1e-100), so the test evaluates given points whose loop
momenta lie inside 1.8 k_F (radial coordinates scaled by 0.3), where the
magnitudes span 1e-36 .. 1e-3."""
import numpy as np
import pytest

import parity

import workloads
from oracle import conventions, integrand as oig

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOTS = [(6, 0, 0, 0), (5, 1, 0, 0)]


def _compare(f, ref, mag, label):
    # the bound of the other per-sample parity tests
    err = np.abs(f[:, 0, :] - ref.real) + np.abs(f[:, 1, :] - ref.imag)
    err = np.maximum(err - 1e-30, 0.0)
    rel = err / np.maximum(mag, 1e-30)
    frac = float(np.mean(rel <= 1e-5))
    print("%s: max err/M %.3e, frac <= 1e-5: %.4f" % (label, rel.max(), frac))
    parity.check(rel, label)


@pytest.fixture(scope="module")
def oracle_ref():
    n = 48
    x = workloads.uniform_points(62, 23, n)
    for c in (0, 3, 7, 11, 15, 19):          # radial coordinate of k_1 .. k_6
        x[c] *= 0.3
    x = x.astype(np.float32).astype(np.float64)
    P = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    ref, mag = oig.eval_roots(x, ROOTS, P, with_l1=True)
    return x, ref, mag


@pytest.mark.parametrize("path", ["specialised", "interpreter"])
def test_order6_per_sample_parity(oracle_ref, path):
    from paper_2403_18840_gb300 import api
    x, ref, mag = oracle_ref
    n = x.shape[1]
    if path == "specialised":
        G = api.Graph(6, roots=ROOTS, budget=1 << 13)
        info = G.jit(threads=256, min_blocks=1, spt=2, unit_cap=12000)
        assert info["enabled"]
    else:
        G = api.Graph(6, roots=ROOTS)
    plan = api.EvalPlan([G], [api.ueg_params(6, 1.0, 1.0 / 25.0, 1.0, 1.0)], [0], n, per_sample=True)
    plan.run(61, 0, points=torch.tensor(x, dtype=torch.float32, device="cuda").contiguous())
    torch.cuda.synchronize()
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)[:len(ROOTS)]
    _compare(f, ref, mag, "order 6 %s" % path)
