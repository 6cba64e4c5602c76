"""Per-sample parity at 2^16 samples per order (Eq. sigma_integration with
the counterterm roots of Eq. sigma_xi_dmu_dlambda) on both contraction
paths: the tape interpreter and the specialised kernel (one sample per
thread; the sample-loop variant with 4 samples per thread, their inputs in
shared memory, units of cost <= 12000 and a barrier after every unit; and
with 2 samples per thread and a 32-float leaf cache).  Orders 3 and 4 with every k-derivative root,
order 5 with the 15 roots of the benchmark; the oracle runs in worker
processes.  Criterion in tests/parity.py."""
import numpy as np
import pytest

import oracle_pool
import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 1 << 16
CASES = [(3, True, 81), (4, True, 82), (5, False, 83)]
VARIANTS = {"interpreter": None,
            "specialised": dict(),
            "specialised_loop": dict(threads=256, min_blocks=1, spt=4, unit_cap=12000, sv_smem=True, sync_every=1),
            "specialised_leaf_cache": dict(threads=256, min_blocks=1, spt=2, unit_cap=12000, sv_smem=True,
                                           sync_every=1, leaf_cache=32),
            "specialised_global_leaf_cache": dict(threads=256, min_blocks=1, spt=3, unit_cap=12000, sv_smem=True,
                                                  sync_every=1, leaf_cache=320, lc_global=True)}


@pytest.fixture(scope="module")
def api():
    from paper_2403_18840_gb300 import api as A
    assert torch.cuda.is_available()
    return A


_REF = {}


def _reference(order, roots, seed):
    if order not in _REF:
        _REF[order] = oracle_pool.eval_roots(order, roots, seed, N)
    return _REF[order]


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("order,with_dk,seed", CASES)
def test_per_sample_parity_2e16(api, order, with_dk, seed, variant):
    opts = VARIANTS[variant]
    G = api.Graph(order, with_dk=with_dk, budget=8192 if opts is not None else None)
    if opts is not None:
        G.jit(**opts)
    plan = api.EvalPlan([G], [api.ueg_params(order, 1.0, 1.0 / 25.0, 1.0, 1.0)], [0], N, per_sample=True)
    plan.run(seed, 0)
    torch.cuda.synchronize()
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)[:len(G.roots)]
    ref, mag = _reference(order, G.roots, seed)
    parity.check(parity.rel_error(f, ref, mag), "order %d %s, %d samples" % (order, variant, N))
