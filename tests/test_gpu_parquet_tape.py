"""GPU parity of tapes compiled from the Dyson-Schwinger / parquet graph:
the library's interpreter runs them (through the C-ABI, Philox samples),
and every root, k-derivative roots included, is compared sample by sample
with the FP64 oracle evaluating the construction's diagrams with the
construction's momentum routing.  Tolerance as for the present tapes
(tests/parity.py)."""
import math

import numpy as np
import pytest

import parity

import parquet_oracle
from oracle import conventions, integrand as oig, philox as ophilox
from paper_2403_18840_gb300 import fdgraph
from paper_2403_18840_gb300 import parquet as P
from paper_2403_18840_gb300 import parquet_graph as PG

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_2403_18840_gb300 import api as A
    assert torch.cuda.is_available()
    return A


@pytest.fixture(scope="module")
def construction():
    return P.Construction()


def _reference(order, roots, x, construction):
    Pm = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    out = np.zeros((len(roots), x.shape[1]), dtype=np.complex128)
    mag = np.zeros((len(roots), x.shape[1]))
    diags = {}
    for r, (n, m, l, dk) in enumerate(roots):
        if n not in diags:
            diags[n] = (parquet_oracle.routed_diagrams(n, construction), oig.map_hypercube(x, n, Pm))
        ds, (kvec, tau, jac) = diags[n]
        for w, d in ds:
            val, l1 = oig.diagram_value(d, kvec, tau, Pm, m, l, dk, return_abs=True)
            line = d.out_vertex // 2
            phase = 1.0 if line == 0 else np.exp(1j * math.pi * x[oig.time_coord(line)])
            out[r] += w * val * phase * jac
            mag[r] += abs(w * d.sign) * l1 * np.abs(jac)
    return out, mag


# specialised-kernel variants: the small shared-memory leaf cache of the
# lower orders and the large global one of the order-6 effective-mass graph
JIT = {"lc24": dict(threads=256, min_blocks=1, spt=2, unit_cap=12000, sv_smem=True, leaf_cache=24),
       "lc2048_global": dict(threads=256, min_blocks=1, spt=1, unit_cap=4000, leaf_cache=2048, lc_global=True)}


@pytest.mark.parametrize("jit", [None, "lc24", "lc2048_global"])
@pytest.mark.parametrize("order,with_dk,n", [(2, True, 3001), (3, True, 2049), (4, False, 700), (5, False, 513)])
def test_parquet_tape_per_sample_parity(api, construction, order, with_dk, n, jit):
    roots = fdgraph.graph_roots(order, with_dk=with_dk)
    tape = PG.parquet_tape(order, roots, budget=8192 if jit else 96, construction=construction).to_bytes()
    G = api.Graph(order, roots, tape=tape)
    if jit:
        G.jit(**JIT[jit])
    plan = api.EvalPlan([G], [api.ueg_params(order, 1.0, 1.0 / 25.0, 1.0, 1.0)], [0], n, per_sample=True)
    seed = 61 + order
    plan.run(seed, 0)
    torch.cuda.synchronize()
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)[:len(roots)]
    x = ophilox.uniforms(seed, 0, 0, np.arange(n), 4 * order - 1)
    ref, mag = _reference(order, roots, x, construction)
    err = np.abs(f[:, 0, :] - ref.real) + np.abs(f[:, 1, :] - ref.imag)
    err = np.maximum(err - 1e-30, 0.0)
    rel = err / np.maximum(mag, 1e-30)
    frac = float(np.mean(rel <= 1e-5))
    print("parquet tape order %d: max err/M %.3e, frac <= 1e-5: %.4f" % (order, rel.max(), frac))
    parity.check(rel, "parquet tape order %d" % order)
