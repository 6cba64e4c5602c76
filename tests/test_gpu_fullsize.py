"""Parity at the benchmark's full size: one order-5 launch of 2^24 samples on a
VEGAS grid of 1024 bins per dimension, with the autotuned specialised kernel
the benchmark times (same variant, tile size and grid).  Sampled outputs are
checked one by one against the FP64 oracle; the reduction and the VEGAS
histogram are checked over all 2^24 samples by properties that hold at any
size (tile partial sums = sums of the per-sample values; every histogram row
sums to the total of the squared |f| sums)."""
import numpy as np
import pytest

import parity

import workloads
from oracle import conventions, integrand as oig, philox as ophilox, vegas as ovegas

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WL = workloads.BENCH_ORDER5
SEED, ITER = 11, 3


def _grid(dim, nb):
    """Seeded non-uniform grid, FP32-representable edges (what the kernel maps with)."""
    e = ovegas.vegas_update(ovegas.uniform_edges(dim, nb), workloads.histogram_like(41, dim, nb), 0.7)
    e = e.astype(np.float32).astype(np.float64)
    e[:, 0], e[:, -1] = 0.0, 1.0
    return e


def test_bench_launch_sampled_parity_and_properties():
    from paper_2403_18840_gb300 import api, autotune, fdgraph
    order, n, nb = WL["order"], WL["n_samples"], WL["n_bins"]
    roots = fdgraph.graph_roots(order)
    params = api.ueg_params(order, WL["rs"], WL["T_over_TF"], WL["lam_over_kF"], WL["kext_over_kF"])
    G, tuned = autotune.tuned_jit_graph(order, roots, params)
    assert api.L.lib().fd_tile_samples(n) == 4096
    e = _grid(G.dim, nb)
    V = api.Vegas(G.dim, nb)
    V.set_edges(e)
    plan = api.EvalPlan([G], [params], [0], n, maps=[V], per_sample=True)
    st = plan.run(SEED, ITER).cpu().numpy()[0]                    # [R][2][2]: mean, var of the mean
    torch.cuda.synchronize()
    f = plan.per_sample[0, :len(roots)]                           # [R][2][n] FP32, on the device

    # sampled outputs against the oracle: both ends, tile edges, random interior
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, 1, 4095, 4096, 4097, n // 2, n - 4097, n - 2, n - 1],
                                    rng.integers(0, n, 39)]))
    got = f[:, :, torch.tensor(idx, device=f.device)].cpu().numpy().astype(np.float64)
    P = conventions.ueg_params(WL["rs"], WL["T_over_TF"], WL["lam_over_kF"], WL["kext_over_kF"])
    u = ophilox.uniforms(SEED, ITER, 0, idx, G.dim)
    x, _, bins = ovegas.vegas_map(e, u)
    rows = np.arange(G.dim)[:, None]
    jd = nb * (e[rows, bins + 1] - e[rows, bins])
    jv = np.stack([np.prod(jd[:4 * r[0] - 1], axis=0) for r in roots])
    ref, mag = oig.eval_roots(x, roots, P, with_l1=True)
    ref, mag = ref * jv, mag * jv
    err = np.abs(got[:, 0] - ref.real) + np.abs(got[:, 1] - ref.imag)
    rel = np.maximum(err - 1e-30, 0.0) / np.maximum(mag, 1e-30)
    print("full size: %d sampled outputs, max err/M %.3e, frac <= 1e-5: %.4f, variant %s"
          % (rel.size, rel.max(), np.mean(rel <= 1e-5), tuned))
    parity.check(rel, "full size")

    # reduction over all samples: tile partials (FP32 warp sums, FP64 across
    # warps and tiles) against the FP64 sum of the per-sample FP32 values
    mean64 = f.double().mean(dim=2).cpu().numpy()                 # [R][2]
    scale = f.double().abs().mean(dim=2).cpu().numpy() + 1e-30
    assert np.all(np.abs(st[:, :, 0] - mean64) <= 1e-6 * scale), np.max(np.abs(st[:, :, 0] - mean64) / scale)
    assert np.all(np.isfinite(st)) and np.all(st[:, :, 1] >= 0)

    # histogram: each coordinate's bins sum to sum_i (sum over value roots of
    # |Re f_i| + |Im f_i|)^2 (FP32 per tile in shared memory, FP64 across tiles)
    value_roots = [r for r, (_, _, _, dk) in enumerate(roots) if not dk]
    hs = f[value_roots].abs().sum(dim=(0, 1), dtype=torch.float64)
    total = float((hs * hs).sum())
    h = V.hist()
    assert h.shape == (G.dim, nb) and np.all(h >= 0)
    rowsum = h.sum(axis=1)
    print("histogram rows / per-sample total: %.3e .. %.3e" % (rowsum.min() / total - 1, rowsum.max() / total - 1))
    assert np.all(np.abs(rowsum / total - 1) <= 1e-5)
