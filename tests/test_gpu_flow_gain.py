"""What the learned proposal gains over the method without it (VEGAS alone).

Order-5 self-energy at r_s = 1, k = k_F: VEGAS is adapted for 8 iterations,
then the affine coupling flow is trained by forward KL on |f| from batches the
method generates (VEGAS first, then the flow itself).  At equal sample counts
the flow must give a lower per-sample variance and a higher variance-adjusted
rate of effective samples than VEGAS, and both estimates must agree.
"""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_flow_beats_vegas_at_order5():
    from paper_2403_18840_gb300 import api, driver, fdgraph
    order = 5
    roots = fdgraph.graph_roots(order)
    p = api.ueg_params(order, 1.0, 1.0 / 25.0, 1.0, 1.0)
    G = api.Graph(order, roots=roots)
    V = api.Vegas(G.dim, 1024)
    driver.adapt_vegas(G, p, V, 1 << 22, 8, seed=21)
    F = api.Flow(G.dim, 8, 128, seed=5)
    losses = driver.train_flow(G, p, F, V, steps=400, batch=1 << 18, lr=1e-3, seed=22, vegas_steps=100,
                               evals_per_batch=2)
    cmp = driver.compare(G, p, V, F, 1 << 22, seed=23)
    print(cmp)
    assert losses[-1] < losses[0] - 1.0
    assert cmp["flow"]["var_per_sample"] < 0.7 * cmp["vegas"]["var_per_sample"]
    assert cmp["flow_over_vegas"] > 1.3
    assert cmp["means_agree_sigma"] < 4.0
