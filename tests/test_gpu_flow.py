"""GPU parity of the affine coupling flow kernels (BF16 tensor cores, FP32
accumulation) against the FP64 oracle under the same BF16 contract."""
import numpy as np
import pytest

import workloads
from oracle import flow as oflow
from oracle import philox as ophilox

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

D, K, H = 19, 8, 128


@pytest.fixture(scope="module")
def api():
    from paper_2403_18840_gb300 import api as A
    return A


@pytest.fixture(autouse=True)
def bf16_oracle():
    oflow.set_precision("bf16")
    yield
    oflow.set_precision("f64")


def _flow(api, seed=1, scale=0.06):
    F = api.Flow(D, K, H, seed=0)
    blob = workloads.normal_blob(seed, F.n_params, scale)
    assert blob.size == oflow.n_params(D, K, H)
    F.set_params(blob)
    return F, blob


def test_param_roundtrip_and_count(api):
    F, blob = _flow(api)
    assert np.array_equal(F.params().astype(np.float64), blob)


def test_sample_parity(api):
    F, blob = _flow(api)
    n = 3000
    x, w = F.sample(21, 2, 3, n)
    torch.cuda.synchronize()
    z = ophilox.uniforms(21, 2, 3, np.arange(n), D)
    xr, lq = oflow.forward(blob, z, D, K, H)
    xg = x.cpu().numpy().astype(np.float64)
    lw = np.log(w.cpu().numpy().astype(np.float64))
    dx = np.abs(xg - xr)
    dl = np.abs(lw + lq)
    print("sample: max |dx| %.3e  max |dlogq| %.3e  p99 %.3e" % (dx.max(), dl.max(), np.quantile(dl, 0.99)))
    assert dx.max() < 2e-3 and np.quantile(dx, 0.99) < 2e-4
    assert dl.max() < 2e-2 and np.quantile(dl, 0.99) < 2e-3


def test_defensive_mixture_parity(api):
    # samples [0, n - n_u): flow; [n - n_u, n): uniform; w = 1 / ((1 - a) q + a), a = n_u / n
    F, blob = _flow(api)
    n = 3000
    x, w, a = F.sample_defensive(21, 2, 3, n, 0.25)
    torch.cuda.synchronize()
    n_u = n - 2560                      # flow share n - floor(0.25 n) = 2250 rounded up to 512s
    assert a == n_u / n
    nf = n - n_u
    u = ophilox.uniforms(21, 2, 3, np.arange(n), D)
    xr = u.copy()
    xr[:, :nf], lq_f = oflow.forward(blob, u[:, :nf], D, K, H)
    _, lq_u = oflow.inverse(blob, u[:, nf:], D, K, H)
    lq = np.concatenate([lq_f, lq_u])
    wr = 1.0 / ((1.0 - a) * np.exp(lq) + a)
    xg = x.cpu().numpy().astype(np.float64)
    wg = w.cpu().numpy().astype(np.float64)
    assert np.array_equal(xg[:, nf:], u[:, nf:])                 # uniform share is the stream itself
    assert np.abs(xg[:, :nf] - xr[:, :nf]).max() < 2e-3
    rel = np.abs(wg / wr - 1.0)
    print("defensive: max rel w %.3e p99 %.3e" % (rel.max(), np.quantile(rel, 0.99)))
    assert rel.max() < 2e-2 and np.quantile(rel, 0.99) < 2e-3
    assert np.all(wg <= 1.0 / a * (1 + 1e-6))


@pytest.mark.parametrize("path", [1, 2])
def test_tensor_paths_agree(api, path):
    # the tcgen05 paths (1: tiles in pairs; 2: warp-specialised) and mma.sync
    # (path 0) compute the same BF16 contract; n spans several 512-sample
    # blocks and a ragged tail
    F, blob = _flow(api)
    n = 5000
    out = {}
    for p in (path, 0):
        F.set_tensor_path(p)
        x, w = F.sample(5, 1, 2, n)
        lq = F.log_density(x)
        xd, wd, _ = F.sample_defensive(5, 1, 2, n, 0.2)
        torch.cuda.synchronize()
        out[p] = [t.cpu().numpy().astype(np.float64) for t in (x, w, lq, xd, wd)]
    F.set_tensor_path(2)
    (x1, w1, l1, xd1, wd1), (x0, w0, l0, xd0, wd0) = out[path], out[0]
    assert np.abs(x1 - x0).max() < 2e-3
    assert np.abs(np.log(w1) - np.log(w0)).max() < 2e-2
    assert np.abs(l1 - l0).max() < 2e-2
    assert np.abs(xd1 - xd0).max() < 2e-3
    assert np.abs(wd1 / wd0 - 1.0).max() < 2e-2
    # the density pass inverts the sampling pass: log q(x) = -log w
    assert np.quantile(np.abs(l1 + np.log(w1)), 0.99) < 2e-3


@pytest.mark.parametrize("path", [1, 2])
def test_tcgen05_path_parity(api, path):
    # the tcgen05 sampling and density passes against the FP64 oracle under the BF16 contract
    F, blob = _flow(api)
    F.set_tensor_path(path)
    n = 3000
    x, w = F.sample(21, 2, 3, n)
    lq = F.log_density(x)
    torch.cuda.synchronize()
    F.set_tensor_path(2)
    z = ophilox.uniforms(21, 2, 3, np.arange(n), D)
    xr, lqr = oflow.forward(blob, z, D, K, H)
    dx = np.abs(x.cpu().numpy().astype(np.float64) - xr)
    dl = np.abs(np.log(w.cpu().numpy().astype(np.float64)) + lqr)
    dd = np.abs(lq.cpu().numpy().astype(np.float64) - lqr)
    print("tcgen05: max |dx| %.3e  max |dlogq| %.3e" % (dx.max(), dl.max()))
    assert dx.max() < 2e-3 and np.quantile(dx, 0.99) < 2e-4
    assert dl.max() < 2e-2 and np.quantile(dl, 0.99) < 2e-3
    assert dd.max() < 2e-2 and np.quantile(dd, 0.99) < 2e-3


def test_log_density_parity_and_consistency(api):
    F, blob = _flow(api)
    n = 2500
    x, w = F.sample(5, 0, 0, n)
    lq = F.log_density(x)
    torch.cuda.synchronize()
    # self-consistency: density of the flow's own samples is 1/w
    a = lq.cpu().numpy().astype(np.float64)
    b = -np.log(w.cpu().numpy().astype(np.float64))
    assert np.quantile(np.abs(a - b), 0.99) < 1e-3
    # parity on given points
    pts = workloads.uniform_points(6, D, n, 0.01, 0.99)
    lq2 = F.log_density(torch.tensor(pts, dtype=torch.float32, device="cuda").contiguous())
    torch.cuda.synchronize()
    _, ref = oflow.inverse(blob, pts, D, K, H)
    d = np.abs(lq2.cpu().numpy().astype(np.float64) - ref)
    print("log density: max %.3e p99 %.3e" % (d.max(), np.quantile(d, 0.99)))
    assert d.max() < 2e-2 and np.quantile(d, 0.99) < 2e-3


def test_gradient_parity(api):
    F, blob = _flow(api)
    n = 4096
    pts = workloads.uniform_points(7, D, n, 0.02, 0.98)
    wts = workloads.positive_weights(8, n)
    loss, g = F.grad(torch.tensor(pts, dtype=torch.float32, device="cuda").contiguous(),
                     torch.tensor(wts, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    Lr, gr, Mr = oflow.loss_and_grad(blob, pts, wts, D, K, H, with_l1=True)
    gg = g.cpu().numpy().astype(np.float64)
    cos = float(gg @ gr / (np.linalg.norm(gg) * np.linalg.norm(gr)))
    rel = float(np.linalg.norm(gg - gr) / np.linalg.norm(gr))
    # element by element: the GPU rounds each gradient operand of a weight
    # GEMM to BF16 (unit roundoff u = 2^-8) where the oracle keeps it in FP64,
    # one rounding per layer on the way back through K layers, so an entry may
    # differ by up to ~K u of its L1 magnitude M (the oracle's absolute-value
    # backward pass)
    ratio = np.abs(gg - gr) / (Mr + 1e-30)
    print("grad: loss %.6f vs %.6f  cos %.6f  rel %.3e  max |dg|/M %.3e  p99 %.3e"
          % (float(loss.item()), Lr, cos, rel, ratio.max(), np.quantile(ratio, 0.99)))
    assert abs(float(loss.item()) - Lr) < 1e-3 * max(1.0, abs(Lr))
    assert ratio.max() <= K * 2.0 ** -8
    assert cos >= 0.999 and rel <= 1e-2


def test_training_reduces_loss_and_first_adam_step(api):
    F, blob = _flow(api, seed=3, scale=0.04)
    n = 8192
    pts = workloads.uniform_points(9, D, n, 0.02, 0.98)
    # a peaked target: weights concentrated near a corner
    wts = np.exp(-20 * np.sum((pts[:4] - 0.3) ** 2, axis=0))
    x = torch.tensor(pts, dtype=torch.float32, device="cuda").contiguous()
    w = torch.tensor(wts, dtype=torch.float32, device="cuda")
    _, g0 = F.grad(x, w)
    p0 = F.params().astype(np.float64)
    losses = F.train(x, w, 1, 1e-3)
    p1 = F.params().astype(np.float64)
    g0 = g0.cpu().numpy().astype(np.float64)
    big = np.abs(g0) > 1e-5
    # first Adam step from zero moments: every parameter moves by lr * sign(grad)
    assert np.allclose((p0 - p1)[big], 1e-3 * np.sign(g0[big]), rtol=2e-3, atol=1e-7)
    more = F.train(x, w, 60, 3e-3)
    print("train losses", losses[0], more[0], more[-1])
    assert more[-1] < more[0] - 0.05


@pytest.mark.parametrize("dim,layers", [(19, 8), (7, 3), (24, 2)])
def test_default_path_many_groups_per_cta(api, dim, layers):
    # n above 152 SMs x 512 samples, so every CTA of the warp-specialised kernel
    # runs several groups (the weight buffers' phases carry over from group to
    # group) and the last group is ragged; odd layer counts end on the other
    # half.  Sampled rows against the oracle, all rows against mma.sync.
    F = api.Flow(dim, layers, H, seed=0)
    blob = workloads.normal_blob(7, F.n_params, 0.06)
    F.set_params(blob)
    n = (1 << 18) + 333
    x, w = F.sample(9, 4, 1, n)
    lq = F.log_density(x)
    xd, wd, a = F.sample_defensive(9, 4, 1, n, 0.3)
    F.set_tensor_path(0)
    x0, w0 = F.sample(9, 4, 1, n)
    lq0 = F.log_density(x)
    F.set_tensor_path(2)
    torch.cuda.synchronize()
    xg, wg, lg = (t.cpu().numpy().astype(np.float64) for t in (x, w, lq))
    assert np.abs(xg - x0.cpu().numpy()).max() < 2e-3
    assert np.abs(np.log(wg) - np.log(w0.cpu().numpy().astype(np.float64))).max() < 2e-2
    assert np.abs(lg - lq0.cpu().numpy()).max() < 2e-2
    assert np.quantile(np.abs(lg + np.log(wg)), 0.99) < 2e-3
    rows = np.unique(np.concatenate([np.arange(64), np.random.default_rng(3).integers(0, n, 1500), np.arange(n - 64, n)]))
    z = ophilox.uniforms(9, 4, 1, rows, dim)
    xr, lqr = oflow.forward(blob, z, dim, layers, H)
    dx = np.abs(xg[:, rows] - xr)
    dl = np.abs(np.log(wg[rows]) + lqr)
    assert dx.max() < 2e-3 and np.quantile(dx, 0.99) < 2e-4
    assert dl.max() < 2e-2 and np.quantile(dl, 0.99) < 2e-3
    # defensive mixture: the flow share ends on a 512-sample boundary
    nf = n - int(round(a * n))
    assert nf % 512 == 0 or nf == n
    xdg = xd.cpu().numpy()
    u = ophilox.uniforms(9, 4, 1, np.arange(nf, n), dim)
    assert np.array_equal(xdg[:, nf:], u.astype(np.float32))
    assert np.abs(xdg[:, :nf] - xg[:, :nf]).max() == 0.0


def test_default_path_at_the_bench_size(api):
    # the launch the flow-vs-VEGAS comparison times: 2^24 samples of the
    # defensive mixture (10 % uniform) on the default path; sampled rows of
    # both shares against the oracle (forward for the flow share, the inverse
    # density for the uniform share), the last rows included
    F, blob = _flow(api)
    n = 1 << 24
    x, w, a = F.sample_defensive(13, 60000, 3, n, 0.1)
    torch.cuda.synchronize()
    nf = n - int(round(a * n))
    rng = np.random.default_rng(8)
    rows_f = np.unique(np.concatenate([np.arange(32), rng.integers(0, nf, 1200), np.arange(nf - 32, nf)]))
    rows_u = np.unique(np.concatenate([np.arange(nf, nf + 32), rng.integers(nf, n, 400), np.arange(n - 32, n)]))
    xs = x[:, torch.as_tensor(np.concatenate([rows_f, rows_u]), device="cuda")].cpu().numpy().astype(np.float64)
    ws = w[torch.as_tensor(np.concatenate([rows_f, rows_u]), device="cuda")].cpu().numpy().astype(np.float64)
    uf = ophilox.uniforms(13, 60000, 3, rows_f, D)
    xr, lq_f = oflow.forward(blob, uf, D, K, H)
    uu = ophilox.uniforms(13, 60000, 3, rows_u, D)
    _, lq_u = oflow.inverse(blob, uu, D, K, H)
    kf = len(rows_f)
    assert np.array_equal(xs[:, kf:], uu)                    # the uniform share is the stream itself
    dx = np.abs(xs[:, :kf] - xr)
    lq = np.concatenate([lq_f, lq_u])
    wr = 1.0 / ((1.0 - a) * np.exp(lq) + a)
    rel = np.abs(ws / wr - 1.0)
    print("bench size: max |dx| %.3e (99%% %.3e), max rel w %.3e (99%% %.3e)" %
          (dx.max(), np.quantile(dx, 0.99), rel.max(), np.quantile(rel, 0.99)))
    assert dx.max() < 2e-3 and np.quantile(dx, 0.99) < 2e-4
    assert rel.max() < 2e-2 and np.quantile(rel, 0.99) < 2e-3
