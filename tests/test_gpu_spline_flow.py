"""GPU parity of the spline flow's sampling and density passes (App. A) with
the FP64 oracle on the same parameters: explicit points, the Philox sample
stream, the density at given points (inverse pass), a sample -> density
round trip, the identity flow, and ragged sample counts.  Both conditioner
paths: FP32 CUDA cores against the FP64 oracle, BF16 tensor cores (the
default) against the oracle under the same BF16 contract."""
import contextlib

import numpy as np
import pytest

import parity
import workloads
from oracle import philox as ophilox, spline_flow as osf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_2403_18840_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def _flatten(flow):
    """The oracle's parameters in the library's order (fd_nsf_set_params)."""
    return flow.flat().astype(np.float32)


def _as_fp32(flow):
    """The oracle flow with its parameters rounded to FP32 (what the GPU holds)."""
    for _, _, net in flow.layers:
        for name in ("w0", "b0", "w1", "b1"):
            setattr(net, name, getattr(net, name).astype(np.float32).astype(np.float64))
        net.blocks = [tuple((w.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
                            for (w, b) in blk) for blk in net.blocks]
    return flow


def _compare(x_gpu, lq_gpu, x_ref, lq_ref, label, inverse=False, bf16=False):
    # Forward: FP32 through 8 layers, a coordinate carries ~1e-6 absolute error
    # and log q (a sum of 8 x D/2 log-derivatives) ~1e-4 in the worst samples.
    # Inverse: each layer divides the error of its input by the spline's
    # derivative there (down to ~0.1 for these parameters), so the errors are
    # ~10x larger: ~2e-5 / 2e-4 for z, 3e-4 / 2e-3 for log q (99 % / max).
    # BF16 conditioner (against the oracle under the same contract, or its
    # own round trip): a value that the GPU sums in FP32 and the oracle in
    # FP64 can round to the neighbouring BF16 value when it lies within its
    # ~1e-7 difference of a rounding boundary -- about 5e-5 of the ~1400
    # roundings of a sample at D = 19 and 8 layers, so ~7 % of the samples
    # carry one such flip (2^-8 in one activation, through the softmax knots
    # up to ~1e-3 in a coordinate and ~0.1 in log q, 10x for the inverse).
    # So 90 % of the samples must meet the FP32 path's 99 % bounds, and every
    # sample the bound of a flip.
    dx = np.abs(x_gpu - x_ref).max(axis=0)
    dl = np.abs(lq_gpu - lq_ref)
    print("%s: max |dx| %.3e (99%% %.3e, 90%% %.3e), max |d log q| %.3e (99%% %.3e, 90%% %.3e)" %
          (label, dx.max(), np.quantile(dx, 0.99), np.quantile(dx, 0.9), dl.max(), np.quantile(dl, 0.99),
           np.quantile(dl, 0.9)))
    bx, bl = ((5e-5, 5e-4), (1e-3, 1e-2)) if inverse else ((5e-6, 5e-5), (1e-4, 1e-3))
    if bf16:
        flip = (1e-1, 1.0) if inverse else (1e-2, 0.2)
        assert np.quantile(dx, 0.9) < bx[0] and dx.max() < flip[0], label
        assert np.quantile(dl, 0.9) < bl[0] and dl.max() < flip[1], label
    else:
        assert np.quantile(dx, 0.99) < bx[0] and dx.max() < bx[1], label
        assert np.quantile(dl, 0.99) < bl[0] and dl.max() < bl[1], label


@contextlib.contextmanager
def _oracle_precision(path):
    osf.set_precision("bf16" if path == 1 else "f64")
    try:
        yield
    finally:
        osf.set_precision("f64")


def _gpu_flow(api, dim, n_layers, flow, path):
    g = api.SplineFlow(dim, n_layers)
    g.set_params(_flatten(flow))
    g.set_tensor_path(path)
    return g


PATHS = [0, 1]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("dim", [19, 5])
def test_forward_matches_oracle(api, dim, path):
    flow = _as_fp32(osf.SplineFlow(dim, 8, seed=11, scale=0.8))
    g = _gpu_flow(api, dim, 8, flow, path)
    n = 3 * 1000 + 77                                        # several blocks and a ragged tail
    z = workloads.uniform_points(12, dim, n)
    x, lq = g.forward(torch.tensor(z, dtype=torch.float32, device="cuda").contiguous())
    with _oracle_precision(path):
        x_ref, lq_ref = flow.forward(z.T)
    _compare(x.cpu().numpy().astype(np.float64), lq.cpu().numpy().astype(np.float64), x_ref.T, lq_ref,
             "forward dim %d path %d" % (dim, path), bf16=path == 1)


@pytest.mark.parametrize("path", PATHS)
def test_sample_stream_matches_oracle(api, path):
    dim, n = 19, 2049
    flow = _as_fp32(osf.SplineFlow(dim, 8, seed=13, scale=0.8))
    g = _gpu_flow(api, dim, 8, flow, path)
    x, lq = g.sample(21, 4, 3, n)
    z = ophilox.uniforms(21, 4, 3, np.arange(n), dim)
    with _oracle_precision(path):
        x_ref, lq_ref = flow.forward(z.T)
    _compare(x.cpu().numpy().astype(np.float64), lq.cpu().numpy().astype(np.float64), x_ref.T, lq_ref,
             "sample path %d" % path, bf16=path == 1)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("dim", [19, 6])
def test_log_density_matches_oracle(api, dim, path):
    flow = _as_fp32(osf.SplineFlow(dim, 8, seed=15, scale=0.8))
    g = _gpu_flow(api, dim, 8, flow, path)
    n = 2 * 1000 + 33
    z0 = workloads.uniform_points(16, dim, n)
    with _oracle_precision(path):
        x_ref, _ = flow.forward(z0.T)                        # points inside the flow's image
        z, lq = g.log_density(torch.tensor(x_ref.T, dtype=torch.float32, device="cuda").contiguous())
        lq_ref, z_ref = flow.log_density(x_ref.astype(np.float32).astype(np.float64))
    _compare(z.cpu().numpy().astype(np.float64), lq.cpu().numpy().astype(np.float64), z_ref.T, lq_ref,
             "log density dim %d path %d" % (dim, path), inverse=True, bf16=path == 1)


@pytest.mark.parametrize("path", PATHS)
def test_sample_then_density_round_trip(api, path):
    # the kept half a layer conditions on is the same in both directions up to
    # FP32 rounding, so the round trip holds to the splines' FP32 arithmetic
    # on the FP32 path and, but for BF16 rounding flips, on the tensor path
    dim, n = 19, 4096
    flow = _as_fp32(osf.SplineFlow(dim, 8, seed=17, scale=0.8))
    g = _gpu_flow(api, dim, 8, flow, path)
    x, lq = g.sample(5, 0, 1, n)
    z, lq2 = g.log_density(x)
    z0 = ophilox.uniforms(5, 0, 1, np.arange(n), dim)
    _compare(z.cpu().numpy().astype(np.float64), lq2.cpu().numpy().astype(np.float64), z0,
             lq.cpu().numpy().astype(np.float64), "round trip path %d" % path, inverse=True, bf16=path == 1)


@pytest.mark.parametrize("path", PATHS)
def test_identity_flow(api, path):
    dim, n = 7, 1000
    flow = osf.SplineFlow(dim, 4, seed=1, zero=True)
    g = _gpu_flow(api, dim, 4, flow, path)
    z = workloads.uniform_points(3, dim, n)
    x, lq = g.forward(torch.tensor(z, dtype=torch.float32, device="cuda").contiguous())
    assert np.max(np.abs(x.cpu().numpy() - z.astype(np.float32))) < 1e-6
    assert np.max(np.abs(lq.cpu().numpy())) < 1e-5


def test_invalid_arguments(api):
    with pytest.raises(api.L.FdError):
        api.SplineFlow(25, 8)
    g = api.SplineFlow(3, 2)
    with pytest.raises(api.L.FdError):
        g.set_params(np.full(g.n_params, np.nan, dtype=np.float32))


@pytest.mark.parametrize("dim,n_layers,n", [(5, 4, 3 * 128 + 77), (19, 2, 300), (6, 3, 1)])
def test_kl_grad_matches_oracle(api, dim, n_layers, n):
    # FP32 per sample against the FP64 oracle's closed-form reverse mode: an
    # FP32 restatement of the same arithmetic lands at ~1e-5 of the gradient's
    # largest entry (99 % of entries ~2e-6) and ~1e-5 relative in l2; the
    # atomic sums add reordering noise of the same size
    flow = _as_fp32(osf.SplineFlow(dim, n_layers, seed=41, scale=0.8))
    g = api.SplineFlow(dim, n_layers)
    g.set_params(_flatten(flow))
    z = workloads.uniform_points(42, dim, n)
    x_ref, _ = flow.forward(z.T)
    x32 = x_ref.astype(np.float32)
    w32 = np.exp(-4.0 * ((x32.astype(np.float64) - 0.4) ** 2).sum(axis=1)).astype(np.float32)
    x = torch.tensor(x32.T, device="cuda").contiguous()
    w = torch.tensor(w32, device="cuda")
    loss, grad = g.kl_grad(x, w)
    gr = flow.kl_grad(x32.astype(np.float64), w32.astype(np.float64), analytic=True)
    lr = flow.kl_loss(x32.astype(np.float64), w32.astype(np.float64))
    gg = grad.cpu().numpy().astype(np.float64)
    err = np.abs(gg - gr)
    scale = np.abs(gr).max()
    print("kl_grad dim %d layers %d n %d: loss %.9f (oracle %.9f), max err %.2e of max |g|, rel l2 %.2e" %
          (dim, n_layers, n, float(loss.item()), lr, err.max() / scale, np.linalg.norm(gg - gr) / np.linalg.norm(gr)))
    assert abs(float(loss.item()) - lr) < 1e-5 * (1.0 + abs(lr))
    assert err.max() < 2e-4 * scale and np.linalg.norm(gg - gr) < 1e-4 * np.linalg.norm(gr)
    # a small step against the gradient lowers the loss the kernel reports
    theta = _flatten(flow)
    g.set_params(theta - 1e-2 * gg.astype(np.float32) / np.linalg.norm(gg))
    loss2, _ = g.kl_grad(x, w)
    assert float(loss2.item()) < float(loss.item())


def test_kl_grad_rejects_deep_flows(api):
    g = api.SplineFlow(3, 17)
    x = torch.full((3, 4), 0.5, device="cuda")
    w = torch.ones(4, device="cuda")
    with pytest.raises(api.L.FdError):
        g.kl_grad(x, w)


def test_training_first_adam_step_and_descent(api):
    # from zero moments the first bias-corrected Adam step moves every
    # parameter by lr g / (|g| + eps), i.e. -lr sign(g) wherever |g| >> eps;
    # the sign is taken from the oracle's gradient where it is unambiguous
    # (|g| above 1e-3 of the largest, far above the GPU/oracle difference),
    # elsewhere only |step| <= lr is required
    dim, n_layers, n, lr = 5, 4, 1000, 1e-3
    flow = _as_fp32(osf.SplineFlow(dim, n_layers, seed=51, scale=0.8))
    theta = _flatten(flow)
    g = api.SplineFlow(dim, n_layers)
    g.set_params(theta)
    z = workloads.uniform_points(52, dim, n)
    x_ref, _ = flow.forward(z.T)
    x32 = x_ref.astype(np.float32)
    w32 = np.exp(-6.0 * ((x32.astype(np.float64) - 0.3) ** 2).sum(axis=1)).astype(np.float32)
    x = torch.tensor(x32.T, device="cuda").contiguous()
    w = torch.tensor(w32, device="cuda")
    losses = g.train(x, w, 1, lr)
    gr = flow.kl_grad(x32.astype(np.float64), w32.astype(np.float64), analytic=True)
    lr_ref = flow.kl_loss(x32.astype(np.float64), w32.astype(np.float64))
    assert abs(losses[0] - lr_ref) < 1e-5 * (1.0 + abs(lr_ref))
    d = g.params().astype(np.float64) - theta.astype(np.float64)
    ulp = 2.0 ** -23 * (1.0 + np.abs(theta.astype(np.float64)))   # rounding of the FP32 update
    big = np.abs(gr) > 1e-3 * np.abs(gr).max()
    assert big.sum() > 0.3 * gr.size
    assert np.all(np.abs(d[big] + lr * np.sign(gr[big])) <= 1e-3 * lr + ulp[big])
    assert np.all(np.abs(d) <= lr * (1.0 + 1e-3) + ulp)
    more = g.train(x, w, 40, lr)
    print("spline flow training: loss %.6f -> %.6f after 41 Adam steps" % (losses[0], more[-1]))
    # the oracle's own Adam on its FP64 gradient goes -0.776 -> -1.885 here
    # (the first sign-sized step overshoots: -0.718)
    assert more[-1] < losses[0] - 0.5
    g.set_params(theta)                                  # a fresh Adam state: the same first step
    assert abs(g.train(x, w, 1, lr)[0] - losses[0]) < 1e-6 * (1.0 + abs(losses[0]))
    d2 = g.params().astype(np.float64) - theta.astype(np.float64)
    assert np.all(np.abs(d2[big] - d[big]) <= 1e-3 * lr + 2 * ulp[big])


def test_sampler_weights_and_integrand_points(api):
    """fd_nsf_sample_w: the sample stream's points with w = 1/q(x) (App. A's
    flow as the proposal): the same points as fd_nsf_sample, w = exp(-log q),
    and as point weights of the integrand they give the oracle's weighted
    integrand at those points."""
    from oracle import conventions, integrand as oig
    g = api.SplineFlow(7, 4)
    g.set_params(workloads.small_params(21, g.n_params))
    n = 3001
    x, lq = g.sample(5, 1, 2, n)
    x2, w = g.draw(5, 1, 2, n)
    torch.cuda.synchronize()
    assert torch.equal(x, x2)
    lqn = lq.cpu().numpy().astype(np.float64)
    assert np.allclose(w.cpu().numpy(), np.exp(-lqn), rtol=2e-6, atol=0)
    G = api.Graph(2, with_dk=True)
    plan = api.EvalPlan([G], [api.ueg_params(2, 1.0, 1.0 / 25.0, 1.0, 1.0)], [0], n, per_sample=True)
    plan.run(5, 1, points=x2, point_w=w)
    torch.cuda.synchronize()
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)[:len(G.roots)]
    P = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    ref, mag = oig.eval_roots(x2.cpu().numpy().astype(np.float64), G.roots, P, with_l1=True)
    wd = w.cpu().numpy().astype(np.float64)
    parity.check(parity.rel_error(f, ref * wd, mag * wd), "integrand on spline-flow points")
