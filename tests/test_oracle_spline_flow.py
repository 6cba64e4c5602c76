"""Pins of the spline-flow oracle (App. A; rational-quadratic splines of
Durkan et al.): identity at the identity parameters; the spline passes
through its knots with the prescribed derivatives there (second-order
one-sided finite differences from both sides); inverse(forward) = id;
log-derivative vs finite differences; the flow's log-density vs a
finite-difference Jacobian determinant; the forward and inverse passes'
densities agree; the density integrates to 1 (grid, and E_z[1/q] = 1)."""
import numpy as np
import pytest

from oracle import spline_flow as sf


def _params(rng, n, scale=1.5):
    K = sf.K_BINS
    return (rng.normal(0, scale, (n, K)), rng.normal(0, scale, (n, K)), rng.normal(0, scale, (n, K - 1)))


def test_identity_parameters_give_the_identity():
    K = sf.K_BINS
    x = np.linspace(0.0, 1.0, 101)
    tw, th = np.zeros((101, K)), np.zeros((101, K))
    td = np.full((101, K - 1), sf.THETA_D_ONE)
    y, logd = sf.rq_forward(x, tw, th, td)
    assert np.allclose(y, x, atol=1e-14) and np.allclose(logd, 0.0, atol=1e-12)
    flow = sf.SplineFlow(5, 4, seed=1, zero=True)
    z = np.random.default_rng(2).random((50, 5))
    xf, logq = flow.forward(z)
    assert np.allclose(xf, z, atol=1e-13) and np.allclose(logq, 0.0, atol=1e-12)


def test_spline_through_knots_with_their_derivatives():
    rng = np.random.default_rng(3)
    tw, th, td = _params(rng, 1)
    X, Y, D = sf.knots(tw, th, td)
    assert np.all(np.diff(X) > 0) and np.all(np.diff(Y) > 0) and np.all(D > 0)
    assert X[0, 0] == 0.0 and X[0, -1] == 1.0 and Y[0, 0] == 0.0 and Y[0, -1] == 1.0
    for k in range(1, sf.K_BINS):
        y, _ = sf.rq_forward(np.array([X[0, k]]), tw, th, td)
        assert abs(y[0] - Y[0, k]) < 1e-13
        # second-order one-sided differences, the step a small part of the bins
        e = 1e-5 * min(X[0, k] - X[0, k - 1], X[0, k + 1] - X[0, k])
        yl, _ = sf.rq_forward(X[0, k] - np.array([2 * e, e, 0.0]), tw, th, td)
        yr, _ = sf.rq_forward(X[0, k] + np.array([0.0, e, 2 * e]), tw, th, td)
        left = (3 * yl[2] - 4 * yl[1] + yl[0]) / (2 * e)
        right = (-3 * yr[0] + 4 * yr[1] - yr[2]) / (2 * e)
        assert abs(left - D[0, k]) < 1e-6 * D[0, k] and abs(right - D[0, k]) < 1e-6 * D[0, k]


def test_monotone_inverse_and_log_derivative():
    rng = np.random.default_rng(4)
    n = 2000
    tw, th, td = _params(rng, n)
    x = rng.random(n)
    y, logd = sf.rq_forward(x, tw, th, td)
    assert np.all((y >= 0) & (y <= 1))
    xs = np.sort(x)
    ys, _ = sf.rq_forward(xs, tw[:1].repeat(n, 0), th[:1].repeat(n, 0), td[:1].repeat(n, 0))
    assert np.all(np.diff(ys) > 0)                              # one spline: monotone
    xb, logdi = sf.rq_inverse(y, tw, th, td)
    assert np.max(np.abs(xb - x)) < 1e-11
    assert np.allclose(logdi, -logd, atol=1e-9)
    h = 1e-6
    xp, xm = np.clip(x + h, 0, 1), np.clip(x - h, 0, 1)
    yp, _ = sf.rq_forward(xp, tw, th, td)
    ym, _ = sf.rq_forward(xm, tw, th, td)
    fd = (yp - ym) / (xp - xm)
    inner = (x > 2e-6) & (x < 1 - 2e-6)
    X, _, _ = sf.knots(tw, th, td)
    away = np.min(np.abs(X - x[:, None]), axis=1) > 1e-5        # finite differences across a knot
    m = inner & away
    assert np.allclose(np.log(fd[m]), logd[m], atol=1e-6)


@pytest.mark.parametrize("dim", [3, 6])
def test_flow_log_density_vs_jacobian_determinant(dim):
    flow = sf.SplineFlow(dim, 4, seed=5, scale=0.8)
    z = np.random.default_rng(6).uniform(0.05, 0.95, (6, dim))
    x, logq = flow.forward(z)
    h = 1e-6
    for i in range(z.shape[0]):
        J = np.zeros((dim, dim))
        for j in range(dim):
            zp, zm = z[i].copy(), z[i].copy()
            zp[j] += h
            zm[j] -= h
            J[:, j] = (flow.forward(zp[None])[0][0] - flow.forward(zm[None])[0][0]) / (2 * h)
        assert abs(-np.log(abs(np.linalg.det(J))) - logq[i]) < 1e-6
    logq2, zb = flow.log_density(x)
    assert np.max(np.abs(zb - z)) < 1e-10 and np.allclose(logq2, logq, atol=1e-9)


def test_density_integrates_to_one():
    # midpoint rule on a grid (a mild flow), and for a sharper one the exact
    # identity E_z[1 / q(T(z))] = volume = 1 over uniform z
    flow = sf.SplineFlow(2, 4, seed=7, scale=0.5)
    m = 800
    g = (np.arange(m) + 0.5) / m
    X, Y = np.meshgrid(g, g, indexing="ij")
    logq, _ = flow.log_density(np.stack([X.ravel(), Y.ravel()], axis=1))
    q = np.exp(logq)
    assert q.max() / q.min() > 2.0                               # a non-trivial density
    assert abs(q.mean() - 1.0) < 1e-3
    sharp = sf.SplineFlow(4, 6, seed=8, scale=1.0)
    z = np.random.default_rng(9).random((200000, 4))
    _, logq = sharp.forward(z)
    r = np.exp(-logq)
    assert abs(r.mean() - 1.0) < 5 * r.std() / np.sqrt(r.size)


def test_flat_parameters_round_trip_and_loss_gradient():
    # a small flow: the parameter vector round-trips, the finite-difference
    # gradient of the forward-KL loss is step-consistent, and a descent step
    # along it lowers the loss
    flow = sf.SplineFlow(2, 1, seed=21, scale=0.8)
    theta = flow.flat()
    z = np.random.default_rng(22).random((40, 2))
    x0, _ = flow.forward(z)
    flow.set_flat(theta)
    x1, _ = flow.forward(z)
    assert np.array_equal(x0, x1) and np.array_equal(flow.flat(), theta)
    rng = np.random.default_rng(23)
    x = rng.uniform(0.02, 0.98, (16, 2))
    w = np.exp(-8 * ((x - 0.3) ** 2).sum(axis=1))              # a peaked target
    g = flow.kl_grad_fd(x, w, h=1e-5)
    assert np.linalg.norm(g) > 0
    # step consistency on the output layer (the parameters the loss moves most)
    out = slice(theta.size - 23 * 9, theta.size)
    sub = sf.SplineFlow(2, 1, seed=21, scale=0.8)
    g2 = np.array([_fd_one(sub, x, w, j, 5e-6) for j in range(out.start, out.stop)])
    assert np.allclose(g[out], g2, rtol=1e-5, atol=1e-9)
    l0 = flow.kl_loss(x, w)
    flow.set_flat(theta - 1e-2 * g / np.linalg.norm(g))
    assert flow.kl_loss(x, w) < l0


def _fd_one(flow, x, w, j, h):
    theta = flow.flat()
    tp, tm = theta.copy(), theta.copy()
    tp[j] += h
    tm[j] -= h
    flow.set_flat(tp)
    lp = flow.kl_loss(x, w)
    flow.set_flat(tm)
    lm = flow.kl_loss(x, w)
    flow.set_flat(theta)
    return (lp - lm) / (2 * h)


def test_reverse_mode_gradient_matches_finite_differences():
    # the chain-rule gradient through the inverse pass (the reference a GPU
    # training pass would be checked against) against whole-flow differences
    rng = np.random.default_rng(23)
    flow = sf.SplineFlow(2, 1, seed=21, scale=0.8)
    x = rng.uniform(0.02, 0.98, (16, 2))
    w = np.exp(-8 * ((x - 0.3) ** 2).sum(axis=1))
    g = flow.kl_grad(x, w)
    gf = flow.kl_grad_fd(x, w, h=1e-5)
    assert np.max(np.abs(g - gf)) < 1e-6 * np.max(np.abs(gf))
    flow = sf.SplineFlow(3, 2, seed=31, scale=0.8)            # two layers: gradients through a later layer
    x = rng.uniform(0.02, 0.98, (12, 3))
    w = rng.random(12)
    g = flow.kl_grad(x, w)
    idx = rng.choice(g.size, 120, replace=False)
    gf = np.array([_fd_one(flow, x, w, j, 1e-5) for j in idx])
    assert np.max(np.abs(g[idx] - gf)) < 1e-6 * max(np.max(np.abs(gf)), 1e-3)



def test_closed_form_spline_partials():
    # the closed-form partials of one spline (what a GPU backward pass would
    # evaluate) against central differences: the gap shrinks as the step
    # squared, to ~2e-6 of the scale at step 1e-6
    rng = np.random.default_rng(5)
    P = rng.normal(0, 1.2, (500, sf.K_BINS * 3 - 1))
    u = rng.uniform(0.01, 0.99, 500)
    a = sf._spline_partials_analytic(u, P)
    f5 = sf._spline_partials(u, P, 1e-5)
    f6 = sf._spline_partials(u, P, 1e-6)
    for x, y5, y6 in zip(a, f5, f6):
        e5 = np.max(np.abs(x - y5) / (np.abs(y5) + 1.0))
        e6 = np.max(np.abs(x - y6) / (np.abs(y6) + 1.0))
        assert e6 < 1e-5 and (e6 < 1e-13 or e6 < 0.05 * e5)     # exact, or second-order convergence
    rng = np.random.default_rng(24)
    flow = sf.SplineFlow(3, 2, seed=31, scale=0.8)
    x = rng.uniform(0.02, 0.98, (12, 3))
    w = rng.random(12)
    assert np.allclose(flow.kl_grad(x, w, analytic=True), flow.kl_grad(x, w), rtol=1e-5, atol=1e-9)


def test_bf16_contract_rounds_only_the_conditioner_inputs():
    # Under the BF16 contract a layer's spline parameters come from BF16
    # weights and BF16 GEMM inputs: with weights, biases and inputs that are
    # exact in BF16 and a conditioner whose hidden values stay BF16-exact (one
    # nonzero W0 entry of 1, identity-like blocks switched off), both modes
    # agree exactly; with general parameters they differ by ~2^-8 relative in
    # the parameters but the flow stays invertible: forward then inverse under
    # the contract returns the input, as the kept half is the same both ways.
    rng = np.random.default_rng(5)
    flow = sf.SplineFlow(6, 4, seed=3, scale=0.8)
    z = rng.uniform(0.05, 0.95, (200, 6))
    try:
        sf.set_precision("bf16")
        x, lq = flow.forward(z)
        lq2, z2 = flow.log_density(x)
    finally:
        sf.set_precision("f64")
    assert np.abs(z2 - z).max() < 1e-9 and np.abs(lq2 - lq).max() < 1e-9
    x64, lq64 = flow.forward(z)
    d = np.abs(x - x64).max()
    assert 1e-6 < d < 5e-2, d                       # the contract changes the flow a little, not a lot
    # exact agreement when nothing needs rounding
    net = flow.layers[0][2]
    net.w0[:] = 0.0
    net.w0[0, 0] = 1.0
    net.b0[:] = 0.0
    for (wa, ba), (wb, bb) in net.blocks:
        wa[:] = 0.0
        ba[:] = 0.0
        wb[:] = 0.0
        bb[:] = 0.0
    net.w1[:] = sf.bf16(net.w1)
    net.b1[:] = 0.0
    u = sf.bf16(rng.uniform(0.0, 1.0, (50, net.w0.shape[0])))
    ref = net(u)
    try:
        sf.set_precision("bf16")
        got = net(u)
    finally:
        sf.set_precision("f64")
    assert np.array_equal(got, ref)
