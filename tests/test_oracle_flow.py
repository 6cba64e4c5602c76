"""Pins for the affine coupling flow oracle (Appendix A, Eqs. NFtransform, coupling_layer)."""
import numpy as np

import workloads
from oracle import flow


def _blob(seed, D, K, H, scale=0.3):
    n = flow.n_params(D, K, H)
    return workloads.normal_blob(seed, n, scale)


def test_inverse_of_forward():
    D, K, H = 7, 4, 16
    blob = _blob(1, D, K, H, 0.1)
    z = workloads.uniform_points(2, D, 64, 0.01, 0.99)
    x, lq = flow.forward(blob, z, D, K, H)
    z2, lq2 = flow.inverse(blob, x, D, K, H)
    assert np.allclose(z2, z, atol=1e-9)
    assert np.allclose(lq2, lq, atol=1e-9)


def test_log_density_matches_numerical_jacobian():
    # log q(x) = -log |det dx/dz|, determinant by central differences + slogdet
    D, K, H = 19, 8, 32
    blob = _blob(3, D, K, H, 0.05)
    z = workloads.uniform_points(4, D, 4, 0.05, 0.95)
    _, lq = flow.forward(blob, z, D, K, H)
    h = 1e-6
    for i in range(z.shape[1]):
        J = np.empty((D, D))
        for j in range(D):
            zp = z[:, i:i + 1].copy()
            zm = zp.copy()
            zp[j] += h
            zm[j] -= h
            J[:, j] = (flow.forward(blob, zp, D, K, H)[0][:, 0] - flow.forward(blob, zm, D, K, H)[0][:, 0]) / (2 * h)
        sign, logdet = np.linalg.slogdet(J)
        assert sign > 0
        assert abs(-logdet - lq[i]) < 1e-5


def test_density_normalised_on_grid():
    D, K, H = 2, 4, 8
    blob = _blob(5, D, K, H, 0.3)
    # Gauss-Legendre in t with x = (1 - cos(pi t)) / 2, which crowds nodes at the
    # faces where the logit-space flow puts its tails
    t, wt = np.polynomial.legendre.leggauss(400)
    t = 0.5 * (t + 1.0)
    wt = 0.5 * wt
    g = 0.5 * (1.0 - np.cos(np.pi * t))
    wg = wt * 0.5 * np.pi * np.sin(np.pi * t)
    X = np.stack(np.meshgrid(g, g, indexing="ij")).reshape(2, -1)
    Wg = np.outer(wg, wg).ravel()
    _, lq = flow.inverse(blob, X, D, K, H)
    integral = float(np.sum(np.exp(lq) * Wg))
    # ReLU kinks limit the quadrature to ~1e-4; a wrong Jacobian term is O(1)
    assert abs(integral - 1.0) < 1e-3


def test_gradient_matches_finite_differences():
    D, K, H = 5, 4, 8
    blob = _blob(6, D, K, H, 0.2)
    x = workloads.uniform_points(7, D, 32, 0.02, 0.98)
    w = workloads.positive_weights(8, 32)
    L, g = flow.loss_and_grad(blob, x, w, D, K, H)
    rng = np.random.default_rng(9)
    idx = rng.choice(blob.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        bp = blob.copy()
        bm = blob.copy()
        bp[i] += h
        bm[i] -= h
        fd = (flow.loss_and_grad(bp, x, w, D, K, H)[0] - flow.loss_and_grad(bm, x, w, D, K, H)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_is_signed_lr():
    # with bias correction the first Adam step moves every parameter by lr * sign(grad)
    blob = np.zeros(5)
    grad = np.array([1.0, -2.0, 3e-3, -4e-5, 0.0])
    new, m, v = flow.adam_step(blob, grad, np.zeros(5), np.zeros(5), 1, 0.01)
    expect = -0.01 * grad / (np.abs(grad) + 1e-8)
    assert np.allclose(new, expect, rtol=1e-6, atol=1e-12)


def test_gradient_magnitude_bounds_the_gradient():
    # the absolute-value backward pass dominates |gradient| entry by entry, and
    # equals it where an entry is one product chain (a bias of the t half of
    # the first layer processed, from one sample)
    D, K, H = 7, 3, 16
    blob = workloads.normal_blob(4, flow.n_params(D, K, H), 0.3)
    x = workloads.uniform_points(5, D, 40, 0.05, 0.95)
    w = workloads.positive_weights(6, 40)
    _, g, M = flow.loss_and_grad(blob, x, w, D, K, H, with_l1=True)
    assert np.all(M >= np.abs(g) * (1 - 1e-12))
    _, g1, M1 = flow.loss_and_grad(blob, x[:, :1], w[:1], D, K, H, with_l1=True)
    b3_g = flow.unpack(g1, D, K, H)[0][5]
    b3_m = flow.unpack(M1, D, K, H)[0][5]
    nb = len(flow.layer_split(D, 0)[1])
    assert np.allclose(b3_m[nb:], np.abs(b3_g[nb:]), rtol=1e-12, atol=0)
    assert np.any(b3_m[:nb] > np.abs(b3_g[:nb]) * (1 + 1e-9)) or np.allclose(b3_m[:nb], np.abs(b3_g[:nb]))
