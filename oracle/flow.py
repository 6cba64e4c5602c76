"""Affine coupling normalizing flow on the unit hypercube (oracle, FP64).

Appendix A: the flow is a composition T = T_K o ... o T_1 of coupling layers
(Eq. coupling_layer): one part of the coordinates passes unchanged and
conditions an invertible map of the other part; the density follows from the
change of variables (Eq. NFtransform) and training minimises the forward KL
divergence, i.e. maximises the weighted log-likelihood of samples of the target.

Readings (the paper's flow is a rational-quadratic spline flow; the build's
configuration asks for affine coupling):
* base z ~ U(0,1)^D, y = logit(z);
* layer l: A = first ceil(D/2) coordinates for even l, the rest for odd l;
  (s_raw, t) = W3 relu(W2 relu(W1 y_A + b1) + b2) + b3, s = S tanh(s_raw / S)
  with S = 5; y_B <- y_B exp(s) + t;
* x = sigmoid(y); log q(x) = -sum log(dx/dz) (p_z = 1);
* loss = -sum_i w_i log q(x_i) / sum_i w_i with w_i = |f(x_i)| / q_s(x_i)
  for samples x_i drawn from any sampler q_s (forward KL with importance weights);
* Adam with beta = (0.9, 0.999), eps = 1e-8.
Parameter blob (FP32 on the GPU, FP64 here), per layer in order:
W1 [H, a], b1 [H], W2 [H, H], b2 [H], W3 [2b, H], b3 [2b]; rows 0..b-1 of W3
give s_raw and rows b..2b-1 give t.

Pinned in tests/test_oracle_flow.py: log q against a finite-difference Jacobian
determinant, normalisation of q on D = 2, inverse(forward(z)) = z, and the
analytic gradient against central finite differences.
"""
import numpy as np

S_CLAMP = 5.0

_PREC = {"mode": "f64"}


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as FP64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def set_precision(mode):
    """'f64' (default) or 'bf16': the configured BF16 weight/activation contract
    (weights and every GEMM input rounded to BF16, FP64 accumulation)."""
    assert mode in ("f64", "bf16")
    _PREC["mode"] = mode


def layer_split(dim, layer):
    h = (dim + 1) // 2
    first = np.arange(0, h)
    second = np.arange(h, dim)
    return (first, second) if layer % 2 == 0 else (second, first)


def param_shapes(dim, n_layers, hidden):
    shapes = []
    for l in range(n_layers):
        A, B = layer_split(dim, l)
        a, b = len(A), len(B)
        shapes.append([(hidden, a), (hidden,), (hidden, hidden), (hidden,), (2 * b, hidden), (2 * b,)])
    return shapes


def n_params(dim, n_layers, hidden):
    return sum(int(np.prod(s)) for layer in param_shapes(dim, n_layers, hidden) for s in layer)


def unpack(blob, dim, n_layers, hidden):
    blob = np.asarray(blob, dtype=np.float64)
    out, off = [], 0
    for layer in param_shapes(dim, n_layers, hidden):
        mats = []
        for s in layer:
            k = int(np.prod(s))
            mats.append(blob[off:off + k].reshape(s))
            off += k
        out.append(mats)
    assert off == blob.size
    return out


def pack(layers):
    return np.concatenate([m.ravel() for layer in layers for m in layer])


def _mlp(p, a):
    W1, b1, W2, b2, W3, b3 = p
    if _PREC["mode"] == "bf16":
        W1, W2, W3, a = bf16(W1), bf16(W2), bf16(W3), bf16(a)
        h1 = bf16(np.maximum(W1 @ a + b1[:, None], 0.0))
        h2 = bf16(np.maximum(W2 @ h1 + b2[:, None], 0.0))
    else:
        h1 = np.maximum(W1 @ a + b1[:, None], 0.0)
        h2 = np.maximum(W2 @ h1 + b2[:, None], 0.0)
    o = W3 @ h2 + b3[:, None]
    return h1, h2, o


def _log_sig_deriv(y):
    # log(sigmoid(y) (1 - sigmoid(y))) = -softplus(y) - softplus(-y)
    return -np.logaddexp(0.0, y) - np.logaddexp(0.0, -y)


def forward(blob, z, dim, n_layers, hidden):
    """z [D, N] in (0,1) -> (x [D, N], log q(x) [N])."""
    layers = unpack(blob, dim, n_layers, hidden)
    z = np.asarray(z, dtype=np.float64)
    y = np.log(z) - np.log1p(-z)
    logdet = -_log_sig_deriv(y).sum(axis=0)         # d y / d z
    for l, p in enumerate(layers):
        A, B = layer_split(dim, l)
        _, _, o = _mlp(p, y[A])
        b = len(B)
        s = S_CLAMP * np.tanh(o[:b] / S_CLAMP)
        t = o[b:]
        y[B] = y[B] * np.exp(s) + t
        logdet = logdet + s.sum(axis=0)
    logdet = logdet + _log_sig_deriv(y).sum(axis=0)  # d x / d y
    x = 1.0 / (1.0 + np.exp(-y))
    return x, -logdet


def inverse(blob, x, dim, n_layers, hidden, keep=False):
    """x [D, N] -> (z [D, N], log q(x) [N]) (and per-layer intermediates if keep)."""
    layers = unpack(blob, dim, n_layers, hidden)
    x = np.asarray(x, dtype=np.float64)
    v = np.log(x) - np.log1p(-x)
    logq = -_log_sig_deriv(v).sum(axis=0)
    saved = [None] * n_layers
    for l in range(n_layers - 1, -1, -1):
        p = layers[l]
        A, B = layer_split(dim, l)
        a = v[A].copy()
        h1, h2, o = _mlp(p, a)
        b = len(B)
        s = S_CLAMP * np.tanh(o[:b] / S_CLAMP)
        t = o[b:]
        v[B] = (v[B] - t) * np.exp(-s)
        logq = logq - s.sum(axis=0)
        if keep:
            saved[l] = (a, h1, h2, s, v[B].copy())
    logq = logq + _log_sig_deriv(v).sum(axis=0)
    z = 1.0 / (1.0 + np.exp(-v))
    if keep:
        return z, logq, saved, v
    return z, logq


def loss_and_grad(blob, x, w, dim, n_layers, hidden, with_l1=False):
    """Weighted forward-KL loss -sum w log q(x) / sum w and its gradient (blob layout).

    with_l1: also the gradient's L1 magnitude per parameter, the same backward
    pass with every term replaced by its absolute value (|W|^T |g| for a
    product, |g_a| + |g_b| for a sum): the scale against which the rounding
    of a lower-precision evaluation of that gradient entry is measured."""
    layers = unpack(blob, dim, n_layers, hidden)
    w = np.asarray(w, dtype=np.float64)
    wn = w / w.sum()
    z, logq, saved, v0 = inverse(blob, x, dim, n_layers, hidden, keep=True)
    loss = -float(np.sum(wn * logq))
    # dL/dv^(0): L_i contains -log(z(1-z)) with z = sigmoid(v0)
    g = -(1.0 - 2.0 * z) * wn[None, :]
    G = np.abs(g)
    mags = []
    grads = []
    for l in range(n_layers):
        W1, b1, W2, b2, W3, b3 = layers[l]
        A, B = layer_split(dim, l)
        a, h1, h2, s, vB = saved[l]
        if _PREC["mode"] == "bf16":
            a = bf16(a)
            W1, W2, W3 = bf16(W1), bf16(W2), bf16(W3)
        es = np.exp(-s)
        gB = g[B]
        g_t = -gB * es
        g_s = -gB * vB + wn[None, :]
        g_sraw = g_s * (1.0 - (s / S_CLAMP) ** 2)
        g_o = np.concatenate([g_sraw, g_t], axis=0)
        dW3 = g_o @ h2.T
        db3 = g_o.sum(axis=1)
        g_h2 = (W3.T @ g_o) * (h2 > 0)
        dW2 = g_h2 @ h1.T
        db2 = g_h2.sum(axis=1)
        g_h1 = (W2.T @ g_h2) * (h1 > 0)
        dW1 = g_h1 @ a.T
        db1 = g_h1.sum(axis=1)
        g_a = W1.T @ g_h1
        g_new = g.copy()
        g_new[B] = gB * es
        g_new[A] = g[A] + g_a
        if with_l1:
            GB = G[B]
            G_o = np.concatenate([(GB * np.abs(vB) + wn[None, :]) * np.abs(1.0 - (s / S_CLAMP) ** 2),
                                  GB * es], axis=0)
            G_h2 = (np.abs(W3).T @ G_o) * (h2 > 0)
            G_h1 = (np.abs(W2).T @ G_h2) * (h1 > 0)
            mags.append([G_h1 @ np.abs(a).T, G_h1.sum(axis=1),
                         G_h2 @ np.abs(h1).T, G_h2.sum(axis=1), G_o @ np.abs(h2).T, G_o.sum(axis=1)])
            G_new = G.copy()
            G_new[B] = GB * es
            G_new[A] = G[A] + np.abs(W1).T @ G_h1
            G = G_new
        g = g_new
        grads.append([dW1, db1, dW2, db2, dW3, db3])
    if with_l1:
        return loss, pack(grads), pack(mags)
    return loss, pack(grads)


def adam_step(blob, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (blob, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return blob - lr * mh / (np.sqrt(vh) + eps), m, v
