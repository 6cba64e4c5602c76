"""VEGAS separable importance map (oracle; test infrastructure).

Sec. IV cites VEGAS (Lepage 1978, 2021) for the separable map
q(x) = prod_k q_k(x_k); the paper does not restate the algorithm, so this
follows Lepage's published method with these readings:

* map: per dimension, edges 0 = e_0 < ... < e_Nb = 1; for y in (0,1),
  i = floor(y Nb), x = e_i + (y Nb - i)(e_{i+1} - e_i), J = prod Nb (e_{i+1} - e_i).
* training data: d[dim, i] = sum over samples whose y falls in bin i of (f J)^2.
* update: smooth d with the 3-point average (2-point at the ends), normalise,
  damp r_i = ((rho_i - 1) / ln rho_i)^alpha with rho_i = dbar_i / sum dbar
  (r = 0 for rho = 0), then place new edges so every new bin holds an equal
  share of sum r, interpolating linearly inside the old bins.

Pinned in tests/test_oracle_vegas.py: identity-grid invariants, monotone edges,
the fixed point of a uniform histogram, and convergence of the grid towards
the known optimal density of separable test functions.
"""
import math

import numpy as np


def uniform_edges(dim, n_bins):
    return np.tile(np.linspace(0.0, 1.0, n_bins + 1), (dim, 1))


def vegas_map(edges, y):
    """y [D, N] in (0,1) -> (x [D, N], jac [N], bin index [D, N])."""
    edges = np.asarray(edges, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    D, Nb1 = edges.shape
    Nb = Nb1 - 1
    i = np.minimum(np.floor(y * Nb).astype(np.int64), Nb - 1)
    frac = y * Nb - i
    rows = np.arange(D)[:, None]
    lo = edges[rows, i]
    width = edges[rows, i + 1] - lo
    x = lo + frac * width
    jac = np.prod(Nb * width, axis=0)
    return x, jac, i


def vegas_histogram(bins, fJ, n_bins):
    """d[dim, bin] = sum of (f J)^2 over samples in each bin."""
    bins = np.asarray(bins)
    D = bins.shape[0]
    w = np.asarray(fJ, dtype=np.float64) ** 2
    d = np.zeros((D, n_bins))
    for k in range(D):
        np.add.at(d[k], bins[k], w)
    return d


def vegas_update(edges, d, alpha=0.5):
    """New edges [D, Nb+1] from the histogram d [D, Nb]."""
    edges = np.asarray(edges, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    D, Nb1 = edges.shape
    Nb = Nb1 - 1
    new = edges.copy()
    for k in range(D):
        dk = d[k]
        sm = np.empty(Nb)
        if Nb == 1:
            sm[0] = dk[0]
        else:
            sm[0] = (dk[0] + dk[1]) / 2.0
            sm[-1] = (dk[-2] + dk[-1]) / 2.0
            for i in range(1, Nb - 1):
                sm[i] = (dk[i - 1] + dk[i] + dk[i + 1]) / 3.0
        S = math.fsum(sm.tolist())
        if not S > 0.0:
            continue
        r = np.zeros(Nb)
        for i in range(Nb):
            rho = sm[i] / S
            if rho <= 0.0:
                r[i] = 0.0
            elif rho >= 1.0:
                r[i] = 1.0
            else:
                r[i] = ((rho - 1.0) / math.log(rho)) ** alpha
        R = math.fsum(r.tolist())
        if not R > 0.0:
            continue
        target = R / Nb
        e = edges[k]
        acc = 0.0
        j = 0
        for t in range(1, Nb):
            want = t * target
            while j < Nb - 1 and acc + r[j] < want:
                acc += r[j]
                j += 1
            # new edge lies inside old bin j
            frac = (want - acc) / r[j] if r[j] > 0 else 0.0
            frac = min(max(frac, 0.0), 1.0)
            new[k, t] = e[j] + frac * (e[j + 1] - e[j])
        new[k, 0] = 0.0
        new[k, Nb] = 1.0
    return new
