"""Pins for the VEGAS oracle (Lepage's separable adaptive map, cited in Sec. IV)."""
import math

import numpy as np

import workloads
from oracle import philox, vegas


def test_identity_grid_map():
    e = vegas.uniform_edges(3, 16)
    y = workloads.uniform_points(1, 3, 1000)
    x, jac, _ = vegas.vegas_map(e, y)
    assert np.allclose(x, y, rtol=0, atol=1e-15)
    assert np.allclose(jac, 1.0, rtol=0, atol=1e-13)


def test_uniform_histogram_is_fixed_point():
    e = vegas.uniform_edges(2, 32)
    new = vegas.vegas_update(e, np.ones((2, 32)), alpha=0.5)
    assert np.allclose(new, e, atol=1e-15)


def test_update_invariants():
    d = workloads.histogram_like(3, 4, 64)
    e = vegas.uniform_edges(4, 64)
    for _ in range(3):
        e = vegas.vegas_update(e, d, alpha=0.5)
        assert np.all(np.diff(e, axis=1) > 0)
        assert np.all(e[:, 0] == 0.0) and np.all(e[:, -1] == 1.0)


def test_convergence_to_optimal_density():
    # for a separable f = prod_k g(x_k) the optimal VEGAS density is |g|
    # normalised; iterate sample -> histogram -> update and compare the grid's
    # density with g on the bins (alpha = 1 for speed of convergence)
    Nb = 32
    e = vegas.uniform_edges(2, Nb)
    g = lambda t: np.exp(-((t - 0.3) / 0.1) ** 2) + 0.05
    for it in range(12):
        y = philox.uniforms(5, it, 0, np.arange(1 << 15), 2)
        x, jac, bins = vegas.vegas_map(e, y)
        f = g(x[0]) * g(x[1])
        d = vegas.vegas_histogram(bins, f * jac, Nb)
        e = vegas.vegas_update(e, d, alpha=1.0)
    # grid density on each bin is 1/(Nb width); compare with normalised g at bin centres
    widths = np.diff(e[0])
    dens = 1.0 / (Nb * widths)
    centres = 0.5 * (e[0, 1:] + e[0, :-1])
    from scipy import integrate
    Z, _ = integrate.quad(g, 0, 1, points=[0.3])
    ref = g(centres) / Z
    rel = np.abs(dens - ref) / ref
    assert np.median(rel) < 0.1
    # and the variance per sample is close to the optimum (int |f|)^2 - I^2 = 0 for f >= 0
    y = philox.uniforms(6, 0, 0, np.arange(1 << 15), 2)
    x, jac, _ = vegas.vegas_map(e, y)
    w = g(x[0]) * g(x[1]) * jac
    assert np.std(w) / np.mean(w) < 0.15


def test_histogram_accumulates_squares():
    bins = np.array([[0, 1, 1, 3]])
    d = vegas.vegas_histogram(bins, np.array([1.0, 2.0, -3.0, 0.5]), 4)
    assert np.array_equal(d, np.array([[1.0, 13.0, 0.0, 0.25]]))
    assert math.isclose(d.sum(), 14.25)
