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


# ---- a hand-worked update (Lepage, J. Comput. Phys. 27 (1978) 192) ----------------
# Two dimensions, four bins each, alpha = 1/2, worked out step by step:
#
# dim 0: edges (0, 1/4, 1/2, 3/4, 1), histogram d = (0, 3, 3, 6)
#   smoothing (3-point mean, 2-point at the ends): (0+3)/2, (0+3+3)/3, (3+3+6)/3,
#   (3+6)/2 = (1.5, 2, 4, 4.5), sum 12 -> rho = (1/8, 1/6, 1/3, 3/8)
#   damping r = ((rho - 1) / ln rho)^(1/2):
#     (-7/8 / ln(1/8))^.5 = 0.648680239866002, (-5/6 / ln(1/6))^.5 = 0.681976677601739,
#     (-2/3 / ln(1/3))^.5 = 0.778990469187241, (-5/8 / ln(3/8))^.5 = 0.798258044049380
#   R = 2.907905430704362, each new bin holds R / 4 = 0.726976357676091:
#     edge 1: cumulative 0.7270 - 0.6487 = 0.0783 into old bin 1, fraction 0.114807617887208
#             -> 1/4 + 0.114807617887208 / 4 = 0.2787019044718021
#     edge 2: 1.4540 - 1.3307 = 0.1234 into old bin 2 -> 1/2 + 0.158276388173376 / 4
#     edge 3: 2.1809 - 2.1096 = 0.0713 into old bin 3 -> 3/4 + 0.089296546279313 / 4
# dim 1: edges (0, 0.1, 0.3, 0.6, 1), histogram d = (8, 0, 0, 0)
#   smoothing: (4, 8/3, 0, 0), sum 20/3 -> rho = (0.6, 0.4, 0, 0)
#   r = ((0.6-1)/ln 0.6)^.5 = 0.884898906987960, ((0.4-1)/ln 0.4)^.5 = 0.809205783940263, 0, 0
#   R / 4 = 0.423526172732056: edges 1 and 2 fall in old bin 0 (fractions 0.478615319091832,
#   0.957230638183663 of its width 0.1), edge 3 in old bin 1 (fraction 0.476614995669233 of 0.2)
HAND_EDGES = np.array([[0.0, 0.2787019044718021, 0.53956909704334399, 0.77232413656982823, 1.0],
                       [0.0, 0.047861531909183165, 0.09572306381836633, 0.19532299913384665, 1.0]])
# the same dim-0 histogram with alpha = 1 (r = (rho - 1) / ln rho: 0.420786053592614,
# 0.465092188792706, 0.606826151084558, 0.637215904889541)
HAND_EDGES_ALPHA1 = np.array([0.0, 0.31003864593338892, 0.57377809380591249, 0.79109118647856169, 1.0])


def test_update_hand_worked_example():
    e = np.array([[0.0, 0.25, 0.5, 0.75, 1.0], [0.0, 0.1, 0.3, 0.6, 1.0]])
    d = np.array([[0.0, 3.0, 3.0, 6.0], [8.0, 0.0, 0.0, 0.0]])
    assert np.max(np.abs(vegas.vegas_update(e, d, alpha=0.5) - HAND_EDGES)) <= 1e-14
    assert np.max(np.abs(vegas.vegas_update(e[:1], d[:1], alpha=1.0)[0] - HAND_EDGES_ALPHA1)) <= 1e-14
