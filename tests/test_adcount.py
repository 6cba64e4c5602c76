"""Counterterm derivatives in the screening shift Lambda by Taylor mode, by
nested first-order AD and by the compiler's monomial expansion (Sec. III.C,
Eqs. taylor_node and chain_rule, Fig. ADscaling): the three give the same
derivatives, which equal finite differences of the plain graph in Lambda,
and their operation counts follow the closed forms of the arithmetic."""
import math

import numpy as np
import pytest

from paper_2403_18840_gb300 import adcount as A
from paper_2403_18840_gb300 import fdgraph


@pytest.mark.parametrize("n", [2, 3])
def test_three_routes_give_the_same_derivatives(n):
    dag, roots, outs = A.sigma_dag(n)
    g, v = A.leaf_values(dag, 11 + n)
    lam = 0.4
    for L in (1, 2, 3):
        te = [t[L] * math.factorial(L) for t in A.taylor_eval(dag, roots, g, v, lam, L)]
        ne = A.nested_eval(dag, roots, g, v, lam, L)
        ee = A.expansion_eval(n, L, g, v, lam)
        for k, o in enumerate(outs):
            scale = abs(te[k]) + 1e-300
            assert abs(ne[k] - te[k]) < 1e-12 * scale
            assert abs(ee[o] - te[k]) < 1e-12 * scale


def test_derivatives_match_finite_differences_in_lambda():
    # the plain graph (no derivatives) evaluated at shifted Lambda: central
    # differences of first and second order against Taylor mode
    n = 3
    dag, roots, _ = A.sigma_dag(n)
    g, v = A.leaf_values(dag, 5)
    lam, h = 0.7, 1e-3

    def plain(x):
        return np.array([t[0] for t in A.taylor_eval(dag, roots, g, v, x, 0)])
    d1 = (plain(lam + h) - plain(lam - h)) / (2 * h)
    d2 = (plain(lam + h) - 2 * plain(lam) + plain(lam - h)) / h ** 2
    te = A.taylor_eval(dag, roots, g, v, lam, 2)
    t1 = np.array([t[1] for t in te])
    t2 = np.array([2 * t[2] for t in te])
    # truncation errors of order h^2 times the third and fourth derivatives,
    # bounded relative to the largest root
    assert np.all(np.abs(d1 - t1) < 1e-5 * np.abs(t1).max())
    assert np.all(np.abs(d2 - t2) < 1e-5 * np.abs(t2).max())


def test_interaction_leaf_series_is_the_closed_form():
    # c / (q^2 + L): k-th Taylor coefficient c (-1)^k / (q^2 + L)^(k+1)
    s = A._v_series(1.5, 2.0, 0.5, 6)
    assert np.allclose(s, [1.5 * (-1) ** k / 2.5 ** (k + 1) for k in range(7)], rtol=1e-15)


def test_hyperdual_product_count_is_three_to_the_l():
    for l in range(7):
        assert A.hyperdual_mul_pairs(l) == 3 ** l


def _product_graph(kinds):
    """A product of leaves (kinds: 'V' depends on Lambda, 'G' does not)."""
    dag = fdgraph.DAG()
    node = None
    for i, k in enumerate(kinds):
        var = ("V", (i + 1,), 0) if k == "V" else ("G", (i + 1,), 0, 0, 0)
        x = dag.var(var)
        node = x if node is None else dag.make("mul", node, x)
    return dag, [node]


def test_counts_follow_the_closed_forms():
    dag, roots = _product_graph("VV")
    for L in range(6):
        assert A.taylor_ops(dag, roots, L) == ((L + 1) ** 2, 2 * L)
        assert A.nested_ops(dag, roots, L) == (2 * 3 ** L - 2 ** L, 2 * L)
    dag, roots = _product_graph("GV")
    for L in range(6):
        assert A.taylor_ops(dag, roots, L)[0] == L + 1
        assert A.nested_ops(dag, roots, L)[0] == 2 ** L
    dag, roots = _product_graph("GG")
    assert A.taylor_ops(dag, roots, 5)[0] == 1 and A.nested_ops(dag, roots, 5)[0] == 1


def test_order4_scaling():
    # without derivatives the three routes count the same graph; Taylor
    # mode's count is a quadratic in L (each node costs 1, L + 1 or (L + 1)^2),
    # nested AD's grows by a factor approaching 3 per order
    rows = A.scaling_table(4, 6)
    assert rows[0][1] == rows[0][2] == rows[0][3]
    t = np.array([r[1] for r in rows], dtype=float)
    assert np.all(np.abs(np.diff(t, 3)) < 1e-9)
    d = np.array([r[2] for r in rows], dtype=float)
    assert 2.5 < d[6] / d[5] < 3.0 and d[6] > 15 * t[6]
    e = np.array([r[3] for r in rows], dtype=float)
    assert np.all(t[1:] < e[1:])
