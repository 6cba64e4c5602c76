"""The evaluation graph of the Dyson-Schwinger / parquet construction (Sec.
II.B-C): expanded into monomials it is exactly the set of self-energy
diagrams (each with total weight 1), every monomial conserves momentum at
every vertex with n independent loop momenta, and the compact evaluation
(shared nodes, tensors over leg times) equals the expanded sum per sample
for arbitrary leaf functions; its operation count is below the plain sum
over diagrams."""
import collections
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2403_18840_gb300 import parquet as P
from paper_2403_18840_gb300 import parquet_graph as PG


@pytest.fixture(scope="module")
def construction():
    return P.Construction()


def _piece(n, out_v, mono):
    nv = 2 * n
    succ, pred, partner = [None] * nv, [None] * nv, [None] * nv
    for leaf in mono:
        if leaf[0] == "G":
            _, _, x, y = leaf
            assert succ[x] is None and pred[y] is None
            succ[x], pred[y] = y, x
        else:
            _, _, a, b = leaf
            partner[a], partner[b] = b, a
    assert pred[0] is None and succ[out_v] is None
    pred[0], succ[out_v] = -1, -1
    assert None not in succ + pred + partner
    return tuple(succ), tuple(pred), tuple(partner)


def _loops(piece):
    """Closed fermion loops of a self-energy piece (cycles off the external path)."""
    succ, pred, _ = piece
    v, seen = pred.index(-1), set()
    while v >= 0:
        seen.add(v)
        v = succ[v]
    loops = 0
    for s0 in range(len(succ)):
        if s0 not in seen:
            loops += 1
            v = s0
            while v not in seen:
                seen.add(v)
                v = succ[v]
    return loops


def _conserves(n, out_v, mono):
    net = np.zeros((2 * n, n + 1), dtype=int)
    net[0, 0] += 1                       # k_ext enters at the in-vertex
    net[out_v, 0] -= 1
    for _, m, x, y in mono:
        net[x] -= m
        net[y] += m
    loops = np.array([m for _, m, _, _ in mono])[:, 1:]
    return not net.any() and np.linalg.matrix_rank(loops) == n


def _leaf_functions(n, seed):
    rng = np.random.default_rng(seed)
    var, tau = rng.normal(0, 1, n + 1), rng.uniform(0, 1, n)

    def mv(m):
        return float(np.dot(m, var))

    def g0(m, x, y):
        return math.exp(-0.3 * mv(m) ** 2) * (1 + 0.5 * math.sin(tau[y] - tau[x] + mv(m)))

    def v(m):
        return 1.0 / (mv(m) ** 2 + 0.5)
    return g0, v


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_graph_expands_to_the_diagrams_and_evaluates_them(construction, n):
    root = PG.Evaluator(n, PG.Expanded(), construction).root()
    weights = collections.defaultdict(Fraction)
    for o, monos in root.items():
        for w, mono in monos:
            assert len(mono) == 3 * n - 1
            assert _conserves(n, o, mono)
            weights[P.canonical(_piece(n, o, mono))] += w
    # every diagram once, with its sign and spin factor (-1)^(n+F) 2^F
    assert set(weights) == set(construction.sigma(n))
    for key, w in weights.items():
        assert w == (-1) ** (n + _loops(P.from_key(key))) * 2 ** _loops(P.from_key(key))
    g0, v = _leaf_functions(n, n)
    S = PG.Scalar(g0, v)
    compact = PG.Evaluator(n, S, construction).root()
    naive = collections.defaultdict(float)
    for o, monos in root.items():
        for w, mono in monos:
            val = float(w)
            for leaf in mono:
                val *= g0(leaf[1], leaf[2] // 2, leaf[3] // 2) if leaf[0] == "G" else v(leaf[1])
            naive[o // 2] += val
    scale = max(abs(x) for x in naive.values())
    assert set(compact) == set(naive)
    assert max(abs(compact[k] - naive[k]) for k in naive) < 1e-12 * scale
    D = len(construction.sigma(n))
    if n >= 2:
        assert S.ops < D * (3 * n - 2) + D - 1


def test_routing_of_a_fully_irreducible_vertex(construction):
    # the envelope diagrams: spanning-tree routing conserves momentum at every
    # vertex, the four legs' momenta given, with three independent loop momenta
    legs = {("in", 0): (0, 1, 0, 0, 0, 0, 0), ("out", 0): (0, 0, 1, 0, 0, 0, 0),
            ("in", 1): (0, 0, 0, 1, 0, 0, 0), ("out", 1): (0, 1, -1, 1, 0, 0, 0)}
    for key in construction.irreducible(3):
        piece = P.from_key(key)
        leaves = PG.route_piece(piece, legs, 6, 4, lambda v: v)
        assert len(leaves) == 6 + 4                 # 6 bare lines, 4 interaction lines
        net = np.zeros((len(piece[0]), 7), dtype=int)
        for (kind, j), vtx in P._leg_vertices(piece).items():
            net[vtx] += np.array(legs[(kind, j)]) * (1 if kind == "in" else -1)
        for _, m, x, y in leaves:
            net[x] -= m
            net[y] += m
        assert not net.any()
        assert np.linalg.matrix_rank(np.array([m for _, m, _, _ in leaves])[:, 4:]) == 3


def test_counterterm_derivatives_on_the_graph(construction):
    # Taylor series in Lambda through the graph: coefficient l times l! equals
    # central differences of the plain graph in Lambda (l = 1, 2)
    n, lam, h = 3, 0.6, 1e-3
    g0, _ = _leaf_functions(n, 7)
    rng = np.random.default_rng(8)
    cq = {}

    def v(m):
        if m not in cq:
            cq[m] = (rng.uniform(0.5, 2.0), rng.uniform(0.5, 3.0))
        return cq[m]
    ser = PG.Evaluator(n, PG.Series(g0, v, lam, 2), construction).root()

    def plain(x):
        out = PG.Evaluator(n, PG.Series(g0, v, x, 0), construction).root()
        return {k: s[0] for k, s in out.items()}
    p0, pp, pm = plain(lam), plain(lam + h), plain(lam - h)
    scale1 = max(abs(s[1]) for s in ser.values())
    scale2 = max(abs(2 * s[2]) for s in ser.values())
    for k, s in ser.items():
        assert abs(s[0] - p0[k]) < 1e-12 * (abs(p0[k]) + 1e-300)
        assert abs((pp[k] - pm[k]) / (2 * h) - s[1]) < 1e-5 * scale1
        assert abs((pp[k] - 2 * p0[k] + pm[k]) / h ** 2 - 2 * s[2]) < 1e-5 * scale2


def test_taylor_and_nested_counts_on_the_graph(construction):
    from paper_2403_18840_gb300 import adcount
    rows = adcount.parquet_scaling_table(4, 6, construction)
    g0, v = _leaf_functions(4, 1)
    S = PG.Scalar(g0, v)
    PG.Evaluator(4, S, construction).root()
    assert rows[0][1] == rows[0][2] == S.ops
    t = np.array([r[1] for r in rows], dtype=float)
    assert np.all(np.abs(np.diff(t, 3)) < 1e-9)          # a quadratic in l
    d = np.array([r[2] for r in rows], dtype=float)
    assert 2.5 < d[6] / d[5] < 3.0 and d[6] > 15 * t[6]


def test_taylor_mode_in_mu_and_lambda_on_the_graph(construction):
    # every counterterm root from one graph: the (mu, Lambda) series through
    # the graph against mixed central differences of the plain graph
    n, D, mu0, lam0, h = 3, 2, 0.2, 0.6, 1e-3
    rng = np.random.default_rng(12)
    var, tau = rng.normal(0, 1, n + 1), rng.uniform(0, 1, n)
    cq = {}

    def v(m):
        if m not in cq:
            cq[m] = (rng.uniform(0.5, 2.0), rng.uniform(0.5, 3.0))
        return cq[m]

    def g_at(mu):
        # a bare line exp(-0.3 (p^2 - mu)) (1 + 0.5 sin(...)): its i-th mu-Taylor
        # coefficient is the value times 0.3^i / i!
        def g0(m, x, y, i):
            pm = float(np.dot(m, var))
            base = math.exp(-0.3 * (pm * pm - mu)) * (1 + 0.5 * math.sin(tau[y] - tau[x] + pm))
            return base * 0.3 ** i / math.factorial(i)
        return g0

    ser = PG.Evaluator(n, PG.BiSeries(g_at(mu0), v, lam0, D), construction).root()

    def plain(mu, lam):
        out = PG.Evaluator(n, PG.BiSeries(g_at(mu), v, lam, 0), construction).root()
        return {k: s[(0, 0)] for k, s in out.items()}
    f = {(a, b): plain(mu0 + a * h, lam0 + b * h) for a in (-1, 0, 1) for b in (-1, 0, 1)}
    for k, s in ser.items():
        fd = {(1, 0): (f[1, 0][k] - f[-1, 0][k]) / (2 * h),
              (0, 1): (f[0, 1][k] - f[0, -1][k]) / (2 * h),
              (2, 0): (f[1, 0][k] - 2 * f[0, 0][k] + f[-1, 0][k]) / h ** 2 / 2,
              (0, 2): (f[0, 1][k] - 2 * f[0, 0][k] + f[0, -1][k]) / h ** 2 / 2,
              (1, 1): (f[1, 1][k] - f[1, -1][k] - f[-1, 1][k] + f[-1, -1][k]) / (4 * h * h)}
        scale = max(abs(x) for x in s.values())
        assert abs(s[(0, 0)] - f[0, 0][k]) < 1e-12 * scale
        for e, d in fd.items():
            assert abs(s[e] - d) < 1e-5 * scale, (k, e)


def test_all_roots_counts(construction):
    from paper_2403_18840_gb300 import adcount
    g0, v = _leaf_functions(4, 1)
    S = PG.Scalar(g0, v)
    PG.Evaluator(4, S, construction).root()
    per, total = adcount.parquet_all_roots_ops(4, construction)
    assert per[4] == S.ops                      # degree 0: the plain graph
    assert total == sum(per.values()) and all(per[n] > 0 for n in per)
