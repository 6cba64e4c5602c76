"""Operation counts of the interaction-counterterm derivatives: Taylor mode
against nested first-order AD (Sec. III.C, Eqs. taylor_node and chain_rule,
Fig. ADscaling).

The counterterm roots Sigma^(n,0,l) are the l-th derivatives in the screening
shift Lambda of the order-n self-energy graph, which depends on Lambda only
through its interaction leaves V(Lambda) = c / (q^2 + Lambda).  Three ways of
computing them, counted on the same hash-consed graph of Sigma^(n) (the
compiler's DAG for the root (n, 0, 0, 0), one sub-graph per out line):

* Taylor mode: every node carries its truncated series in Lambda to order L
  (coefficients 0..L, all counterterm orders at once); a sum of two
  Lambda-dependent series costs L + 1 adds, a product (L + 1)^2 multiply-adds
  (Cauchy product), a product with a Lambda-independent node L + 1.
* Nested first-order AD: forward mode applied l times, i.e. every node a
  hyper-dual number with 2^l components (one per subset of the l nesting
  directions); a product of two Lambda-dependent numbers is the subset
  convolution, 3^l multiplies and 3^l - 2^l adds, a sum 2^l adds, a product
  with a Lambda-independent node 2^l multiplies.
* Expansion (the compiler's present route for one root): the root's Leibniz
  expansion into monomials over leaf Taylor coefficients, factorised by
  greedy Horner and hash-consed, counted like `fdgraph.contraction_ops`.

Counting rule everywhere: a multiply or an add is 1, an FMA 2; the leaves'
own series (V^[k] = -V^[k-1] / (q^2 + Lambda), one multiply per order) are
reported separately.  The evaluators below compute the same quantities
numerically, so that tests can check the three routes against each other and
against finite differences in Lambda.
"""
import itertools
import math

import numpy as np

from . import fdgraph
from . import parquet as P
from . import parquet_graph as PG


def sigma_dag(n, l=0):
    """(dag, roots, keys): the hash-consed graph of the root (n, 0, l, 0), one
    root node per out line (keys = the out lines), products and sums shared
    across out lines."""
    polys = fdgraph.root_polynomials(n, [(n, 0, l, 0)])
    dag = fdgraph.DAG()
    dag.scope = None
    keys = sorted(polys)
    roots = [fdgraph.horner(dag, polys[k]) for k in keys]
    return dag, roots, [k[1] for k in keys]


def _reachable(dag, roots):
    seen = set()
    stack = list(roots)
    while stack:
        u = stack.pop()
        if u in seen:
            continue
        seen.add(u)
        node = dag.nodes[u]
        if node[0] in ("mul", "add"):
            stack.extend(node[1:])
        elif node[0] == "mulc":
            stack.append(node[1])
        elif node[0] == "fma":
            stack.extend(node[1:4])
    return sorted(seen)                      # children are created before parents


def _dependence(dag, order):
    dep = {}
    for u in order:
        node = dag.nodes[u]
        k = node[0]
        if k == "var":
            dep[u] = node[1][0] in ("V", "Vd")
        elif k == "const":
            dep[u] = False
        elif k == "mulc":
            dep[u] = dep[node[1]]
        else:
            kids = node[1:4] if k == "fma" else node[1:]
            dep[u] = any(dep[c] for c in kids)
    return dep


def _mul_cost(da, db, dense_mul, scalar_mul):
    if da and db:
        return dense_mul
    if da or db:
        return scalar_mul
    return 1


def _add_cost(da, db, dense_add):
    return dense_add if (da and db) else 1


def _count(dag, roots, dense_mul, scalar_mul, dense_add):
    order = _reachable(dag, roots)
    dep = _dependence(dag, order)
    ops = 0
    n_v = 0
    for u in order:
        node = dag.nodes[u]
        k = node[0]
        if k == "var":
            n_v += dep[u]
        elif k == "add":
            ops += _add_cost(dep[node[1]], dep[node[2]], dense_add)
        elif k == "mul":
            ops += _mul_cost(dep[node[1]], dep[node[2]], dense_mul, scalar_mul)
        elif k == "mulc":
            ops += scalar_mul if dep[node[1]] else 1
        elif k == "fma":
            x, a, b = node[1:4]
            ops += _mul_cost(dep[x], dep[a], dense_mul, scalar_mul)
            ops += _add_cost(dep[x] or dep[a], dep[b], dense_add)
    return ops, n_v


def taylor_ops(dag, roots, L):
    """(contraction ops, leaf ops) of Taylor mode to order L (all of 0..L)."""
    ops, n_v = _count(dag, roots, (L + 1) ** 2, L + 1, L + 1)
    return ops, n_v * L


def nested_ops(dag, roots, l):
    """(contraction ops, leaf ops) of forward-mode AD nested l times (the
    l-th derivative and every lower mixed derivative along the way)."""
    ops, n_v = _count(dag, roots, 2 * 3 ** l - 2 ** l, 2 ** l, 2 ** l)
    return ops, n_v * l


def expansion_ops(n, l):
    """Contraction ops of the root (n, 0, l, 0) compiled the present way
    (Leibniz expansion, Horner, hash-consing), and its V-leaf series ops."""
    dag, roots, _ = sigma_dag(n, l)
    ops, _ = _count(dag, roots, 1, 1, 1)
    n_v = len({dag.nodes[u][1][1] for u in _reachable(dag, roots)
               if dag.nodes[u][0] == "var" and dag.nodes[u][1][0] == "V"})
    return ops, n_v * l


def scaling_table(n, l_max):
    """Rows (l, Taylor ops, nested ops, expansion ops) for Sigma^(n,0,l)."""
    dag, roots, _ = sigma_dag(n)
    rows = []
    for l in range(l_max + 1):
        t, tl = taylor_ops(dag, roots, l)
        d, dl = nested_ops(dag, roots, l)
        e, el = expansion_ops(n, l)
        rows.append((l, t + tl, d + dl, e + el))
    return rows


def parquet_scaling_table(n, l_max, construction=None):
    """Rows (l, Taylor ops, nested ops) for Sigma^(n,0,l) on the Dyson-Schwinger
    / parquet evaluation graph (`parquet_graph`), the graph the paper's
    comparison uses; V-leaf series included."""
    C = construction or P.Construction()
    rows = []
    for l in range(l_max + 1):
        t = PG.DerivativeCount(l, "taylor")
        PG.Evaluator(n, t, C).root()
        d = PG.DerivativeCount(l, "nested")
        PG.Evaluator(n, d, C).root()
        rows.append((l, t.total(), d.total()))
    return rows


def parquet_all_roots_ops(order, construction=None):
    """Contraction ops of every root (n, m, l) with n + m + l = order from the
    Dyson-Schwinger / parquet graphs of Sigma^(1..order), each in Taylor mode
    in (mu, Lambda) to total degree order - n; leaves excluded.  Returns
    {n: ops} and the total."""
    C = construction or P.Construction()
    per = {}
    for n in range(1, order + 1):
        alg = PG.BiTaylorCount(order - n)
        ev = PG.Evaluator(n, alg, C)
        ev.root()
        per[n] = alg.ops
    return per, sum(per.values())


# ---- numerical evaluation of the same three routes ---------------------------

def leaf_values(dag, seed):
    """Seeded leaf data: a value per G leaf, (c, q^2) per interaction momentum."""
    rng = np.random.default_rng(seed)
    g, v = {}, {}
    for node in dag.nodes:
        if node[0] != "var":
            continue
        var = node[1]
        if var[0] == "G":
            g.setdefault(var[1:4], rng.uniform(-1.0, 1.0))
        elif var[0] == "V":
            v.setdefault(var[1], (rng.uniform(0.5, 2.0), rng.uniform(0.5, 3.0)))
    return g, v


def _v_series(c, q2, lam, L):
    """Taylor coefficients of c / (q^2 + Lambda) at lam, orders 0..L."""
    r = 1.0 / (q2 + lam)
    out = [c * r]
    for _ in range(L):
        out.append(-out[-1] * r)
    return np.array(out)


def _cauchy(a, b):
    L = len(a) - 1
    return np.array([sum(a[i] * b[k - i] for i in range(k + 1)) for k in range(L + 1)])


def _eval(dag, roots, leaf, mul, add, scale):
    val = {}
    for u in _reachable(dag, roots):
        node = dag.nodes[u]
        k = node[0]
        if k == "var":
            val[u] = leaf(node[1])
        elif k == "const":
            val[u] = scale(node[1])
        elif k == "add":
            val[u] = add(val[node[1]], val[node[2]])
        elif k == "mul":
            val[u] = mul(val[node[1]], val[node[2]])
        elif k == "mulc":
            val[u] = val[node[1]] * node[2]
        elif k == "fma":
            val[u] = add(mul(val[node[1]], val[node[2]]), val[node[3]])
    return [val[r] for r in roots]


def taylor_eval(dag, roots, g, v, lam, L):
    """Per root the Taylor coefficients 0..L in Lambda (Taylor mode)."""
    def leaf(var):
        if var[0] == "G":
            s = np.zeros(L + 1)
            s[0] = g[var[1:4]]
            return s
        return _v_series(*v[var[1]], lam, L)

    def scale(c):
        s = np.zeros(L + 1)
        s[0] = c
        return s
    return _eval(dag, roots, leaf, _cauchy, lambda a, b: a + b, scale)


def _subset_conv(a, b):
    n = len(a)
    out = np.zeros(n)
    for s in range(n):
        t = s
        while True:                           # every subset t of s
            out[s] += a[t] * b[s ^ t]
            if t == 0:
                break
            t = (t - 1) & s
    return out


def nested_eval(dag, roots, g, v, lam, l):
    """Per root the l-th derivative in Lambda by nested forward mode
    (hyper-dual numbers with 2^l components; the last is d^l / dLambda^l)."""
    n = 1 << l

    def leaf(var):
        s = np.zeros(n)
        if var[0] == "G":
            s[0] = g[var[1:4]]
            return s
        c, q2 = v[var[1]]
        for m in range(n):                    # component m: derivative of order popcount(m)
            k = bin(m).count("1")
            s[m] = c * (-1) ** k * math.factorial(k) / (q2 + lam) ** (k + 1)
        return s

    def scale(c):
        s = np.zeros(n)
        s[0] = c
        return s
    return [x[n - 1] for x in _eval(dag, roots, leaf, _subset_conv, lambda a, b: a + b, scale)]


def expansion_eval(n, l, g, v, lam):
    """Per out line the root (n, 0, l, 0) from its monomial expansion (leaf
    Taylor coefficients; the expansion carries the factor l!)."""
    polys = fdgraph.root_polynomials(n, [(n, 0, l, 0)])
    out = {}
    for key, P in polys.items():
        tot = 0.0
        for mono, coef in P.items():
            t = float(coef)
            for var in mono:
                if var[0] == "G":
                    t *= g[var[1:4]]
                else:
                    t *= _v_series(*v[var[1]], lam, var[2])[var[2]]
            tot += t
        out[key[1]] = tot
    return out


def hyperdual_mul_pairs(l):
    """Brute-force count of the subset-convolution products (A, B disjoint
    subsets of l directions): the closed form is 3^l."""
    return sum(1 for a, b in itertools.product(range(1 << l), repeat=2) if a & b == 0)
