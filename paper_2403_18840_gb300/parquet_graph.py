"""Evaluation graph of the Dyson-Schwinger / parquet construction and its
operation count (Sec. II.B-C, Figs. parquet_graph and parquet_benchmark).

The construction of `parquet.py` is evaluated per sample as a graph of
shared nodes.  Each node is a group of sub-diagrams with the same order,
kind, external momenta and internal variables: its own loop momenta and
interaction-line times.  Each join takes a new loop momentum and hands
contiguous blocks of variables to its parts, in a fixed order: the join's
own loop first, then the left part, the right part and the two dressed
lines.  A node is a tensor over the times of the lines its external legs
sit on, because the bare lines that join it to other nodes depend on those
times.  Joins contract these indices.

The recursion runs over an algebra:

* `Scalar`: values are numbers, nodes are memoised, and every multiply and
  add in a node's evaluation is counted once.  This is the compact graph's
  N_op (leaves excluded, as in `fdgraph.contraction_ops`).
* `Expanded`: values are lists of weighted monomials over leaves
  ('G', momentum, from vertex, to vertex) and ('V', momentum, vertex,
  vertex).  The expansion is the plain sum over diagrams, each with the
  momentum routing the construction gives it.

Momenta are integer coefficient tuples over (k_ext, p_1, ..., p_n).  Each
interaction line l has time variable l; its two ends are vertices 2l and
2l + 1.
"""
import collections
import math
from fractions import Fraction

import numpy as np

from . import fdgraph
from . import parquet as P


def _vec(n, i=None):
    v = [0] * (n + 1)
    if i is not None:
        v[i] = 1
    return tuple(v)


def _add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def _sub(a, b):
    return tuple(x - y for x, y in zip(a, b))


class Scalar:
    """Numbers; multiplies and adds counted in `ops`."""

    def __init__(self, g0, v):
        self.g0, self.v = g0, v          # leaf functions: g0(mom, from_line, to_line), v(mom)
        self.ops = 0

    def index(self, vertex):
        return vertex // 2                # a node's tensor index: the line (its time)

    def leaf_g(self, mom, x, y):
        return self.g0(mom, x, y)

    def leaf_v(self, mom, a, b):
        return self.v(mom)

    def one(self):
        return 1.0

    def mul(self, *xs):
        r = xs[0]
        for x in xs[1:]:
            r = r * x
        self.ops += len(xs) - 1
        return r

    def scale(self, w, x):
        if w == 1:
            return x
        self.ops += 1
        return float(w) * x

    def acc(self, d, key, x):
        if key in d:
            d[key] = d[key] + x
            self.ops += 1
        else:
            d[key] = x


class DerivativeCount:
    """Operation counts of derivatives in the screening shift Lambda, which
    enters through the interaction leaves only: values are True when they
    depend on Lambda.  Taylor mode to order L (mode 'taylor') or forward
    mode nested L times (mode 'nested'), with the costs of `adcount`: a
    product of two dependent values (L + 1)^2 or 2 3^L - 2^L, a product with
    an independent value L + 1 or 2^L, a sum of two dependent values L + 1 or
    2^L, anything else 1; each distinct interaction leaf L (its series)."""

    def __init__(self, L, mode):
        self.L = L
        if mode == "taylor":
            self.dd, self.di, self.add = (L + 1) ** 2, L + 1, L + 1
        else:
            self.dd, self.di, self.add = 2 * 3 ** L - 2 ** L, 2 ** L, 2 ** L
        self.ops = 0
        self.v_leaves = set()

    def index(self, vertex):
        return vertex // 2

    def leaf_g(self, mom, x, y):
        return False

    def leaf_v(self, mom, a, b):
        self.v_leaves.add(mom)
        return True

    def one(self):
        return False

    def mul(self, *xs):
        r = xs[0]
        for x in xs[1:]:
            self.ops += self.dd if (r and x) else self.di if (r or x) else 1
            r = r or x
        return r

    def scale(self, w, x):
        if w == 1:
            return x
        self.ops += self.di if x else 1
        return x

    def acc(self, d, key, x):
        if key in d:
            self.ops += self.add if (d[key] and x) else 1
            d[key] = d[key] or x
        else:
            d[key] = x

    def total(self):
        return self.ops + len(self.v_leaves) * self.L


class Series:
    """Truncated Taylor series in the screening shift Lambda (numpy arrays of
    length L + 1): the interaction leaves carry c / (q^2 + Lambda) expanded
    at lam, everything else is constant in Lambda.  v(mom) returns (c, q^2)."""

    def __init__(self, g0, v, lam, L):
        self.np, self.g0, self.v, self.lam, self.L = np, g0, v, lam, L

    def index(self, vertex):
        return vertex // 2

    def _const(self, x):
        s = self.np.zeros(self.L + 1)
        s[0] = x
        return s

    def leaf_g(self, mom, x, y):
        return self._const(self.g0(mom, x, y))

    def leaf_v(self, mom, a, b):
        c, q2 = self.v(mom)
        r = 1.0 / (q2 + self.lam)
        return self.np.array([c * r * (-r) ** k for k in range(self.L + 1)])

    def one(self):
        return self._const(1.0)

    def mul(self, *xs):
        r = xs[0]
        for x in xs[1:]:
            r = self.np.array([sum(r[i] * x[k - i] for i in range(k + 1)) for k in range(self.L + 1)])
        return r

    def scale(self, w, x):
        return float(w) * x

    def acc(self, d, key, x):
        d[key] = d[key] + x if key in d else x


def _support(kind, D):
    """Exponents (i, j) of mu^i Lambda^j a series of this kind carries to total degree D."""
    if kind == "const":
        return frozenset({(0, 0)})
    if kind == "mu":
        return frozenset((i, 0) for i in range(D + 1))
    if kind == "lam":
        return frozenset((0, j) for j in range(D + 1))
    return frozenset((i, j) for i in range(D + 1) for j in range(D + 1 - i))


class BiSeries:
    """Truncated Taylor series in (mu, Lambda) to total degree D, as dicts
    {(i, j): coefficient}: the bare lines depend on mu, the interaction lines
    on Lambda.  g0(mom, x, y, i) is the i-th mu-Taylor coefficient of a bare
    line, v(mom) = (c, q^2) an interaction c / (q^2 + Lambda) at lam."""

    def __init__(self, g0, v, lam, D):
        self.g0, self.v, self.lam, self.D = g0, v, lam, D

    def index(self, vertex):
        return vertex // 2

    def leaf_g(self, mom, x, y):
        return {(i, 0): self.g0(mom, x, y, i) for i in range(self.D + 1)}

    def leaf_v(self, mom, a, b):
        c, q2 = self.v(mom)
        r = 1.0 / (q2 + self.lam)
        return {(0, j): c * r * (-r) ** j for j in range(self.D + 1)}

    def one(self):
        return {(0, 0): 1.0}

    def mul(self, *xs):
        r = xs[0]
        for x in xs[1:]:
            out = {}
            for (i1, j1), a in r.items():
                for (i2, j2), b in x.items():
                    if i1 + i2 + j1 + j2 <= self.D:
                        k = (i1 + i2, j1 + j2)
                        out[k] = out.get(k, 0.0) + a * b
            r = out
        return r

    def scale(self, w, x):
        return {k: float(w) * v for k, v in x.items()}

    def acc(self, d, key, x):
        if key in d:
            y = dict(d[key])
            for k, v in x.items():
                y[k] = y.get(k, 0.0) + v
            d[key] = y
        else:
            d[key] = x


class BiTaylorCount:
    """Operation count of Taylor mode in (mu, Lambda) to total degree D (all
    counterterm orders of one Sigma^(n) at once): values are the exponent
    supports; a product costs one multiply per pair of exponents within the
    degree plus the adds that merge equal exponents, a sum one add per common
    exponent.  Leaves excluded, as in `fdgraph.contraction_ops`."""

    def __init__(self, D):
        self.D = D
        self.ops = 0

    def index(self, vertex):
        return vertex // 2

    def leaf_g(self, mom, x, y):
        return _support("mu", self.D)

    def leaf_v(self, mom, a, b):
        return _support("lam", self.D)

    def one(self):
        return _support("const", self.D)

    def mul(self, *xs):
        r = xs[0]
        for x in xs[1:]:
            pairs = [(a[0] + b[0], a[1] + b[1]) for a in r for b in x if sum(a) + sum(b) <= self.D]
            out = frozenset(pairs)
            self.ops += len(pairs) + (len(pairs) - len(out))
            r = out
        return r

    def scale(self, w, x):
        if w != 1:
            self.ops += len(x)
        return x

    def acc(self, d, key, x):
        if key in d:
            self.ops += len(d[key] & x)
            d[key] = d[key] | x
        else:
            d[key] = x


class DagEmit:
    """Emits Taylor mode in (mu, Lambda) to total degree D as nodes of a
    shared `fdgraph.DAG`, in the compiler's leaf vocabulary: ('G', mom,
    line_dst, line_src, i) for the i-th mu-coefficient of a bare line and
    ('V', mom, j) for the j-th Lambda-coefficient of an interaction line,
    momenta padded to the tape's order and taken up to overall sign.
    Values are {(i, j, e): node}; e = 1 is the first derivative in the
    external momentum (with dk: the leaves 'Gd' / 'Vd' of lines that carry
    k_ext, products by the Leibniz rule), e = 0 otherwise."""

    def __init__(self, dag, D, order, dk=False):
        self.dag, self.D, self.order, self.dk = dag, D, order, dk

    def index(self, vertex):
        return vertex // 2

    def _mom(self, mom):
        m = tuple(mom) + (0,) * (self.order + 1 - len(mom))
        return fdgraph._canon_mom(m)[0]

    def leaf_g(self, mom, x, y):
        cm = self._mom(mom)
        out = {(i, 0, 0): self.dag.var(("G", cm, y, x, i)) for i in range(self.D + 1)}
        if self.dk and cm[0] != 0:
            out.update({(i, 0, 1): self.dag.var(("Gd", cm, y, x, i)) for i in range(self.D + 1)})
        return out

    def leaf_v(self, mom, a, b):
        cm = self._mom(mom)
        out = {(0, j, 0): self.dag.var(("V", cm, j)) for j in range(self.D + 1)}
        if self.dk and cm[0] != 0:
            out.update({(0, j, 1): self.dag.var(("Vd", cm, j)) for j in range(self.D + 1)})
        return out

    def one(self):
        return {(0, 0, 0): self.dag.const(1.0)}

    def mul(self, *xs):
        r = xs[0]
        for x in xs[1:]:
            out = {}
            for (i1, j1, e1), a in sorted(r.items()):
                for (i2, j2, e2), b in sorted(x.items()):
                    if i1 + i2 + j1 + j2 > self.D or e1 + e2 > 1:
                        continue
                    k = (i1 + i2, j1 + j2, e1 + e2)
                    out[k] = self.dag.make("fma", a, b, out[k]) if k in out else self.dag.make("mul", a, b)
            r = out
        return r

    def scale(self, w, x):
        if w == 1:
            return x
        return {k: self.dag.make("mulc", u, float(w)) for k, u in x.items()}

    def acc(self, d, key, x):
        if key in d:
            y = dict(d[key])
            for k, u in x.items():
                y[k] = self.dag.make("add", y[k], u) if k in y else u
            d[key] = y
        else:
            d[key] = x


def parquet_outputs(order, roots, construction=None, share="root"):
    """(dag, outputs) for roots [(n, m, l, dk)] of an order-`order` tape from
    the Dyson-Schwinger / parquet graphs: Sigma^(n) in Taylor mode to total
    degree order - n (and first order in k_ext when any root has dk), root
    (n, m, l, dk) = m! l! times the (m, l, dk) coefficient, one output per
    out line.  share: "root" (default) builds each root's graph on its own
    (products and sums shared within the root only, as the compiler's own
    tapes do; each root keeps only the Taylor coefficients it needs, so its
    leaf families stay narrow and its temporaries die with it), "n" shares
    within the roots of one Sigma^(n), "all" across every root."""
    C = construction or P.Construction()
    dag = fdgraph.DAG()
    with_dk = any(r[3] for r in roots)
    series = {}
    outputs = []
    for r, (n, m, l, dk) in enumerate(roots):
        scope = {"root": (n, r), "n": n, "all": None}[share]
        if (n, scope) not in series:
            dag.scope = scope
            series[(n, scope)] = Evaluator(n, DagEmit(dag, order - n, order, with_dk), C).root()
        for o, coefs in sorted(series[(n, scope)].items()):
            if (m, l, dk) not in coefs:
                continue
            node = coefs[(m, l, dk)]
            f = math.factorial(m) * math.factorial(l)
            if f != 1:
                node = dag.make("mulc", node, float(f))
            outputs.append((r, o, node))
    return dag, outputs


def parquet_tape(order, roots, budget=96, bundle=4, window=32, construction=None, share="root"):
    """The parquet graphs of the roots compiled into the tape format."""
    dag, outputs = parquet_outputs(order, roots, construction, share)
    return fdgraph.compile_dag(order, roots, dag, outputs, budget, bundle, window)


class Expanded:
    """Weighted monomials over vertex-level leaves."""

    def index(self, vertex):
        return vertex

    def leaf_g(self, mom, x, y):
        return [(Fraction(1), (("G", mom, x, y),))]

    def leaf_v(self, mom, a, b):
        return [(Fraction(1), (("V", mom, a, b),))]

    def one(self):
        return [(Fraction(1), ())]

    def mul(self, *xs):
        out = [(Fraction(1), ())]
        for x in xs:
            out = [(w1 * w2, m1 + m2) for (w1, m1) in out for (w2, m2) in x]
        return out

    def scale(self, w, x):
        return [(w * c, m) for (c, m) in x]

    def acc(self, d, key, x):
        d.setdefault(key, []).extend(x)


DIRECT, EXCHANGED = 0, 1       # a 4-point piece's fermion paths: in1 -> out1, or in1 -> out2
LOOP = -2                      # a closed fermion loop: its sign and its spin sum


def path_class(piece):
    """(DIRECT or EXCHANGED, closed fermion loops inside) of a 4-point piece."""
    succ, pred, _ = piece
    v = pred.index(-1)
    on_path = set()
    while True:
        on_path.add(v)
        if succ[v] < 0:
            cls = DIRECT if succ[v] == -1 else EXCHANGED
            break
        v = succ[v]
    v = pred.index(-2)
    while True:
        on_path.add(v)
        if succ[v] < 0:
            break
        v = succ[v]
    loops, seen = 0, set(on_path)
    for s0 in range(len(succ)):
        if s0 in seen:
            continue
        loops += 1
        v = s0
        while v not in seen:
            seen.add(v)
            v = succ[v]
    return cls, loops


def route_piece(piece, leg_moms, n_var, ms, line_of):
    """Momentum routing of one diagram piece: leg momenta given
    ({('in'|'out', j): mom}), chords of a spanning tree carry the loop
    variables ms, ms+1, ..., tree lines follow from conservation.  Returns
    the leaves [('G', mom, x, y) / ('V', mom, a, b)] with vertices mapped by
    line_of (piece vertex -> global vertex)."""
    succ, pred, partner = piece
    nv = len(succ)
    edges = [("G", v, succ[v]) for v in range(nv) if succ[v] >= 0]
    edges += [("V", v, partner[v]) for v in range(nv) if 0 <= v < partner[v]]
    parent = list(range(nv))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    tree, chords = [], []
    for e in edges:
        ra, rb = find(e[1]), find(e[2])
        if ra != rb:
            parent[ra] = rb
            tree.append(e)
        else:
            chords.append(e)
    mom = {}
    for k, e in enumerate(chords):
        mom[e] = _vec(n_var, ms + k)
    # net momentum entering each vertex from legs and known lines
    need = [_vec(n_var) for _ in range(nv)]
    legs = P._leg_vertices(piece)
    for (kind, j), v in legs.items():
        m = leg_moms[(kind, j)]
        need[v] = _add(need[v], m) if kind == "in" else _sub(need[v], m)
    for e, m in mom.items():
        need[e[1]] = _sub(need[e[1]], m)
        need[e[2]] = _add(need[e[2]], m)
    rest = list(tree)
    while rest:
        deg = collections.Counter()
        for e in rest:
            deg[e[1]] += 1
            deg[e[2]] += 1
        for e in rest:
            a, b = e[1], e[2]
            if deg[a] == 1:           # a's balance fixes e (leaving a)
                m = need[a]
                mom[e] = m
                need[a] = _sub(need[a], m)
                need[b] = _add(need[b], m)
                rest.remove(e)
                break
            if deg[b] == 1:           # b's balance fixes e (entering b)
                m = _vec(n_var)
                m = _sub(m, need[b])
                mom[e] = m
                need[b] = _add(need[b], m)
                need[a] = _sub(need[a], m)
                rest.remove(e)
                break
    leaves = []
    for e, m in mom.items():
        leaves.append((e[0], m, line_of(e[1]), line_of(e[2])))
    return leaves


class Evaluator:
    """The construction as a recursion over an algebra (Scalar or Expanded),
    memoised on (node, arguments)."""

    def __init__(self, order, alg, construction=None):
        self.n = order
        self.alg = alg
        self.C = construction or P.Construction()
        self.memo = {}

    def _m(self, key, fn):
        if key not in self.memo:
            self.memo[key] = fn()
        return self.memo[key]

    # a dressed line from vertex x to vertex y, momentum K, k orders of insertions
    # x, y, and every tensor key below, are vertex indices of the algebra
    # (lines for Scalar, vertices for Expanded)
    def chain(self, k, K, x, y, ms, ts):
        return self._m(("chain", k, K, x, y, ms, ts), lambda: self._chain(k, K, x, y, ms, ts))

    def _chain(self, k, K, x, y, ms, ts):
        A = self.alg
        if k == 0:
            return A.leaf_g(K, x, y)
        # G0(x -> first insertion) times the rest, which does not depend on x
        return A.mul(A.leaf_g(K, x, A.index(2 * ts)), self.chain_tail(k, K, y, ms, ts))

    def chain_tail(self, k, K, y, ms, ts):
        """sum over the first insertion Sigma^(p) and its out-vertex o of
        Sigma^(p)[o] times the dressed line of order k - p from o to y."""
        return self._m(("tail", k, K, y, ms, ts), lambda: self._chain_tail(k, K, y, ms, ts))

    def _chain_tail(self, k, K, y, ms, ts):
        A = self.alg
        out = {}
        for p in range(1, k + 1):
            for o, s in self.sigma(p, K, ms, ts).items():
                A.acc(out, 0, A.mul(s, self.chain(k - p, K, o, y, ms + p, ts + p)))
        return out[0]

    # Sigma^(N)(K) over its out-vertex; in-vertex 2 ts, loop q = ms
    def sigma(self, N, K, ms, ts):
        return self._m(("sigma", N, K, ms, ts), lambda: self._sigma(N, K, ms, ts))

    def _sigma(self, N, K, ms, ts):
        A = self.alg
        q = _vec(self.n, ms)
        a, b = A.index(2 * ts), A.index(2 * ts + 1)
        out = {}
        for i in range(N):
            # the loop momentum runs on the bare line into Gamma3, the
            # interaction line a -> b carries the rest
            g3 = self.gamma3(i, q, K, ms + 1, ts + 1, b)
            vline = {x: A.mul(A.leaf_v(_sub(K, q), a, b), self.chain(N - i - 1, q, a, x, ms + 1 + i, ts + 1 + i))
                     for x in {x for (x, _) in g3}}
            for (x, o), val in g3.items():
                A.acc(out, o, A.mul(vline[x], val))
        return out

    # Gamma3 over (in-vertex, out-vertex); b its interaction end (outside)
    def gamma3(self, N, Kin, Kout, ms, ts, b):
        return self._m(("g3", N, Kin, Kout, ms, ts, b), lambda: self._gamma3(N, Kin, Kout, ms, ts, b))

    def _gamma3(self, N, Kin, Kout, ms, ts, b):
        A = self.alg
        if N == 0:
            return {(b, b): A.one()}                 # the bare vertex: b itself
        # b takes in the boson momentum Kout - Kin; Gamma4 legs (in1, out1, in2, out2)
        p = _vec(self.n, ms)
        out = {}
        for i in range(N):
            M = N - i - 1
            legs = (Kin, Kout, _add(p, _sub(Kout, Kin)), p)
            g4 = self.gamma4(i, legs, ms + 1, ts, None)
            m1, t1 = ms + 1 + i, ts + i + 1
            pairs = {(u, w) for (_, _, _, u, w) in g4}
            bubble = {}                          # [G G]^(M) from b to u and from w back to b
            for (u, w) in pairs:
                for j in range(M + 1):
                    A.acc(bubble, (u, w), A.mul(self.chain(j, legs[2], b, u, m1, t1),
                                                self.chain(M - j, legs[3], w, b, m1 + j, t1 + j)))
            # a direct vertex (in2 -> out2) closes a fermion loop through b: -2
            loop, through = {}, {}
            for (cls, x, o, u, w), val in g4.items():
                A.acc(loop if cls == DIRECT else through, (x, o), A.mul(val, bubble[(u, w)]))
            for k, v in loop.items():
                A.acc(out, k, A.scale(LOOP, v))
            for k, v in through.items():
                A.acc(out, k, v)
        return out

    # Gamma4 over (in1, out1, in2, out2) vertices; irr: None, 'ph' or 'pp'
    def gamma4(self, N, legs, ms, ts, irr):
        return self._m(("g4", N, legs, ms, ts, irr), lambda: self._gamma4(N, legs, ms, ts, irr))

    def _gamma4(self, N, legs, ms, ts, irr):
        A = self.alg
        out = {}
        for k, v in self.irreducible(N, legs, ms, ts).items():
            A.acc(out, k, v)
        for c in ("ph", "phbar", "pp"):
            if irr == "ph" and c == "ph":
                continue
            if irr == "pp" and c == "pp":
                continue
            for k, v in self.phi(c, N, legs, ms, ts).items():
                A.acc(out, k, v)
        return out

    def irreducible(self, N, legs, ms, ts):
        return self._m(("irr", N, legs, ms, ts), lambda: self._irreducible(N, legs, ms, ts))

    def _irreducible(self, N, legs, ms, ts):
        A = self.alg
        K1, K3, K2, K4 = legs
        out = {}
        if N == 0:
            a, b = A.index(2 * ts), A.index(2 * ts + 1)
            A.acc(out, (DIRECT, a, a, b, b), A.leaf_v(_sub(K1, K3), a, b))
            A.acc(out, (EXCHANGED, a, b, b, a), A.leaf_v(_sub(K1, K4), a, b))
            return out
        leg_moms = {("in", 0): K1, ("out", 0): K3, ("in", 1): K2, ("out", 1): K4}
        polys = {}
        for key, w in self.C.irreducible(N).items():
            piece = P.from_key(key)
            # the piece's interaction lines in order of first vertex -> lines ts, ts+1, ...
            succ, pred, partner = piece
            lines = {}
            for v in range(len(succ)):
                lo = min(v, partner[v])
                if lo not in lines:
                    lines[lo] = len(lines)
            glob = {v: 2 * (ts + lines[min(v, partner[v])]) + (0 if v < partner[v] else 1) for v in range(len(succ))}
            leaves = route_piece(piece, leg_moms, self.n, ms, lambda v: A.index(glob[v]))
            lg = P._leg_vertices(piece)
            cls, loops = path_class(piece)
            idx = (cls,) + tuple(A.index(glob[lg[k]]) for k in (("in", 0), ("out", 0), ("in", 1), ("out", 1)))
            poly = polys.setdefault(idx, {})
            mono = tuple(sorted(leaves))
            poly[mono] = poly.get(mono, 0) + w * LOOP ** loops
        # the node's diagrams factorised together (greedy Horner, hash-consed)
        dag = fdgraph.DAG()
        dag.scope = None
        memo = {}
        for idx, poly in polys.items():
            A.acc(out, idx, self._dag_value(dag, fdgraph.horner(dag, poly), memo))
        return out

    def _dag_value(self, dag, u, memo):
        if u in memo:
            return memo[u]
        A = self.alg
        node = dag.nodes[u]
        kind = node[0]
        if kind == "var":
            kd, m, x, y = node[1]
            val = A.leaf_g(m, x, y) if kd == "G" else A.leaf_v(m, x, y)
        elif kind == "mul":
            val = A.mul(self._dag_value(dag, node[1], memo), self._dag_value(dag, node[2], memo))
        elif kind == "mulc":
            val = A.scale(node[2], self._dag_value(dag, node[1], memo))
        elif kind in ("add", "fma"):
            if kind == "add":
                first = self._dag_value(dag, node[1], memo)
                second = self._dag_value(dag, node[2], memo)
            else:
                first = A.mul(self._dag_value(dag, node[1], memo), self._dag_value(dag, node[2], memo))
                second = self._dag_value(dag, node[3], memo)
            d = {}
            A.acc(d, 0, first)
            A.acc(d, 0, second)
            val = d[0]
        else:
            raise ValueError("unexpected node %r" % (node,))
        memo[u] = val
        return val

    def phi(self, c, N, legs, ms, ts):
        return self._m(("phi", c, N, legs, ms, ts), lambda: self._phi(c, N, legs, ms, ts))

    def _phi(self, c, N, legs, ms, ts):
        A = self.alg
        out = {}
        if N == 0:
            return out
        K1, K3, K2, K4 = legs
        if c == "phbar":
            # the ph join with the composite's out-legs exchanged
            inner = self.phi("ph", N, (K1, K4, K2, K3), ms, ts)
            return {(1 - cls, a, d, cc, b): v for (cls, a, b, cc, d), v in inner.items()}
        p = _vec(self.n, ms)
        half = Fraction(1, 2) if c == "pp" else Fraction(1)
        for i in range(N):
            for j in range(N - i):
                for k in range(N - i - j):
                    l = N - 1 - i - j - k
                    mL, tL = ms + 1, ts
                    mR, tR = mL + i, tL + i + 1
                    m1, t1 = mR + j, tR + j + 1
                    m2, t2 = m1 + k, t1 + k
                    if c == "ph":
                        P1, P2 = p, _add(p, _sub(K3, K1))
                        L = self.gamma4(i, (K1, K3, P2, P1), mL, tL, None)
                        R = self.gamma4(j, (P1, P2, K2, K4), mR, tR, "ph")
                        # L[a,b,x,y] G(y->u) G(v->x) R[u,v,c,d]
                        us = {u for (_, u, _, _, _) in R}
                        vs = {v for (_, _, v, _, _) in R}
                        M1 = {}
                        for (cl, a, b, x, y), lv in L.items():
                            for u in us:
                                A.acc(M1, (cl, a, b, x, u), A.mul(lv, self.chain(k, P1, y, u, m1, t1)))
                        M2 = {}
                        for (cl, a, b, x, u), mv in M1.items():
                            for v in vs:
                                A.acc(M2, (cl, a, b, u, v), A.mul(mv, self.chain(l, P2, v, x, m2, t2)))
                        # both direct: L.in2 -> L.out2 -> R.in1 -> R.out1 -> L.in2 is a loop (-2);
                        # both exchanged: exchanged; otherwise direct.  A direct L
                        # therefore meets -2 R_direct + R_exchanged (formed once)
                        rd = {}
                        for (cr, u, v, cc, d), rv in R.items():
                            A.acc(rd, (u, v, cc, d), A.scale(LOOP, rv) if cr == DIRECT else rv)
                        for (cl, a, b, u, v), nv in M2.items():
                            if cl == DIRECT:
                                for (u2, v2, cc, d), rv in rd.items():
                                    if (u2, v2) == (u, v):
                                        A.acc(out, (DIRECT, a, b, cc, d), A.mul(nv, rv))
                            else:
                                for (cr, u2, v2, cc, d), rv in R.items():
                                    if (u2, v2) == (u, v):
                                        A.acc(out, (cr, a, b, cc, d), A.mul(nv, rv))
                    else:
                        P1, P2 = p, _sub(_add(K1, K2), p)
                        L = self.gamma4(i, (K1, P1, K2, P2), mL, tL, None)
                        R = self.gamma4(j, (P1, K3, P2, K4), mR, tR, "pp")
                        # L[a,x,b,y] G(x->u) G(y->v) R[u,c,v,d] / 2; no loop forms,
                        # the composite is exchanged when exactly one part is
                        us = {u for (_, u, _, _, _) in R}
                        vs = {v for (_, _, _, v, _) in R}
                        M1 = {}
                        for (cl, a, x, b, y), lv in L.items():
                            for u in us:
                                A.acc(M1, (cl, a, b, y, u), A.mul(lv, self.chain(k, P1, x, u, m1, t1)))
                        M2 = {}
                        for (cl, a, b, y, u), mv in M1.items():
                            for v in vs:
                                A.acc(M2, (cl, a, b, u, v), A.mul(mv, self.chain(l, P2, y, v, m2, t2)))
                        for (cr, u, cc, v, d), rv in R.items():
                            for (cl, a, b, u2, v2), nv in M2.items():
                                if (u2, v2) == (u, v):
                                    A.acc(out, (cl ^ cr, a, cc, b, d), A.scale(half, A.mul(nv, rv)))
        return out

    def root(self):
        """Sigma^(n)(k_ext) over its out-vertex (index), with the sign
        (-1)^n of its n interaction lines (the loops' -2 are inside)."""
        out = self.sigma(self.n, _vec(self.n, 0), 1, 0)
        if self.n % 2 == 0:
            return out
        return {k: self.alg.scale(-1, v) for k, v in out.items()}
