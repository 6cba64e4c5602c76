"""Self-energy diagrams built bottom-up from the Dyson-Schwinger and parquet
equations (Sec. II.B-C: Eqs. Dyson, sigma_pq, vertex3, parquet_eqns and
phi_ph - phi_pp; the cycle of Fig. graph_construct).

Diagrams are topologies of instantaneous interaction lines and bare fermion
lines (the same objects the enumerator of `fdgraph` produces), held as
*pieces* with labelled external legs:

* a 4-point vertex Gamma4 has two incoming legs (in1, in2) and two outgoing
  legs (out1, out2), amputated (no self-energy insertion on a leg) and
  connected; all leg assignments are distinct diagrams (no antisymmetrised
  vertices), so the bare vertex of order 0 is two diagrams, the interaction
  line with the legs paired directly (in1 -> out1 at one end) or exchanged
  (in1 -> out2);
* a 3-point vertex Gamma3 has a fermion in-leg, a fermion out-leg and one
  interaction end b whose partner is outside;
* a self-energy Sigma has one in-leg and one out-leg.

The order of a piece is its number of interaction lines for Sigma and
Gamma3, and that number minus one for Gamma4 (the bare vertex is order 0).

The equations, in these terms (each diagram must come out exactly once):

* G^(k): a bare line dressed by a chain of self-energy insertions of total
  order k (Dyson).
* Sigma^(N) = sum_i V G^(N-i-1) Gamma3^(i): a new vertex a (the external
  in-leg) whose interaction partner is Gamma3's end b and whose line runs
  through a dressed line into Gamma3.
* Gamma3^(N) = sum_i Gamma4^(i) [G G]^(N-i-1): a new vertex b whose out-line
  runs (dressed) into Gamma4's in2 and whose in-line comes (dressed) from
  Gamma4's out2; Gamma3's legs are Gamma4's in1 and out1.  Gamma3^(0) is the
  bare vertex.
* Gamma4^(N) = I^(N) + Phi^ph + Phi^phbar + Phi^pp.  A channel splits the four
  legs into two pairs, ph: {in1, out1 | in2, out2}, phbar: {in1, out2 | in2,
  out1}, pp: {in1, in2 | out1, out2}; a diagram is reducible in a channel
  when cutting two bare lines separates the pairs, and in at most one
  channel.  Phi^c = sum over i+j+k+l = N-1 of L in Gamma4^(i) joined to
  R in Gamma4_c^(j) (R irreducible in the channel of the join, as seen by
  its own legs) through two dressed lines of orders k and l:
  ph: L.out2 -> R.in1 and R.out1 -> L.in2, legs (L.in1, L.out1, R.in2,
  R.out2); phbar: the same join with the composite's out-legs exchanged;
  pp: L.out1 -> R.in1 and L.out2 -> R.in2, legs (L.in1, R.out1, L.in2,
  R.out2), with weight 1/2 (each diagram arises from both assignments of
  the two parallel lines to L's out-legs).  Choosing R irreducible makes the
  join unique (the cut nearest R's external legs).
* I^(N), the fully irreducible vertex: the bare vertex at order 0; above it,
  the order-N vertices that no channel's reducible part contains, found by
  enumerating all order-N vertices (none at orders 1 and 2, the 64 envelope
  diagrams at order 3).  The paper builds I bottom-up as well (Fig.
  envelope_diag) but only sketches the rule, so the remainder stands in.

Multiplicities are carried as exact fractions; every generated diagram must
end with weight 1, which the tests check against the enumerator.
"""
import collections
import functools
import itertools
from fractions import Fraction

# A piece is a tuple (succ, pred, partner) of equal-length tuples over its
# vertices.  succ[v]: the vertex v's fermion line runs to, or -(j+1) for the
# out-leg j; pred[v]: the vertex whose line runs into v, or -(j+1) for the
# in-leg j; partner[v]: the other end of v's interaction line, or -1 for
# Gamma3's open end.


def _dfs_order(succ, pred, partner, start):
    order, seen, stack = [], set(), [start]
    while stack:
        v = stack.pop()
        if v < 0 or v in seen:
            continue
        seen.add(v)
        order.append(v)
        # explored in the order succ, pred, partner (pushed in reverse)
        stack.append(partner[v])
        stack.append(pred[v])
        stack.append(succ[v])
    return order


def canonical(piece):
    """Canonical key of a connected piece: vertices relabelled in a depth-first
    order from the in-leg 1 vertex that depends only on the structure, so
    two pieces are isomorphic (legs fixed) exactly when their keys agree.
    None if the piece is not connected."""
    succ, pred, partner = piece
    start = pred.index(-1)
    order = _dfs_order(succ, pred, partner, start)
    if len(order) != len(succ):
        return None
    lab = {v: k for k, v in enumerate(order)}

    def enc(w):
        return lab[w] if w >= 0 else w
    return tuple((enc(succ[v]), enc(pred[v]), enc(partner[v])) for v in order)


def from_key(key):
    """The piece of a canonical key (its vertices in canonical order)."""
    return (tuple(k[0] for k in key), tuple(k[1] for k in key), tuple(k[2] for k in key))


# ---- structural tests -------------------------------------------------------

def _components(n, edges):
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for a, b in edges:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    return [find(a) for a in range(n)]


def _lines(piece):
    succ, pred, partner = piece
    g = [(v, succ[v]) for v in range(len(succ)) if succ[v] >= 0]
    vl = {(min(v, partner[v]), max(v, partner[v])) for v in range(len(succ)) if partner[v] >= 0}
    return g, sorted(vl)


def _leg_vertices(piece):
    """{('in', j) or ('out', j): vertex}."""
    succ, pred, _ = piece
    legs = {}
    for v in range(len(succ)):
        if succ[v] < 0:
            legs[("out", -succ[v] - 1)] = v
        if pred[v] < 0:
            legs[("in", -pred[v] - 1)] = v
    return legs


def amputated(piece):
    """No bare line is a bridge (a bridge would isolate a self-energy
    insertion on a leg)."""
    g, vl = _lines(piece)
    n = len(piece[0])
    for e in g:
        rest = [x for x in g if x != e] + vl
        comp = _components(n, rest)
        if len(set(comp)) > 1:
            return False
    return True


def tadpole_free(piece):
    """No interaction line whose removal leaves a part without legs (such a
    line carries zero momentum)."""
    g, vl = _lines(piece)
    n = len(piece[0])
    legs = _leg_vertices(piece)
    for e in vl:
        comp = _components(n, g + [x for x in vl if x != e])
        with_legs = {comp[v] for v in legs.values()}
        if set(comp) - with_legs:
            return False
    return True


CHANNELS = {"ph": ({("in", 0), ("out", 0)}, {("in", 1), ("out", 1)}),
            "phbar": ({("in", 0), ("out", 1)}, {("in", 1), ("out", 0)}),
            "pp": ({("in", 0), ("in", 1)}, {("out", 0), ("out", 1)})}


def reducible(piece, channel):
    """Gamma4 reducible in `channel`: two bare lines whose cut separates the
    channel's two leg pairs into two connected parts."""
    g, vl = _lines(piece)
    n = len(piece[0])
    legs = _leg_vertices(piece)
    left, right = CHANNELS[channel]
    for e1, e2 in itertools.combinations(g, 2):
        comp = _components(n, [x for x in g if x != e1 and x != e2] + vl)
        if len(set(comp)) != 2:
            continue
        cl = {comp[legs[x]] for x in left}
        cr = {comp[legs[x]] for x in right}
        if len(cl) == 1 and len(cr) == 1 and cl != cr:
            return True
    return False


# ---- brute force (the check, and the fully irreducible vertex) ---------------

def brute_gamma4(n_lines):
    """All connected, amputated, tadpole-free 4-point vertices with n_lines
    interaction lines (every leg assignment distinct): {key: piece}."""
    nv = 2 * n_lines
    X1, X2 = nv, nv + 1
    partner = tuple(v ^ 1 for v in range(nv))
    out = {}
    for perm in itertools.permutations(range(nv + 2)):
        if perm[X1] >= nv or perm[X2] >= nv:
            continue                                  # a leg runs straight to a leg
        succ = tuple(-1 if perm[v] == X1 else -2 if perm[v] == X2 else perm[v] for v in range(nv))
        pred = [0] * nv
        for v in range(nv):
            if succ[v] >= 0:
                pred[succ[v]] = v
        pred[perm[X1]] = -1
        pred[perm[X2]] = -2
        piece = (succ, tuple(pred), partner)
        key = canonical(piece)
        if key is None or key in out:
            continue
        p = from_key(key)
        if amputated(p) and tadpole_free(p):
            out[key] = p
    return out


def enumerate_gamma4(n_lines):
    """The same set as brute_gamma4, built by following fermion lines: from
    in-leg 1's vertex, each step sends the current vertex's line to an out-leg,
    to a vertex already named (the free end of an introduced interaction
    line) or to the first end of a new interaction line; a finished path or
    loop continues at in-leg 2's vertex (any named or new vertex) and then at
    the smallest named vertex not yet passed.  Duplicates are removed by the
    canonical key."""
    nv = 2 * n_lines
    succ = [None] * nv
    pred = [None] * nv
    partner = tuple(v ^ 1 for v in range(nv))
    out = {}

    def finish():
        piece = (tuple(succ), tuple(pred), partner)
        key = canonical(piece)
        if key is not None and key not in out:
            p = from_key(key)
            if amputated(p) and tadpole_free(p):
                out[key] = p

    def named_free(nl):
        return [w for w in range(2 * nl) if pred[w] is None]

    def next_start(nl, outs_used, in2_done):
        """Continue after a path or loop ends."""
        if not in2_done:
            cands = named_free(nl) + ([2 * nl] if nl < n_lines else [])
            for w in cands:
                nl2 = nl + 1 if w == 2 * nl else nl
                pred[w] = -2
                walk(w, nl2, outs_used, True, None)
                pred[w] = None
            return
        free = [w for w in range(2 * nl) if pred[w] is None]
        if not free:
            if nl == n_lines and len(outs_used) == 2:
                finish()
            return
        st = free[0]
        walk(st, nl, outs_used, True, st)

    def walk(v, nl, outs_used, in2_done, loop_start):
        # v has its pred set (or is a loop start); choose succ[v]
        choices = []
        if loop_start is None:
            choices += [-(j + 1) for j in (0, 1) if (j not in outs_used)]
        for w in range(2 * nl):
            if pred[w] is None and w != loop_start:
                choices.append(w)
        if loop_start is not None:
            choices.append(loop_start)
        if nl < n_lines:
            choices.append(2 * nl)
        for w in choices:
            if w < 0:
                succ[v] = w
                next_start(nl, outs_used | {-w - 1}, in2_done)
                succ[v] = None
                continue
            nl2 = nl + 1 if (nl < n_lines and w == 2 * nl) else nl
            succ[v] = w
            if w == loop_start:
                pred[w] = v
                next_start(nl2, outs_used, in2_done)
                pred[w] = None
            else:
                pred[w] = v
                walk(w, nl2, outs_used, in2_done, loop_start)
                pred[w] = None
            succ[v] = None

    pred[0] = -1
    walk(0, 1, frozenset(), False, None)
    return out


def irreducible_remainder(N, reducible_parts):
    """I^(N): the order-N vertices (N + 1 interaction lines, enumerated) that
    no channel's reducible part contains.  The reducible parts must cover each
    of their diagrams exactly once and only enumerated diagrams."""
    full = enumerate_gamma4(N + 1)
    red = collections.defaultdict(Fraction)
    for part in reducible_parts:
        for k, w in part.items():
            red[k] += w
    assert all(w == 1 for w in red.values()) and set(red) <= set(full)
    return {k: Fraction(1) for k in full if k not in red}


# ---- joining pieces ------------------------------------------------------------

class _Builder:
    """Disjoint union of pieces; open legs are joined by bare lines or
    declared legs of the result."""

    def __init__(self):
        self.succ, self.pred, self.partner = [], [], []

    def vertex(self):
        self.succ.append(None)
        self.pred.append(None)
        self.partner.append(None)
        return len(self.succ) - 1

    def add(self, piece):
        """Add a piece; returns (ins, outs, open_end) with its leg vertices."""
        off = len(self.succ)
        succ, pred, partner = piece
        ins, outs, end = {}, {}, None
        for v in range(len(succ)):
            s, p, q = succ[v], pred[v], partner[v]
            self.succ.append(s + off if s >= 0 else None)
            self.pred.append(p + off if p >= 0 else None)
            self.partner.append(q + off if q >= 0 else None)
            if s < 0:
                outs[-s - 1] = v + off
            if p < 0:
                ins[-p - 1] = v + off
            if q < 0:
                end = v + off
        return ins, outs, end

    def line(self, u, w):
        assert self.succ[u] is None and self.pred[w] is None
        self.succ[u] = w
        self.pred[w] = u

    def dressed(self, u, w, chain):
        """A bare line from u to w with the self-energy insertions of chain."""
        for s in chain:
            ins, outs, _ = self.add(s)
            self.line(u, ins[0])
            u = outs[0]
        self.line(u, w)

    def piece(self):
        assert None not in self.succ and None not in self.pred and None not in self.partner
        return (tuple(self.succ), tuple(self.pred), tuple(self.partner))


def _mark(b, v, kind, j):
    if kind == "in":
        assert b.pred[v] is None
        b.pred[v] = -(j + 1)
    else:
        assert b.succ[v] is None
        b.succ[v] = -(j + 1)


def _swap_outs(piece):
    succ, pred, partner = piece
    sw = {-1: -2, -2: -1}
    return (tuple(sw.get(s, s) for s in succ), pred, partner)


def _add_to(acc, piece, w):
    key = canonical(piece)
    assert key is not None
    acc[key] += w


# ---- the equations ---------------------------------------------------------------

def _memo(method):
    """Memoise a method on its instance (the cache dies with the instance)."""
    @functools.wraps(method)
    def wrapper(self, *args):
        cache = self.__dict__.setdefault("_cache", {})
        key = (method.__name__,) + args
        if key not in cache:
            cache[key] = method(self, *args)
        return cache[key]
    return wrapper


class Construction:
    """Pieces of every kind and order, built from lower orders and memoised:
    each a {canonical key: weight} multiset."""

    def __init__(self, irreducible=None):
        # fully irreducible vertex by order (order 0 is the bare vertex);
        # orders not given are found as the irreducible remainder
        self._irr = dict(irreducible or {})

    # Sigma^(N)
    @_memo
    def sigma(self, N):
        acc = collections.defaultdict(Fraction)
        for i in range(N):
            for k3, w3 in self.gamma3(i).items():
                g3 = from_key(k3)
                for chain, wc in self.chains(N - i - 1):
                    b = _Builder()
                    a = b.vertex()
                    ins, outs, end = b.add(g3)
                    b.partner[a], b.partner[end] = end, a
                    _mark(b, a, "in", 0)
                    b.dressed(a, ins[0], chain)
                    _mark(b, outs[0], "out", 0)
                    _add_to(acc, b.piece(), w3 * wc)
        return dict(acc)

    # G^(k): chains of self-energy insertions of total order k
    @_memo
    def chains(self, k):
        if k == 0:
            return ((), Fraction(1)),
        out = []
        for first in range(1, k + 1):
            for ks, ws in self.sigma(first).items():
                for rest, wr in self.chains(k - first):
                    out.append(((from_key(ks),) + rest, ws * wr))
        return tuple(out)

    # Gamma3^(N)
    @_memo
    def gamma3(self, N):
        if N == 0:
            return {canonical(((-1,), (-1,), (-1,))): Fraction(1)}
        acc = collections.defaultdict(Fraction)
        for i in range(N):
            for k4, w4 in self.gamma4(i).items():
                g4 = from_key(k4)
                M = N - i - 1
                for j in range(M + 1):
                    for c1, w1 in self.chains(j):
                        for c2, w2 in self.chains(M - j):
                            b = _Builder()
                            bv = b.vertex()
                            ins, outs, _ = b.add(g4)
                            b.partner[bv] = -1
                            b.dressed(bv, ins[1], c1)
                            b.dressed(outs[1], bv, c2)
                            _mark(b, ins[0], "in", 0)
                            _mark(b, outs[0], "out", 0)
                            _add_to(acc, b.piece(), w4 * w1 * w2)
        return dict(acc)

    # Gamma4^(N) and its channel parts
    @_memo
    def gamma4(self, N):
        acc = collections.defaultdict(Fraction)
        for k, w in self.irreducible(N).items():
            acc[k] += w
        for c in ("ph", "phbar", "pp"):
            for k, w in self.phi(c, N).items():
                acc[k] += w
        return {k: w for k, w in acc.items() if w != 0}

    @_memo
    def irreducible(self, N):
        if N == 0:
            direct = ((-1, -2), (-1, -2), (1, 0))
            exchange = ((-2, -1), (-1, -2), (1, 0))
            return {canonical(direct): Fraction(1), canonical(exchange): Fraction(1)}
        if N in self._irr:
            return dict(self._irr[N])
        return irreducible_remainder(N, [self.phi(c, N) for c in ("ph", "phbar", "pp")])

    @_memo
    def gamma4_irreducible_in(self, join, N):
        """Gamma4 minus its part reducible in the channel of the join (ph for
        the ph and phbar joins, pp for the pp join), in the piece's own legs."""
        acc = collections.defaultdict(Fraction, self.gamma4(N))
        for k, w in self.phi("ph" if join in ("ph", "phbar") else "pp", N).items():
            acc[k] -= w
        return {k: w for k, w in acc.items() if w != 0}

    @_memo
    def phi(self, c, N):
        acc = collections.defaultdict(Fraction)
        if N == 0:
            return {}
        if c == "phbar":
            for k, w in self.phi("ph", N).items():
                _add_to(acc, _swap_outs(from_key(k)), w)
            return dict(acc)
        half = Fraction(1, 2) if c == "pp" else Fraction(1)
        for i, j, kk in itertools.product(range(N), repeat=3):
            l = N - 1 - i - j - kk
            if l < 0:
                continue
            for kl, wl in self.gamma4(i).items():
                L = from_key(kl)
                for kr, wr in self.gamma4_irreducible_in(c, j).items():
                    R = from_key(kr)
                    for c1, w1 in self.chains(kk):
                        for c2, w2 in self.chains(l):
                            b = _Builder()
                            li, lo, _ = b.add(L)
                            ri, ro, _ = b.add(R)
                            if c == "ph":
                                b.dressed(lo[1], ri[0], c1)
                                b.dressed(ro[0], li[1], c2)
                                legs = (li[0], lo[0], ri[1], ro[1])
                            else:
                                b.dressed(lo[0], ri[0], c1)
                                b.dressed(lo[1], ri[1], c2)
                                legs = (li[0], ro[0], li[1], ro[1])
                            _mark(b, legs[0], "in", 0)
                            _mark(b, legs[1], "out", 0)
                            _mark(b, legs[2], "in", 1)
                            _mark(b, legs[3], "out", 1)
                            _add_to(acc, b.piece(), half * wl * wr * w1 * w2)
        return dict(acc)
