"""Feynman-graph compiler: self-energy diagrams -> instruction tape for ``fd_graph_load``.

The paper's compiler (Sec. V.A, Fig. compiler_prx_final) turns diagrams into a
computational graph IR whose leaves are propagators and interactions and whose
internal nodes are products and sums (Sec. II.B, Fig. factorization), applies
Taylor-mode differentiation for the counterterms (Sec. III.C, Eqs. taylor_node,
chain_rule) and emits code.  Here the back end emits a flat, topologically
ordered instruction tape that the GPU interpreter executes per sample.

Pipeline
1. Generate every connected Green's-function topology of order n directly in
   canonical form (canonical-order depth-first construction of the fermion
   permutation) and keep the one-particle-irreducible, tadpole-free ones
   (criteria read off the momentum routing: a fermion line with no loop
   momentum is a bridge, an interaction line with zero momentum is a tadpole).
2. Route momenta and times with the project convention (spanning tree of all
   interaction lines plus fermion lines taken in descending source order; the
   n fermion chords carry k_1..k_n in ascending source order; k_ext runs from
   vertex 0 to the out-vertex along the tree).
3. Expand each requested root Sigma^(n,m,l) (and its k-derivative) into
   monomials over Taylor coefficients of the leaves: G leaves carry
   c_j = (d/dmu)^j G0 / j!, V leaves c_l = (d/dLambda)^l V / l!, so the
   Leibniz multinomials are absorbed (Eq. taylor_node); d/dk acts through the
   lines that carry k_ext.
4. Factorise every (root, out-line) polynomial by greedy multivariate Horner
   (always pull out the most frequent leaf) and hash-cons the result into one
   DAG shared by all roots (the shared-subexpression graph of Sec. II.B).
5. Schedule the DAG depth-first, compute each leaf family just before its
   first use, allocate per-sample slots by liveness, and serialise.

Tape format, version 4 (little endian; sections 16-byte aligned):
  header  16 x u32: magic 'FDTP', version, order, dim, n_roots, n_slots,
          n_instr, root_table_off, instr_off, total_bytes, n_g_leaves,
          n_v_leaves, n_arith, n_consts, reserved x2
  roots   n_roots x (u8 n, u8 m, u8 l, u8 dk, u16 0, u16 0)
  instr   n_instr x u64, low to high: op:6 | d:14 | a:14 | b:14 | c:14, except
          the words that follow a BUNDLE header (four u16 slot indices each).
          Leaf ops keep in `a` a signed 2-bit coefficient per momentum
          variable (k_ext, k_1..k_N; 1 = +1, 3 = -1) and in the upper bits the
          two interaction lines (3 bits each), the Taylor order (3 bits),
          the d/dk flag and (G leaves, bit 44) the precise flag: the family
          is the only G line of a root's value (the order-1 diagram),
          evaluated in double-float arithmetic.  RACC: `a` = value slot, `b` = out-line; RFLUSH:
          `d` = root index; CONST: float in the high 32 bits.
Per-sample state: slot 0 = 0.0, slot 1 = 1.0 and slots 2..N+1 = hypercube time
of interaction lines 0..N-1 (written by the kernel), then constants, leaf
families and temporaries; loop momenta, Jacobians and root accumulators live
in registers or fixed extra slots of the interpreter.
"""
import collections
import math
import struct
import sys

MAGIC = 0x50544446  # 'FDTP'
VERSION = 4

# opcodes (keep in sync with csrc/fd_internal.cuh)
OP_FMA = 1      # (reserved; products and sums travel in bundles)
OP_GLEAF = 2    # S[d..] = Taylor coefficients of G0; momentum mask, lines la/lb, M, dk
OP_VLEAF = 3    # S[d..] = Taylor coefficients of V; momentum mask, L, dk
OP_RACC = 4     # root accumulator += S[a] * exp(i pi x_line)   (line 0: phase 1)
OP_RFLUSH = 5   # root r complete: weight by its Jacobian, reduce, reset the accumulator
OP_CONST = 6    # S[d] = f32 immediate (high 32 bits)
OP_NOP = 7      # padding (keeps bundles inside one tape chunk)
OP_BUNDLE = 8   # the next n (1..8) words are independent FMAs S[d] = S[a] S[b] + S[c]
                #   (u16 d, a, b, c; MUL: c = slot 0 = 0.0; ADD: b = slot 1 = 1.0):
                #   the kernel loads all operands, computes, then stores all results
CHUNK_WORDS = 1024   # tape chunk the GPU stages at a time; bundles never straddle one
MAX_BUNDLE = 8
OP_END = 63


# --------------------------------------------------------------------------
# 1. topology generation (canonical depth-first construction)
# --------------------------------------------------------------------------

def generate_connected(n):
    """All connected topologies of order n as canonical permutations (X = 2n)."""
    X = 2 * n
    out = []
    sigma = [-1] * (2 * n)
    visited = [False] * (2 * n)

    def next_loop_start(nl):
        for v in range(2 * nl):
            if not visited[v]:
                return v
        return -1

    def rec(v, nl, loop_start):
        # v: current vertex (already visited); choose sigma[v]
        cands = [X if loop_start < 0 else loop_start]
        cands += [w for w in range(2 * nl) if not visited[w]]
        if nl < n:
            cands.append(2 * nl)       # first vertex of a new interaction line
        for w in cands:
            new_nl = nl + 1 if (nl < n and w == 2 * nl) else nl
            sigma[v] = w
            if w == X or w == loop_start:
                # cycle closed: next loop starts at the smallest unvisited labelled vertex
                st = next_loop_start(new_nl)
                if st < 0:
                    if new_nl == n:
                        out.append(tuple(sigma))
                else:
                    visited[st] = True
                    rec(st, new_nl, st)
                    visited[st] = False
            else:
                visited[w] = True
                rec(w, new_nl, loop_start)
                visited[w] = False
            sigma[v] = -1

    visited[0] = True
    rec(0, 1, -1)
    return out


# --------------------------------------------------------------------------
# 2. routing
# --------------------------------------------------------------------------

class Routed:
    __slots__ = ("n", "sigma", "sign", "out_line", "g_lines", "v_lines")

    def __init__(self, n, sigma, sign, out_line, g_lines, v_lines):
        self.n = n
        self.sigma = sigma
        self.sign = sign
        self.out_line = out_line
        self.g_lines = g_lines   # list of (mom tuple, line_dst, line_src)
        self.v_lines = v_lines   # list of mom tuples


def route_topology(n, sigma):
    X = 2 * n
    nv = 2 * n
    out_v = sigma.index(X)
    gsrc = [v for v in range(nv) if sigma[v] != X]
    comp = list(range(nv))

    def root(a):
        while comp[a] != a:
            a = comp[a]
        return a

    tree = collections.defaultdict(list)   # vertex -> [(nbr, ('g'|'v', id), dir)]
    for i in range(n):
        comp[root(2 * i)] = root(2 * i + 1)
        tree[2 * i].append((2 * i + 1, ("v", i), 1))
        tree[2 * i + 1].append((2 * i, ("v", i), -1))
    chords = []
    for v in sorted(gsrc, reverse=True):
        ra, rb = root(v), root(sigma[v])
        if ra == rb:
            chords.append(v)
        else:
            comp[ra] = rb
            tree[v].append((sigma[v], ("g", v), 1))
            tree[sigma[v]].append((v, ("g", v), -1))
    chords.sort()
    mom = {("g", v): [0] * (n + 1) for v in gsrc}
    mom.update({("v", i): [0] * (n + 1) for i in range(n)})

    def push(a, b, col):
        # depth-first search for the tree path a -> b, then add +-1 along it
        stack = [(a, None)]
        parent = {a: None}
        while stack:
            u, _ = stack.pop()
            if u == b:
                break
            for w, e, d in tree[u]:
                if w not in parent:
                    parent[w] = (u, e, d)
                    stack.append((w, None))
        u = b
        while parent[u] is not None:
            p, e, d = parent[u]
            mom[e][col] += d
            u = p

    push(0, out_v, 0)
    for j, c in enumerate(chords):
        mom[("g", c)][j + 1] += 1
        push(sigma[c], c, j + 1)
    # closed loops for the sign
    seen = [False] * nv
    v = 0
    while v != X:
        seen[v] = True
        v = sigma[v]
    F = 0
    for u in range(nv):
        if not seen[u]:
            F += 1
            w = u
            while not seen[w]:
                seen[w] = True
                w = sigma[w]
    g_lines = [(tuple(mom[("g", v)]), sigma[v] // 2, v // 2) for v in gsrc]
    v_lines = [tuple(mom[("v", i)]) for i in range(n)]
    sign = (-1) ** (n + F) * 2 ** F
    return Routed(n, tuple(sigma), sign, out_v // 2, g_lines, v_lines)


def self_energy_diagrams(n):
    """1PI, tadpole-free self-energy diagrams of order n with their routing."""
    out = []
    for s in generate_connected(n):
        r = route_topology(n, s)
        if all(any(c != 0 for c in m[1:]) for (m, _, _) in r.g_lines) and \
           all(any(c != 0 for c in m) for m in r.v_lines):
            out.append(r)
    return out


# --------------------------------------------------------------------------
# 3. monomials over leaf Taylor coefficients
# --------------------------------------------------------------------------

def _canon_mom(m):
    """Momentum up to overall sign (eps and q^2 are even): leading nonzero > 0."""
    for c in m:
        if c != 0:
            return (tuple(m), 1) if c > 0 else (tuple(-x for x in m), -1)
    return (tuple(m), 1)


def _compositions(total, parts):
    if parts == 0:
        if total == 0:
            yield ()
        return
    if parts == 1:
        yield (total,)
        return
    for first in range(total + 1):
        for rest in _compositions(total - first, parts - 1):
            yield (first,) + rest


def root_polynomials(order, roots):
    """{(root index, out line): {monomial (sorted tuple of vars): coefficient}}.

    vars: ('G', mom, la, lb, j) / ('Gd', mom, la, lb, j) / ('V', mom, j) / ('Vd', mom, j)
    with mom the canonical-sign momentum; root values are m! l! times the
    Taylor-coefficient sums.
    """
    polys = collections.defaultdict(lambda: collections.defaultdict(int))
    need = {}
    by_n = collections.defaultdict(list)
    for r, (n, m, l, dk) in enumerate(roots):
        by_n[n].append((r, m, l, dk))
    for n, rl in by_n.items():
        for d in self_energy_diagrams(n):
            pad = (0,) * (order - n)      # momenta live in the order-N variable space
            gl = []
            for (mom, la, lb) in d.g_lines:
                cm, sg = _canon_mom(tuple(mom) + pad)
                gl.append((cm, la, lb))
            vl = [_canon_mom(tuple(mom) + pad)[0] for mom in d.v_lines]
            for (r, m, l, dk) in rl:
                fac = d.sign * math.factorial(m) * math.factorial(l)
                P = polys[(r, d.out_line)]
                for mg in _compositions(m, len(gl)):
                    gv = [("G",) + gl[e] + (mg[e],) for e in range(len(gl))]
                    for lv in _compositions(l, len(vl)):
                        vv = [("V", vl[v], lv[v]) for v in range(len(vl))]
                        if dk == 0:
                            P[tuple(sorted(gv + vv))] += fac
                            continue
                        for e in range(len(gl)):
                            if gl[e][0][0] != 0:
                                g2 = list(gv)
                                g2[e] = ("Gd",) + gv[e][1:]
                                P[tuple(sorted(g2 + vv))] += fac
                        for v in range(len(vl)):
                            if vl[v][0] != 0:
                                v2 = list(vv)
                                v2[v] = ("Vd",) + vv[v][1:]
                                P[tuple(sorted(gv + v2))] += fac
    # drop cancelled monomials
    out = {}
    for key, P in polys.items():
        Q = {mono: c for mono, c in P.items() if c != 0}
        if Q:
            out[key] = Q
    return out


# --------------------------------------------------------------------------
# 4. greedy multivariate Horner into a hash-consed DAG
# --------------------------------------------------------------------------

class DAG:
    """Hash-consed expression DAG.  Leaves and constants are shared globally;
    products and sums are shared within the current `scope` (one root
    polynomial), which bounds how long a shared temporary stays alive."""

    def __init__(self):
        self.nodes = []          # (kind, args)
        self.index = {}
        self.scope = None

    def make(self, kind, *args):
        if kind in ("mul", "add"):
            args = tuple(sorted(args))
        key = (kind,) + tuple(args)
        ikey = key if kind in ("var", "const") else key + (self.scope,)
        if ikey in self.index:
            return self.index[ikey]
        self.nodes.append(key)
        self.index[ikey] = len(self.nodes) - 1
        return len(self.nodes) - 1

    def var(self, v):
        return self.make("var", v)

    def const(self, c):
        return self.make("const", float(c))


def horner(dag, poly):
    """Node for sum_mono coef * prod(mono) by greedy multivariate Horner."""
    monos = list(poly.items())
    return _horner(dag, monos)


def _product(dag, mono, coef):
    node = None
    for v in mono:
        x = dag.var(v)
        node = x if node is None else dag.make("mul", node, x)
    if node is None:
        return dag.const(coef)
    if coef != 1:
        node = dag.make("mulc", node, float(coef))
    return node


def _horner(dag, monos):
    if len(monos) == 1:
        mono, coef = monos[0]
        return _product(dag, mono, coef)
    cnt = collections.Counter()
    for mono, _ in monos:
        for v in set(mono):
            cnt[v] += 1
    best = max(cnt.values()) if cnt else 0
    if best <= 1:
        # no shared factor: plain sum of products
        node = None
        for mono, coef in monos:
            t = _product(dag, mono, coef)
            node = t if node is None else dag.make("add", node, t)
        return node
    x = min(v for v, c in cnt.items() if c == best)
    A, B = [], []
    for mono, coef in monos:
        if x in mono:
            l = list(mono)
            l.remove(x)
            A.append((tuple(l), coef))
        else:
            B.append((mono, coef))
    # merge constant monomials of A
    consts = sum(c for mo, c in A if len(mo) == 0)
    A = [(mo, c) for mo, c in A if len(mo) > 0]
    if consts != 0:
        A.append(((), consts))
    hA = _horner(dag, A)
    xn = dag.var(x)
    if B:
        hB = _horner(dag, B)
        return dag.make("fma", xn, hA, hB)
    return dag.make("mul", xn, hA)


# --------------------------------------------------------------------------
# 5. scheduling, leaf families, slot allocation, serialisation
# --------------------------------------------------------------------------

def _enc_fma(d, a, b, c):
    """FMA word inside a bundle: four u16 slot indices (d, a, b, c), low to high."""
    for v in (d, a, b, c):
        assert 0 <= v < 16384
    return d | (a << 16) | (b << 32) | (c << 48)


LEAF_PRECISE_BIT = 44


def _enc_leaf(op, d, mask, la, lb, M, dk, precise=False):
    assert 0 <= d < 16384 and 0 <= mask < 16384 and 0 <= la < 8 and 0 <= lb < 8 and 0 <= M < 8
    assert not precise or op == OP_GLEAF
    return (op | (d << 6) | (mask << 20) | (la << 34) | (lb << 37) | (M << 40) | (int(dk) << 43)
            | (int(precise) << LEAF_PRECISE_BIT))


def _enc_racc(a, line):
    return OP_RACC | (a << 20) | (line << 34)


def _enc_flush(r):
    return OP_RFLUSH | (r << 6)


def _enc_const(d, f):
    bits = struct.unpack("<I", struct.pack("<f", f))[0]
    return OP_CONST | (d << 6) | (bits << 32)


def mom_mask(mom):
    """2 bits per momentum variable (k_ext, k_1..k_N) read as a signed 2-bit
    integer: 0 = absent, 1 = +1, 3 = -1."""
    m = 0
    for j, c in enumerate(mom):
        if c == 1:
            m |= 1 << (2 * j)
        elif c == -1:
            m |= 3 << (2 * j)
        else:
            assert c == 0
    return m


class Tape:
    def __init__(self, order, roots, words, n_slots, stats):
        self.order = order
        self.roots = roots
        self.words = words
        self.n_slots = n_slots
        self.stats = stats

    def to_bytes(self):
        n_roots = len(self.roots)
        rt_off = 64
        rt_size = (8 * n_roots + 15) // 16 * 16
        ins_off = rt_off + rt_size
        total = (ins_off + 8 * len(self.words) + 15) // 16 * 16
        st = self.stats
        hdr = struct.pack("<16I", MAGIC, VERSION, self.order, 4 * self.order - 1, n_roots, self.n_slots,
                          len(self.words), rt_off, ins_off, total, st.get("g_leaves", 0), st.get("v_leaves", 0),
                          st.get("arith", 0), st.get("consts", 0), 0, 0)
        rt = b"".join(struct.pack("<4B2H", n, m, l, dk, 0, 0) for (n, m, l, dk) in self.roots)
        rt += b"\0" * (rt_size - len(rt))
        out = hdr + rt + struct.pack("<%dQ" % len(self.words), *self.words)
        return out + b"\0" * (total - len(out))


def fixed_slots(order):
    """Slots the kernel prologue writes: 0 = 0.0, 1 = 1.0, then the hypercube time
    coordinate of interaction lines 0..N-1 (line 0: 0)."""
    return 2 + order


class SlotAllocator:
    """First-fit allocator of contiguous per-sample slots above a fixed base."""

    def __init__(self, base):
        self.top = base
        self.free = []          # sorted (start, length)
        self.live = 0
        self.peak = base

    def alloc(self, k):
        self.live += k
        for i, (st, ln) in enumerate(self.free):
            if ln >= k:
                if ln == k:
                    self.free.pop(i)
                else:
                    self.free[i] = (st + k, ln - k)
                return st
        st = self.top
        self.top += k
        self.peak = max(self.peak, self.top)
        return st

    def release(self, st, k):
        self.live -= k
        self.free.append((st, k))
        self.free.sort()
        merged = []
        for a, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((a, l))
        if merged and merged[-1][0] + merged[-1][1] == self.top:
            self.top = merged[-1][0]
            merged.pop()
        self.free = merged


def _kids(key):
    kind = key[0]
    if kind in ("mul", "add"):
        return [key[1], key[2]]
    if kind == "fma":
        return [key[1], key[2], key[3]]
    if kind == "mulc":
        return [key[1]]
    return []


def compile_graph(order, roots, budget=96, bundle=4, window=32):
    """Compile roots [(n, m, l, dk)] of an order-`order` graph into a Tape.

    budget: per-sample slots the scheduler tries to keep leaf families and
    temporaries within; leaf families beyond it are evicted (farthest next use
    first) and recomputed when needed again.
    bundle, window: up to `bundle` mutually independent products/sums found
    within the next `window` scheduled operations are issued as one bundle,
    which the interpreter executes with all operand loads first (ILP).
    """
    assert 1 <= bundle <= MAX_BUNDLE
    sys.setrecursionlimit(max(sys.getrecursionlimit(), 100000))
    N = order
    for (n, m, l, dk) in roots:
        assert 1 <= n <= N and m >= 0 and l >= 0 and dk in (0, 1)
    polys = root_polynomials(order, roots)
    dag = DAG()
    outputs = []
    for (r, o) in sorted(polys):
        dag.scope = (r, o)
        outputs.append((r, o, horner(dag, polys[(r, o)])))
    return compile_dag(order, roots, dag, outputs, budget, bundle, window)


def compile_dag(order, roots, dag, outputs, budget=96, bundle=4, window=32):
    """Schedule, allocate and serialise a built DAG: outputs [(root index, out
    line, node)] accumulate into the roots [(n, m, l, dk)]; leaves are
    ('G', mom, line_dst, line_src, j) / ('Gd', ...) / ('V', mom, j) /
    ('Vd', mom, j) with mom over (k_ext, k_1..k_order) up to overall sign."""
    assert 1 <= bundle <= MAX_BUNDLE
    sys.setrecursionlimit(max(sys.getrecursionlimit(), 100000))
    N = order

    # ---- pass 1: linear schedule (post-order, largest-need child first) ------
    need = {}

    def need_of(u):
        stk = [(u, False)]
        while stk:
            x, done = stk.pop()
            if x in need:
                continue
            ks = _kids(dag.nodes[x])
            if not done:
                stk.append((x, True))
                stk.extend((k, False) for k in ks if k not in need)
                continue
            if not ks:
                need[x] = 0
                continue
            nk = sorted((need[k] for k in ks), reverse=True)
            need[x] = max(max(v + i for i, v in enumerate(nk)), 1)
        return need[u]

    items = []            # ('node', u) | ('racc', u, line) | ('flush', r)
    emitted = set()
    by_root = collections.defaultdict(list)
    for (r, o, node) in outputs:
        by_root[r].append((o, node))
    for r in range(len(roots)):
        for (o, node) in by_root.get(r, []):
            stk = [(node, False)]
            while stk:
                u, done = stk.pop()
                if u in emitted:
                    continue
                key = dag.nodes[u]
                if key[0] in ("var", "const"):
                    emitted.add(u)
                    continue
                ks = _kids(key)
                if not done:
                    stk.append((u, True))
                    for k in sorted(ks, key=need_of):
                        if k not in emitted:
                            stk.append((k, False))
                    continue
                emitted.add(u)
                items.append(("node", u))
            items.append(("racc", node, o))
        items.append(("flush", r))

    # ---- pass 1b: bundles of independent FMAs (list scheduling, lookahead window)
    groups = []
    done = set()
    taken = [False] * len(items)
    front = 0
    while front < len(items):
        while front < len(items) and taken[front]:
            front += 1
        if front >= len(items):
            break
        it = items[front]
        if it[0] != "node":
            groups.append([it])
            taken[front] = True
            continue
        bund = []
        for j in range(front, min(len(items), front + window)):
            if taken[j] or items[j][0] != "node":
                continue
            u = items[j][1]
            ks = [k for k in _kids(dag.nodes[u]) if dag.nodes[k][0] not in ("var", "const")]
            if all(k in done for k in ks):
                bund.append(j)
                if len(bund) == bundle:
                    break
        for j in bund:
            taken[j] = True
        for j in bund:
            done.add(items[j][1])
        groups.append([items[j] for j in bund])

    # leaf families
    gfam, vfam = {}, {}
    for key in dag.nodes:
        if key[0] != "var":
            continue
        v = key[1]
        if v[0] in ("G", "Gd"):
            fk = ("G", v[1], v[2], v[3])
            M, dk = gfam.get(fk, (0, False))
            gfam[fk] = (max(M, v[4]), dk or v[0] == "Gd")
        else:
            fk = ("V", v[1])
            L, dk = vfam.get(fk, (0, False))
            vfam[fk] = (max(L, v[2]), dk or v[0] == "Vd")

    def fam_of(v):
        return ("G", v[1], v[2], v[3]) if v[0] in ("G", "Gd") else ("V", v[1])

    # G families evaluated in double-float arithmetic: those reachable from an
    # order-1 root, whose value is one diagram with one G line (no other line's
    # terms share its magnitude, so the zeros of its mu-derivatives need ~48
    # significant bits)
    precise = set()
    stk = [node for (r, _, node) in outputs if roots[r][0] == 1]
    seen = set()
    while stk:
        u = stk.pop()
        if u in seen:
            continue
        seen.add(u)
        key = dag.nodes[u]
        if key[0] == "var":
            if key[1][0] in ("G", "Gd"):
                precise.add(fam_of(key[1]))
            continue
        stk.extend(_kids(key))

    def width(fk):
        M, dk = gfam[fk] if fk[0] == "G" else vfam[fk]
        return (M + 1) * (2 if dk else 1)

    def operands(item):
        if item[0] == "node":
            return _kids(dag.nodes[item[1]])
        if item[0] == "racc":
            return [item[1]]
        return []

    # uses: families by group position, node use counts
    fam_pos = collections.defaultdict(list)
    node_uses = collections.Counter()
    for pos, grp in enumerate(groups):
        for it in grp:
            for k in operands(it):
                key = dag.nodes[k]
                if key[0] == "var":
                    if not fam_pos[fam_of(key[1])] or fam_pos[fam_of(key[1])][-1] != pos:
                        fam_pos[fam_of(key[1])].append(pos)
                else:
                    node_uses[k] += 1
    fam_ptr = collections.Counter()

    # ---- pass 2: slots under the budget ---------------------------------------
    consts = sorted({key[1] for key in dag.nodes if key[0] == "const"} |
                    {key[2] for key in dag.nodes if key[0] == "mulc"})
    alloc = SlotAllocator(fixed_slots(N))
    words = []
    stats = collections.Counter()
    const_slot = {0.0: 0, 1.0: 1}
    for c in consts:
        if c not in const_slot:
            const_slot[c] = alloc.alloc(1)
            words.append(_enc_const(const_slot[c], c))
            stats["consts"] += 1
    resident = {}           # family -> slot
    node_slot = {}

    def next_use(fk, pos):
        lst = fam_pos[fk]
        i = fam_ptr[fk]
        while i < len(lst) and lst[i] < pos:
            i += 1
        fam_ptr[fk] = i
        return lst[i] if i < len(lst) else None

    def evict_for(k, pos, protect):
        while alloc.live + k > budget:
            cand = None
            far = -1
            for fk in resident:
                if fk in protect:
                    continue
                nu = next_use(fk, pos)
                d = 1 << 60 if nu is None else nu
                if d > far:
                    far, cand = d, fk
            if cand is None:
                return
            alloc.release(resident.pop(cand), width(cand))
            stats["evictions"] += 1

    def ensure(fk, pos, protect):
        if fk in resident:
            return resident[fk]
        w = width(fk)
        evict_for(w, pos, protect)
        d = alloc.alloc(w)
        if fk[0] == "G":
            _, mom, la, lb = fk
            M, dk = gfam[fk]
            words.append(_enc_leaf(OP_GLEAF, d, mom_mask(mom), la, lb, M, dk, fk in precise))
            stats["g_leaves"] += 1
        else:
            _, mom = fk
            L, dk = vfam[fk]
            words.append(_enc_leaf(OP_VLEAF, d, mom_mask(mom), 0, 0, L, dk))
            stats["v_leaves"] += 1
        resident[fk] = d
        return d

    def slot_of(k, pos, protect):
        key = dag.nodes[k]
        if key[0] == "var":
            v = key[1]
            fk = fam_of(v)
            base = ensure(fk, pos, protect)
            M = gfam[fk][0] if fk[0] == "G" else vfam[fk][0]
            j = v[4] if fk[0] == "G" else v[2]
            if v[0] in ("Gd", "Vd"):
                j += M + 1
            return base + j
        if key[0] == "const":
            return const_slot[key[1]]
        return node_slot[k]

    def drop_dead(pos):
        for fk in list(resident):
            if next_use(fk, pos + 1) is None:
                alloc.release(resident.pop(fk), width(fk))

    def emit(word):
        words.append(word)

    def pad_to_fit(n):
        # keep the next n words inside one tape chunk
        if len(words) // CHUNK_WORDS != (len(words) + n - 1) // CHUNK_WORDS:
            while len(words) % CHUNK_WORDS:
                words.append(OP_NOP)
                stats["nops"] += 1

    def fma_word(u, ks, d):
        kind = dag.nodes[u][0]
        if kind == "mul":
            return _enc_fma(d, ks[0], ks[1], 0)
        if kind == "add":
            return _enc_fma(d, ks[0], 1, ks[1])
        if kind == "fma":
            return _enc_fma(d, ks[0], ks[1], ks[2])
        return _enc_fma(d, ks[0], const_slot[dag.nodes[u][2]], 0)     # mulc

    for pos, grp in enumerate(groups):
        protect = {fam_of(dag.nodes[k][1]) for it in grp for k in operands(it) if dag.nodes[k][0] == "var"}
        if grp[0][0] == "node":
            # operands first (leaf families are computed here when not resident)
            opslots = [[slot_of(k, pos, protect) for k in operands(it)] for it in grp]
            for it in grp:
                for k in operands(it):
                    if dag.nodes[k][0] not in ("var", "const"):
                        node_uses[k] -= 1
            for it in grp:
                for k in set(operands(it)):
                    if dag.nodes[k][0] not in ("var", "const") and node_uses[k] == 0 and k in node_slot:
                        alloc.release(node_slot.pop(k), 1)
                        node_uses[k] = -1
            dests = []
            for it in grp:
                evict_for(1, pos, protect)
                dests.append(alloc.alloc(1))
            pad_to_fit(len(grp) + 1)
            emit(OP_BUNDLE | (len(grp) << 6))
            for it, ks, d in zip(grp, opslots, dests):
                emit(fma_word(it[1], ks, d))
            stats["bundles"] += 1
            for it, d in zip(grp, dests):
                node_slot[it[1]] = d
            stats["arith"] += len(grp)
        else:
            it = grp[0]
            if it[0] == "racc":
                k = it[1]
                s_ = slot_of(k, pos, protect)
                pad_to_fit(1)
                emit(_enc_racc(s_, it[2]))
                if dag.nodes[k][0] not in ("var", "const"):
                    node_uses[k] -= 1
                    if node_uses[k] == 0:
                        alloc.release(node_slot.pop(k), 1)
                stats["racc"] += 1
            else:
                pad_to_fit(1)
                emit(_enc_flush(it[1]))
        drop_dead(pos)
    pad_to_fit(1)
    words.append(OP_END)
    stats["slots"] = alloc.peak
    stats["budget"] = budget
    stats["dag_nodes"] = len(emitted)
    return Tape(N, list(roots), words, alloc.peak, dict(stats))


def graph_roots(order, with_dk=False):
    """Root list of an order-N graph: all (n, m, l) with n + m + l = N."""
    roots = []
    for dk in ((0, 1) if with_dk else (0,)):
        for n in range(order, 0, -1):
            for m in range(order - n + 1):
                roots.append((n, m, order - n - m, dk))
    return roots


# --------------------------------------------------------------------------
# algorithmic work per sample (roofline accounting)
# --------------------------------------------------------------------------

def _g_family_work(M, dk):
    """(FP32 flops, FP32 instructions) of one G family as written in the
    kernel's recurrence (an FMA is 2 flops and 1 instruction)."""
    f = i = 6                               # dx* (2), tau*, -eps tau*, sign and phi factors (2)
    Mx = M + dk
    for k in range(Mx):
        f += 2 * (k + 1) + 4                # Phi_hat convolution (k + 1 FMAs), scale, Psi, A
        i += (k + 1) + 4
    if Mx:
        for j in range(Mx + 1):
            f += 2 * (j + 1)                # c_j convolution
            i += j + 1
    if dk:
        f += 2 * (M + 1) + 1
        i += 2 * (M + 1) + 1
    return f, i


def _g_family_flops(M, dk):
    return _g_family_work(M, dk)[0]


# per-sample map in double-float arithmetic (counted from the kernel's code):
# a VEGAS coordinate, a loop momentum (radius, polar and azimuthal factors with
# the table-based cos / sin, three double-float products, the grid split,
# Jacobian), the phase and weight of an interaction-line time
MAP_VEGAS_FLOPS = 28
MAP_MOMENTUM_FLOPS, MAP_MOMENTUM_SFU = 190, 2
MAP_TIME_FLOPS, MAP_TIME_SFU = 3, 1


def _g_family_df_instr(M, dk):
    """FP32 instructions of one double-float G family (g_family_df) as
    written: eps from exact products (~100), the double-float exponential
    (~250), the Fermi factor's reciprocal and psi (~35), tau* and the common
    factor with the accurate expf (~50); per recurrence step k (k inner
    products of ~22 instructions, five products and a negation, ~41) and per
    coefficient sum j >= 1 (~16 + 22 (j - 1)); 2 per k-derivative output."""
    Mx = M + dk
    i = 435
    for k in range(Mx):
        i += 22 * k + 41
    for j in range(1, Mx + 1):
        i += 16 + 22 * (j - 1)
    if dk:
        i += 2 * (M + 1) + 1
    return i


def _leaf_work(w, instr=False):
    """(fp32 flops, sfu ops) of one leaf word (with instr: FP32 instructions
    in place of flops, an FMA counting once).

    Momentum: grid and remainder sums, 6 (t - 1) for t terms.  G: eps from the
    sums (fd_eps: 6 FMAs, a product and 3 sums: 19 flops, 10 instructions),
    p_z 1, the time difference of two nonzero lines 12, Fermi factor 3 + 2 SFU,
    then the family (_g_family_work + 1 SFU).  A G family with the precise
    flag has the same operations (flops) and executes them in double-float
    arithmetic (instructions: _g_family_df_instr).  V: q = grid +
    remainder 3, |q|^2 5 (3 instructions), 1 / (q^2 + Lambda) 1 + 1 SFU, 8 pi 1,
    the powers (L + dk), the d/dk outputs 2 + 2 (L + 1).
    """
    op = w & 63
    mask = (w >> 20) & 16383
    terms = sum(1 for j in range(7) if (mask >> (2 * j)) & 3)
    M = (w >> 40) & 7
    dk = (w >> 43) & 1
    sums = 6 * max(terms - 1, 0)
    if op == OP_GLEAF:
        la, lb = (w >> 34) & 7, (w >> 37) & 7
        td = 12 if (la != lb and la and lb) else 0
        gf, gi = _g_family_work(M, dk)
        fam = (10 if instr else 19) + 1 + 3 + (gi if instr else gf)
        if instr and (w >> LEAF_PRECISE_BIT) & 1:
            return sums + td + _g_family_df_instr(M, dk), 3
        return sums + td + fam, 3
    return sums + 3 + (3 if instr else 5) + 2 + (M + dk) + ((2 + 2 * (M + 1)) if dk else 0), 1


def _map_work(dim, order, n_roots):
    flops = MAP_VEGAS_FLOPS * dim + MAP_MOMENTUM_FLOPS * order + MAP_TIME_FLOPS * (order - 1) + 2 * n_roots
    sfu = MAP_MOMENTUM_SFU * order + MAP_TIME_SFU * (order - 1)
    return flops, sfu


def _leaf_rank_cost(w):
    """The generator's cost of a leaf family for ranking leaf-cache candidates
    (csrc/fd_jit.cu leaf_cost, the same arithmetic)."""
    mask = (w >> 20) & 16383
    terms = sum(1 for j in range(7) if (mask >> (2 * j)) & 3)
    M, dk = (w >> 40) & 7, (w >> 43) & 1
    Mx = M + dk
    c = 6.0 * max(terms - 1, 0)
    if (w & 63) == OP_GLEAF:
        c += 36.0 + 3.0 * 8.0
        for k in range(Mx):
            c += (k + 1) + 4
        if Mx:
            for j in range(Mx + 1):
                c += j + 1
    else:
        c += 12.0 + 8.0 + Mx
    return c


def specialised_work(data, root_units=True, unit_cap=None, cross_roots=False, instr=False, leaf_cache=0,
                     return_cache=False):
    """(fp32_flops, sfu_ops) per sample executed by the specialised kernel.

    The kernel evaluates every root-accumulate slice of the tape as straight-line
    code; leaves shared between slices are recomputed in each compilation unit,
    so the leaf work exceeds the tape's.  Units as the generator forms them: one
    per root with root_units, else one per slice; with unit_cap (the sample-loop
    kernels) consecutive slices of a root, or across roots with cross_roots,
    packed while FMAs + 30 per distinct leaf stay within the cap.  Same counting
    rule as tape_work (with instr: FP32 instructions, an FMA counting once).
    leaf_cache = K: the families the generator caches (used by two or more
    units, the most recomputation saved per float first, up to K floats per
    sample) are computed once per sample and read by the units.  With
    return_cache: the number of cached floats instead.
    """
    hdr = struct.unpack("<16I", data[:64])
    order, dim, n_roots, n_instr, ins_off = hdr[2], hdr[3], hdr[4], hdr[6], hdr[8]
    words = struct.unpack("<%dQ" % n_instr, data[ins_off:ins_off + 8 * n_instr])
    ins = []                     # (op, word index, bundle size)
    k = 0
    while k < n_instr:
        op = words[k] & 63
        if op == OP_BUNDLE:
            n = (words[k] >> 6) & 15
            ins.append((op, k, n))
            k += n + 1
            continue
        if op == OP_END:
            break
        if op != OP_NOP:
            ins.append((op, k, 0))
        k += 1
    slices = []                  # per slice: root, set of (instr, member) FMAs, set of leaf instrs
    root = 0
    for i, (op, wk, _) in enumerate(ins):
        if op == OP_RFLUSH:
            root += 1
            continue
        if op != OP_RACC:
            continue
        need = {(words[wk] >> 20) & 16383}
        fmas, leaves = set(), set()
        for j in range(i - 1, -1, -1):
            oj, wj, nj = ins[j]
            if oj == OP_BUNDLE:
                kept = [q for q in range(nj) if (words[wj + 1 + q] & 0xFFFF) in need]
                for q in kept:
                    need.discard(words[wj + 1 + q] & 0xFFFF)
                for q in kept:
                    m = words[wj + 1 + q]
                    need.update(((m >> 16) & 0xFFFF, (m >> 32) & 0xFFFF, m >> 48))
                    fmas.add((j, q))
            elif oj in (OP_GLEAF, OP_VLEAF):
                w = words[wj]
                d = (w >> 6) & 16383
                no = (((w >> 40) & 7) + 1) * (2 if (w >> 43) & 1 else 1)
                if any(d + q in need for q in range(no)):
                    need.difference_update(range(d, d + no))
                    leaves.add(j)
            elif oj == OP_CONST:
                need.discard((words[wj] >> 6) & 16383)
        slices.append((root, fmas, leaves))
    units = []                   # per unit: [root of its first slice, FMAs, leaves]
    for r, fmas, leaves in slices:
        if units and (cross_roots or units[-1][0] == r):
            grown_f, grown_l = units[-1][1] | fmas, units[-1][2] | leaves
            if unit_cap is None:
                fits = root_units
            else:
                fits = len(grown_f) + 30 * len(grown_l) <= unit_cap
            if fits:
                units[-1][1], units[-1][2] = grown_f, grown_l
                continue
        units.append([r, set(fmas), set(leaves)])
    cached = set()
    if return_cache:
        leaf_cache = leaf_cache or 0
    if leaf_cache > 0:
        uses = collections.Counter()
        for _, _, leaves in units:
            for j in leaves:
                uses[j] += 1

        def width(j):
            w = words[ins[j][1]]
            return (((w >> 40) & 7) + 1) * (2 if (w >> 43) & 1 else 1)
        cand = sorted(((-_leaf_rank_cost(words[ins[j][1]]) * (c - 1) / width(j), j) for j, c in uses.items() if c >= 2))
        used = 0
        for _, j in cand:
            if used + width(j) <= leaf_cache:
                cached.add(j)
                used += width(j)
    if return_cache:
        return sum((((words[ins[j][1]] >> 40) & 7) + 1) * (2 if (words[ins[j][1]] >> 43) & 1 else 1) for j in cached)
    flops = sfu = 0
    for j in cached:
        f, u = _leaf_work(words[ins[j][1]], instr)
        flops += f
        sfu += u
    for _, fmas, leaves in units:
        for (j, q) in fmas:
            m = words[ins[j][1] + 1 + q]
            flops += 1 if (instr or (m >> 48) == 0 or ((m >> 32) & 0xFFFF) == 1) else 2
        for j in leaves:
            if j in cached:
                continue
            f, u = _leaf_work(words[ins[j][1]], instr)
            flops += f
            sfu += u
    n_racc = len(slices)
    mf, mu = _map_work(dim, order, n_roots)
    return flops + 4 * n_racc + mf, sfu + mu


def contraction_ops(data):
    """Operation count N_op of a serialised tape's contraction: products and
    sums as written, an FMA counted as 2 (leaves and weighting excluded)."""
    hdr = struct.unpack("<16I", data[:64])
    n_instr, ins_off = hdr[6], hdr[8]
    words = struct.unpack("<%dQ" % n_instr, data[ins_off:ins_off + 8 * n_instr])
    ops = 0
    k = 0
    while k < n_instr:
        w = words[k]
        op = w & 63
        if op == OP_BUNDLE:
            n = (w >> 6) & 15
            for q in range(n):
                m = words[k + 1 + q]
                ops += 1 if ((m >> 48) == 0 or ((m >> 32) & 0xFFFF) == 1) else 2
            k += n + 1
            continue
        if op == OP_END:
            break
        k += 1
    return ops


def tape_work(data):
    """(fp32_flops, sfu_ops) per sample of a serialised tape, map and weighting
    included.

    Counting rule (FMA = 2 flops, other arithmetic 1): tape FMA as written
    (a multiply by slot 1 = 1.0 or an add of slot 0 = 0.0 counts 1); leaves
    per _leaf_work; RACC 4; per sample the double-float map per _map_work
    (28 per VEGAS dimension, 190 + 2 SFU (sqrt, reciprocal) per loop
    momentum, 3 + 1 SFU per time), 2 per root for the Jacobian.
    """
    hdr = struct.unpack("<16I", data[:64])
    order, dim, n_roots, n_instr, ins_off = hdr[2], hdr[3], hdr[4], hdr[6], hdr[8]
    words = struct.unpack("<%dQ" % n_instr, data[ins_off:ins_off + 8 * n_instr])
    flops = 0
    sfu = 0
    k = 0
    while k < len(words):
        w = words[k]
        op = w & 63
        if op == OP_BUNDLE:
            n = (w >> 6) & 15
            for q in words[k + 1:k + 1 + n]:
                b = (q >> 32) & 0xFFFF
                c = (q >> 48) & 0xFFFF
                flops += 1 if (c == 0 or b == 1) else 2
            k += 1 + n
            continue
        if op in (OP_GLEAF, OP_VLEAF):
            f, u = _leaf_work(w)
            flops += f
            sfu += u
        elif op == OP_RACC:
            flops += 4
        k += 1
    mf, mu = _map_work(dim, order, n_roots)
    return flops + mf, sfu + mu
