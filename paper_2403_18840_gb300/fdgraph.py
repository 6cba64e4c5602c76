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

Tape format (little endian; all sections 16-byte aligned):
  header  16 x u32: magic 'FDTP', version, order, dim, n_roots, n_slots,
          n_instr, root_table_off, instr_off, total_bytes, n_mom_ops,
          n_g_leaves, n_v_leaves, n_arith, reserved x2
  roots   n_roots x (u8 n, u8 m, u8 l, u8 dk, u16 slot_re, u16 slot_im)
  instr   n_instr x u64: op:6 | d:13 | a:13 | b:13 | c:13 | imm:6 (low to high);
          ops with a float immediate keep it in the high 32 bits instead of
          b/c/imm.
Fixed slot layout (written by the kernel prologue before the tape runs):
  0: constant 0; 1..4: k_ext record (0, 0, k, k^2); 5+4(j-1)..: record of k_j
  (px, py, pz, p^2) for j = 1..N; then the hypercube time coordinate of
  interaction lines 1..N-1; then cos(pi x), sin(pi x) of those lines; then the
  root accumulators (re, im), which the prologue zeroes.
"""
import collections
import itertools
import math
import struct
import sys

MAGIC = 0x50544446  # 'FDTP'
VERSION = 1

# opcodes (keep in sync with csrc/fd_tape.cuh)
OP_MOM = 1      # S[d..d+3] = record(S[a..a+2] + sgn * S[b..b+2]); imm bit0: sgn<0
OP_FERMI = 2    # S[d..d+3] = (eps, phi, 1-phi, pz) from momentum record a
OP_GLEAF = 3    # S[d..] = Taylor coeffs of G0 from Fermi record a, times S[b]-S[c]; imm = M | dk<<3 | ks<<4
OP_VLEAF = 4    # S[d..] = Taylor coeffs of V from momentum record a; imm = L | dk<<3 | ks<<4
OP_MUL = 5      # S[d] = S[a] * S[b]
OP_FMA = 6      # S[d] = S[a] * S[b] + S[c]
OP_ADD = 7      # S[d] = S[a] + S[b]
OP_MULC = 8     # S[d] = S[a] * f32(hi)
OP_ROOT = 9     # S[d] += S[a] * S[b]; S[d+1] += S[a] * S[c]   (phase cos/sin of the out line)
OP_ROOT0 = 10   # S[d] += S[a]                                   (out line 0: phase 1)
OP_CONST = 11   # S[d] = f32(hi)
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
    def __init__(self):
        self.nodes = []          # (kind, args)
        self.index = {}

    def make(self, kind, *args):
        if kind in ("mul", "add"):
            args = tuple(sorted(args))
        key = (kind,) + tuple(args)
        if key in self.index:
            return self.index[key]
        self.nodes.append(key)
        self.index[key] = len(self.nodes) - 1
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

def _enc(op, d=0, a=0, b=0, c=0, imm=0):
    assert 0 <= d < 8192 and 0 <= a < 8192 and 0 <= b < 8192 and 0 <= c < 8192 and 0 <= imm < 64
    return op | (d << 6) | (a << 19) | (b << 32) | (c << 45) | (imm << 58)


def _enc_f(op, d, a, f):
    bits = struct.unpack("<I", struct.pack("<f", f))[0]
    assert 0 <= d < 8192 and 0 <= a < 8192
    return op | (d << 6) | (a << 19) | (bits << 32)


class Tape:
    def __init__(self, order, roots, words, n_slots, root_slots, stats):
        self.order = order
        self.roots = roots
        self.words = words
        self.n_slots = n_slots
        self.root_slots = root_slots
        self.stats = stats

    def to_bytes(self):
        n_roots = len(self.roots)
        hdr_size = 64
        rt_off = hdr_size
        rt_size = (8 * n_roots + 15) // 16 * 16
        ins_off = rt_off + rt_size
        total = ins_off + 8 * len(self.words)
        total = (total + 15) // 16 * 16
        st = self.stats
        hdr = struct.pack("<16I", MAGIC, VERSION, self.order, 4 * self.order - 1, n_roots,
                          self.n_slots, len(self.words), rt_off, ins_off, total,
                          st["mom_ops"], st["g_leaves"], st["v_leaves"], st["arith"], 0, 0)
        rt = b"".join(struct.pack("<4B2H", n, m, l, dk, self.root_slots[i][0], self.root_slots[i][1])
                      for i, (n, m, l, dk) in enumerate(self.roots))
        rt += b"\0" * (rt_size - len(rt))
        ins = struct.pack("<%dQ" % len(self.words), *self.words)
        out = hdr + rt + ins
        return out + b"\0" * (total - len(out))


def prologue_layout(order):
    N = order
    lay = {"zero": 0, "kext": 1}
    lay["k"] = {j: 5 + 4 * (j - 1) for j in range(1, N + 1)}
    t0 = 5 + 4 * N
    lay["tx"] = {0: 0}
    for i in range(1, N):
        lay["tx"][i] = t0 + i - 1
    p0 = t0 + N - 1
    lay["cos"] = {i: p0 + 2 * (i - 1) for i in range(1, N)}
    lay["sin"] = {i: p0 + 2 * (i - 1) + 1 for i in range(1, N)}
    lay["end"] = p0 + 2 * (N - 1)
    return lay


class SlotAllocator:
    """First-fit allocator of contiguous per-sample slots above a fixed base."""

    def __init__(self, base):
        self.base = base
        self.top = base
        self.free = []          # sorted list of (start, length)

    def alloc(self, k):
        for i, (st, ln) in enumerate(self.free):
            if ln >= k:
                if ln == k:
                    self.free.pop(i)
                else:
                    self.free[i] = (st + k, ln - k)
                return st
        st = self.top
        self.top += k
        return st

    def release(self, st, k):
        self.free.append((st, k))
        self.free.sort()
        merged = []
        for a, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((a, l))
        # give back a trailing block
        if merged and merged[-1][0] + merged[-1][1] == self.top:
            self.top = merged[-1][0]
            merged.pop()
        self.free = merged


def _mom_parent(mom):
    nz = [i for i, c in enumerate(mom) if c != 0]
    if len(nz) == 1:
        assert mom[nz[0]] == 1, "canonical momenta start with a positive coefficient"
        return None, nz[0], 1
    last = nz[-1]
    par = list(mom)
    c = par[last]
    par[last] = 0
    return tuple(par), last, c


def compile_graph(order, roots):
    """Compile the roots [(n, m, l, dk)] of an order-`order` graph into a Tape."""
    sys.setrecursionlimit(max(sys.getrecursionlimit(), 100000))
    N = order
    for (n, m, l, dk) in roots:
        assert 1 <= n <= N and m >= 0 and l >= 0 and dk in (0, 1)
    polys = root_polynomials(order, roots)
    dag = DAG()
    outputs = []      # (root index, out line, node)
    for (r, o) in sorted(polys):
        outputs.append((r, o, horner(dag, polys[(r, o)])))

    # ---- use counts --------------------------------------------------------
    def kids_of(key):
        kind = key[0]
        if kind in ("mul", "add"):
            return [key[1], key[2]]
        if kind == "fma":
            return [key[1], key[2], key[3]]
        if kind == "mulc":
            return [key[1]]
        return []

    uses = collections.Counter()
    reachable = set()
    stack = [node for _, _, node in outputs]
    for _, _, node in outputs:
        uses[node] += 1
    while stack:
        u = stack.pop()
        if u in reachable:
            continue
        reachable.add(u)
        for k in kids_of(dag.nodes[u]):
            uses[k] += 1
            stack.append(k)

    # leaf families and their total use counts
    gfam, vfam = {}, {}
    fam_uses = collections.Counter()
    for u in reachable:
        key = dag.nodes[u]
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
        fam_uses[fk] += uses[u]

    # momentum records needed (with parents) and their use counts
    lay = prologue_layout(N)
    fixed_mom = {}
    for j in range(N + 1):
        m = [0] * (N + 1)
        m[j] = 1
        fixed_mom[tuple(m)] = lay["kext"] if j == 0 else lay["k"][j]
    mom_uses = collections.Counter()
    needed = set()

    def need(mom):
        if mom in fixed_mom or mom in needed:
            return
        needed.add(mom)
        par, _, _ = _mom_parent(mom)
        if par is not None:
            mom_uses[par] += 1
            need(par)

    fermi_uses = collections.Counter()
    for fk in gfam:
        need(fk[1])
        fermi_uses[fk[1]] += 1
    for mom in set(fk[1] for fk in gfam):
        mom_uses[mom] += 1            # its Fermi record
    for fk in vfam:
        need(fk[1])
        mom_uses[fk[1]] += 1          # its V family

    # ---- emission ------------------------------------------------------------
    n_roots = len(roots)
    root_slots = [(lay["end"] + 2 * r, lay["end"] + 2 * r + 1) for r in range(n_roots)]
    alloc = SlotAllocator(lay["end"] + 2 * n_roots)
    words = []
    stats = collections.Counter()
    mom_slot = dict(fixed_mom)
    fermi_slot = {}
    fam_slot = {}          # family key -> (slot, width)
    leaf_slot = {}
    node_slot = {}
    const_slot = {}

    def drop_mom(mom):
        if mom in fixed_mom:
            return
        mom_uses[mom] -= 1
        if mom_uses[mom] == 0:
            alloc.release(mom_slot.pop(mom), 4)

    def mom_record(mom):
        if mom in mom_slot:
            return mom_slot[mom]
        par, k, c = _mom_parent(mom)
        pa = mom_record(par)
        d = alloc.alloc(4)
        kslot = fixed_mom[tuple(1 if i == k else 0 for i in range(N + 1))]
        words.append(_enc(OP_MOM, d=d, a=pa, b=kslot, imm=1 if c < 0 else 0))
        stats["mom_ops"] += 1
        mom_slot[mom] = d
        drop_mom(par)
        return d

    def fermi_record(mom):
        if mom in fermi_slot:
            return fermi_slot[mom]
        m = mom_record(mom)
        d = alloc.alloc(4)
        words.append(_enc(OP_FERMI, d=d, a=m))
        stats["fermi_ops"] += 1
        fermi_slot[mom] = d
        drop_mom(mom)
        return d

    def family(fk):
        if fk in fam_slot:
            return
        if fk[0] == "G":
            _, mom, la, lb = fk
            M, dk = gfam[fk]
            f = fermi_record(mom)
            width = (M + 1) * (2 if dk else 1)
            d = alloc.alloc(width)
            imm = M | (int(dk) << 3) | ((mom[0] + 1) << 4)
            words.append(_enc(OP_GLEAF, d=d, a=f, b=lay["tx"][la], c=lay["tx"][lb], imm=imm))
            stats["g_leaves"] += 1
            fermi_uses[mom] -= 1
            if fermi_uses[mom] == 0:
                alloc.release(fermi_slot.pop(mom), 4)
            for j in range(M + 1):
                leaf_slot[("G", mom, la, lb, j)] = d + j
                if dk:
                    leaf_slot[("Gd", mom, la, lb, j)] = d + M + 1 + j
        else:
            _, mom = fk
            L, dk = vfam[fk]
            m = mom_record(mom)
            width = (L + 1) * (2 if dk else 1)
            d = alloc.alloc(width)
            imm = L | (int(dk) << 3) | ((mom[0] + 1) << 4)
            words.append(_enc(OP_VLEAF, d=d, a=m, imm=imm))
            stats["v_leaves"] += 1
            drop_mom(mom)
            for j in range(L + 1):
                leaf_slot[("V", mom, j)] = d + j
                if dk:
                    leaf_slot[("Vd", mom, j)] = d + L + 1 + j
        fam_slot[fk] = (d, width)

    def fam_key(v):
        return ("G", v[1], v[2], v[3]) if v[0] in ("G", "Gd") else ("V", v[1])

    def consume(k):
        """One use of node k has been emitted; free its storage at the last use."""
        uses[k] -= 1
        if uses[k]:
            return
        key = dag.nodes[k]
        if key[0] == "var":
            fk = fam_key(key[1])
            fam_uses[fk] -= 1
            if fam_uses[fk] == 0:
                st, w = fam_slot.pop(fk)
                alloc.release(st, w)
        elif key[0] == "const":
            pass
        else:
            alloc.release(node_slot[k], 1)

    # register-need estimate (Sethi-Ullman on the tree view of the DAG); leaves
    # count 0 because their families are allocated on demand
    need_cache = {}

    def need_of(u):
        if u in need_cache:
            return need_cache[u]
        stk = [(u, False)]
        while stk:
            x, done = stk.pop()
            if x in need_cache:
                continue
            ks = kids_of(dag.nodes[x])
            if not done:
                stk.append((x, True))
                stk.extend((k, False) for k in ks if k not in need_cache)
                continue
            if not ks:
                need_cache[x] = 0 if dag.nodes[x][0] in ("var", "const") else 1
                continue
            nk = sorted((need_cache[k] for k in ks), reverse=True)
            need_cache[x] = max(max(v + i for i, v in enumerate(nk)), 1)
        return need_cache[u]

    def materialise(nid):
        stack = [(nid, False)]
        while stack:
            u, expanded = stack.pop()
            if u in node_slot:
                continue
            key = dag.nodes[u]
            kind = key[0]
            if kind == "var":
                family(fam_key(key[1]))
                node_slot[u] = leaf_slot[key[1]]
                continue
            if kind == "const":
                c = key[1]
                if c not in const_slot:
                    d = alloc.alloc(1)
                    words.append(_enc_f(OP_CONST, d, 0, c))
                    const_slot[c] = d
                node_slot[u] = const_slot[c]
                continue
            kids = kids_of(key)
            if not expanded:
                stack.append((u, True))
                # evaluate the child with the largest need first
                for k in sorted(kids, key=need_of):
                    if k not in node_slot:
                        stack.append((k, False))
                continue
            ks = [node_slot[k] for k in kids]
            d = alloc.alloc(1)
            if kind == "mul":
                words.append(_enc(OP_MUL, d=d, a=ks[0], b=ks[1]))
            elif kind == "add":
                words.append(_enc(OP_ADD, d=d, a=ks[0], b=ks[1]))
            elif kind == "fma":
                words.append(_enc(OP_FMA, d=d, a=ks[0], b=ks[1], c=ks[2]))
            else:
                words.append(_enc_f(OP_MULC, d, ks[0], key[2]))
            stats["arith"] += 1
            node_slot[u] = d
            for k in kids:
                consume(k)
        return node_slot[nid]

    for (r, o, node) in outputs:
        sl = materialise(node)
        re, im = root_slots[r]
        if o == 0:
            words.append(_enc(OP_ROOT0, d=re, a=sl))
        else:
            words.append(_enc(OP_ROOT, d=re, a=sl, b=lay["cos"][o], c=lay["sin"][o]))
        stats["root_ops"] += 1
        consume(node)
    words.append(_enc(OP_END))
    stats["slots"] = alloc.top if not alloc.free else max(alloc.top, max(a + l for a, l in alloc.free))
    stats["peak_slots"] = _peak(words)
    stats["dag_nodes"] = len(reachable)
    return Tape(N, list(roots), words, stats["peak_slots"], root_slots, dict(stats))


def _peak(words):
    """Highest slot index touched by the tape + 1 (the per-sample state size)."""
    hi = 0
    for w in words:
        op = w & 63
        d = (w >> 6) & 8191
        if op == OP_END:
            continue
        if op in (OP_MOM, OP_FERMI):
            hi = max(hi, d + 4)
        elif op in (OP_GLEAF, OP_VLEAF):
            imm = (w >> 58) & 63
            M = imm & 7
            dk = (imm >> 3) & 1
            hi = max(hi, d + (M + 1) * (2 if dk else 1))
        elif op == OP_ROOT:
            hi = max(hi, d + 2)
        else:
            hi = max(hi, d + 1)
    return hi


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

def _g_family_flops(M, dk):
    """FP32 flops of one G family (FMA = 2) as written in the kernel's recurrence."""
    f = 5                                   # dx, tau, tau*, -eps tau*, times phi
    Mx = M + dk
    for k in range(Mx):
        f += 2 * (k + 1) + 4                # Phi_hat convolution, scale, Psi, A
    if Mx:
        for j in range(Mx + 1):
            f += 2 * (j + 1)                # c_j convolution
    if dk:
        f += 2 * (M + 1) + 1
    return f


def tape_work(data):
    """(fp32_flops, sfu_ops) per sample of a serialised tape, prologue and epilogue included.

    Counting rule (FMA = 2 flops, everything else 1): tape arithmetic as
    written; MOM 8; FERMI 4 + 2 SFU (exp, rcp); G family per _g_family_flops
    + 1 SFU (exp); V family 2 + (L + dk) + (dk: 2 + 2(L+1)) + 1 SFU (rcp);
    per sample the map: 6 per VEGAS dimension, 14 + 2 SFU (sincospi, sqrt)
    per loop momentum, 3 + 1 SFU per time, and 2 per root for the Jacobian.
    """
    hdr = struct.unpack("<16I", data[:64])
    order, dim, n_roots, n_instr, ins_off = hdr[2], hdr[3], hdr[4], hdr[6], hdr[8]
    words = struct.unpack("<%dQ" % n_instr, data[ins_off:ins_off + 8 * n_instr])
    flops = 0
    sfu = 0
    for w in words:
        op = w & 63
        imm = (w >> 58) & 63
        if op in (OP_MUL, OP_ADD, OP_MULC, OP_ROOT0):
            flops += 1
        elif op == OP_FMA:
            flops += 2
        elif op == OP_ROOT:
            flops += 4
        elif op == OP_MOM:
            flops += 8
        elif op == OP_FERMI:
            flops += 4
            sfu += 2
        elif op == OP_GLEAF:
            flops += _g_family_flops(imm & 7, (imm >> 3) & 1)
            sfu += 1
        elif op == OP_VLEAF:
            L, dk = imm & 7, (imm >> 3) & 1
            flops += 2 + (L + dk) + ((2 + 2 * (L + 1)) if dk else 0)
            sfu += 1
    flops += 6 * dim + 14 * order + 3 * (order - 1) + 2 * n_roots
    sfu += 2 * order + (order - 1)
    return flops, sfu
