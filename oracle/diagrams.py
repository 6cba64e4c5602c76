"""Self-energy diagram topologies and their momentum/time routing (oracle).

Sec. II.A, Eq. sigma_integration: Sigma^(n) sums n-th order topologies with n
instantaneous interaction lines (2n vertices).  Topologies come from the
brute-force enumerator ``enum_diagrams.c`` (every Wick contraction, reduced to
a canonical form).  Kept: connected, one-particle irreducible (no single
fermion line separates the external legs) and free of tadpoles (no interaction
line whose removal detaches a piece: such a line carries q = 0, excluded by the
q != 0 sum of Eq. ueg_action).

Sign and spin factor: (-1)^(n+F) 2^F for F closed fermion loops, with
G0 = -<T psi psi^dagger> (standard Matsubara convention, G = 1/(i w - eps - Sigma)).

Routing convention (shared by oracle and GPU graph builder as a stated rule,
implemented separately on each side): on canonical vertex labels,
  * fermion line g_v runs v -> sigma(v) (momentum along the fermion arrow);
    interaction line i runs 2i -> 2i+1;
  * spanning tree: all interaction lines, then fermion lines in DESCENDING order
    of their source label, each added when it joins two components;
  * the n fermion lines left out (chords) carry the loop momenta k_1..k_n in
    ASCENDING order of source label;
  * k_ext enters at vertex 0 and leaves at the out-vertex along the tree path;
    a chord's momentum returns along the tree path from its head to its tail.
Times: interaction line i has time tau_i, tau_0 = 0; fermion line v -> w has
tau = tau_line(w) - tau_line(v); equal times mean 0^-.
"""
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_cache = {}


def enumerator_path():
    """Compile enum_diagrams.c with gcc (once) and return the binary path."""
    exe = os.path.join(_BUILD, "enum_diagrams")
    src = os.path.join(_HERE, "enum_diagrams.c")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = exe + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-o", tmp, src])
        os.replace(tmp, exe)
    return exe


@dataclass(frozen=True)
class Topology:
    n: int
    sigma: tuple          # canonical permutation, X encoded as 2n
    F: int                # closed fermion loops
    one_pi: bool
    tadpole_free: bool
    multiplicity: int     # permutations with sigma(X)=0 mapping here


def all_connected(n):
    """All connected Green's-function topologies of order n (brute force)."""
    with _lock:
        if n in _cache:
            return _cache[n]
        out = subprocess.run([enumerator_path(), str(n)], check=True,
                             capture_output=True, text=True).stdout
        tops = []
        for line in out.splitlines():
            f = [int(t) for t in line.split()]
            tops.append(Topology(n=n, sigma=tuple(f[4:]), F=f[1], one_pi=bool(f[2]),
                                 tadpole_free=bool(f[3]), multiplicity=f[0]))
        tops.sort(key=lambda t: t.sigma)
        _cache[n] = tops
        return tops


def self_energy_topologies(n):
    """Connected, 1PI, tadpole-free self-energy topologies of order n."""
    return [t for t in all_connected(n) if t.one_pi and t.tadpole_free]


@dataclass
class RoutedDiagram:
    n: int
    sigma: tuple
    sign: float                 # (-1)^(n+F) 2^F
    out_vertex: int
    g_src: np.ndarray           # [2n-1] source vertex of each fermion line
    g_dst: np.ndarray           # [2n-1] target vertex
    g_mom: np.ndarray           # [2n-1, n+1] integer coefficients on (k_ext, k_1..k_n)
    v_mom: np.ndarray           # [n, n+1]
    g_tau: np.ndarray           # [2n-1, 2] (line of target, line of source): tau = t[a] - t[b]


def route(top):
    """Apply the routing convention of this module to one topology."""
    n = top.n
    X = 2 * n
    s = top.sigma
    nv = 2 * n
    out_v = [v for v in range(nv) if s[v] == X][0]
    gl = [v for v in range(nv) if s[v] != X]          # fermion lines by source
    parent = list(range(nv))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    # tree adjacency: (neighbor, edge kind, edge id, +1 if traversed along its direction)
    adj = [[] for _ in range(nv)]
    for i in range(n):
        parent[find(2 * i)] = find(2 * i + 1)
        adj[2 * i].append((2 * i + 1, "v", i, +1))
        adj[2 * i + 1].append((2 * i, "v", i, -1))
    chords = []
    for v in sorted(gl, reverse=True):
        a, b = find(v), find(s[v])
        if a != b:
            parent[a] = b
            adj[v].append((s[v], "g", v, +1))
            adj[s[v]].append((v, "g", v, -1))
        else:
            chords.append(v)
    chords.sort()
    assert len(chords) == n

    def tree_path(a, b):
        """Edges (kind, id, dir) along the unique tree path a -> b."""
        prev = {a: None}
        stack = [a]
        while stack:
            u = stack.pop()
            for (w, kind, eid, d) in adj[u]:
                if w not in prev:
                    prev[w] = (u, kind, eid, d)
                    stack.append(w)
        path = []
        u = b
        while prev[u] is not None:
            p, kind, eid, d = prev[u]
            path.append((kind, eid, d))
            u = p
        return path

    gidx = {v: j for j, v in enumerate(gl)}
    g_mom = np.zeros((2 * n - 1, n + 1), dtype=np.int64)
    v_mom = np.zeros((n, n + 1), dtype=np.int64)

    def add(kind, eid, d, col):
        if kind == "g":
            g_mom[gidx[eid], col] += d
        else:
            v_mom[eid, col] += d

    for kind, eid, d in tree_path(0, out_v):
        add(kind, eid, d, 0)
    for j, c in enumerate(chords):
        g_mom[gidx[c], j + 1] += 1
        for kind, eid, d in tree_path(s[c], c):
            add(kind, eid, d, j + 1)
    g_tau = np.array([[s[v] // 2, v // 2] for v in gl], dtype=np.int64)
    return RoutedDiagram(n=n, sigma=s, sign=float((-1) ** (n + top.F) * 2 ** top.F),
                         out_vertex=out_v, g_src=np.array(gl), g_dst=np.array([s[v] for v in gl]),
                         g_mom=g_mom, v_mom=v_mom, g_tau=g_tau)


def routed_self_energy(n):
    return [route(t) for t in self_energy_topologies(n)]


def check_conservation(d):
    """Momentum conservation at every vertex (returns max violation, 0 if exact)."""
    n = d.n
    nv = 2 * n
    bal = np.zeros((nv, n + 1), dtype=np.int64)
    bal[0, 0] += 1                      # k_ext enters at vertex 0
    bal[d.out_vertex, 0] -= 1           # and leaves at the out-vertex
    for j in range(2 * n - 1):
        bal[d.g_dst[j]] += d.g_mom[j]
        bal[d.g_src[j]] -= d.g_mom[j]
    for i in range(n):
        bal[2 * i + 1] += d.v_mom[i]
        bal[2 * i] -= d.v_mom[i]
    return int(np.abs(bal).max())
