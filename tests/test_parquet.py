"""The Dyson-Schwinger / parquet construction of self-energy diagrams (Sec.
II.B-C) against brute force: the 4-point vertices it builds equal every
connected, amputated, tadpole-free 4-leg diagram found by trying all
fermion permutations (orders 0-2), each exactly once; the self-energy
diagrams it builds equal the oracle's enumerated topologies (every Wick
contraction, reduced to canonical form; orders 1-5), each exactly once, and
at order 6 (31 130 diagrams) the compiler's own enumeration."""
import pytest

from oracle import diagrams as od
from paper_2403_18840_gb300 import fdgraph
from paper_2403_18840_gb300 import parquet as P


def _piece_of_topology(n, sigma):
    """A self-energy topology (fermion permutation, X = 2n the external line,
    interaction lines (2i, 2i+1)) as a piece with one in- and one out-leg."""
    X = 2 * n
    succ = tuple(-1 if sigma[v] == X else sigma[v] for v in range(2 * n))
    pred = [None] * (2 * n)
    for v in range(2 * n):
        if sigma[v] != X:
            pred[sigma[v]] = v
    assert pred.count(None) == 1
    pred[pred.index(None)] = -1
    return succ, tuple(pred), tuple(v ^ 1 for v in range(2 * n))


@pytest.fixture(scope="module")
def construction():
    return P.Construction()


@pytest.mark.parametrize("N", [0, 1, 2])
def test_vertices_equal_brute_force(construction, N):
    gen = construction.gamma4(N)
    assert set(gen.values()) == {1}
    assert set(gen) == set(P.brute_gamma4(N + 1))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_self_energy_equals_enumeration(construction, n):
    gen = construction.sigma(n)
    assert set(gen.values()) == {1}
    ref = [P.canonical(_piece_of_topology(n, t.sigma)) for t in od.self_energy_topologies(n)]
    assert len(set(ref)) == len(ref)
    assert set(gen) == set(ref)


def test_channels_exclusive_and_irreducible_parts(construction):
    # every order-2 vertex is reducible in exactly one channel (none is fully
    # irreducible below order 3), and the construction's channel parts are
    # the reducible ones
    g4 = construction.gamma4(2)
    for key in g4:
        p = P.from_key(key)
        assert sum(P.reducible(p, c) for c in P.CHANNELS) == 1
    for c in P.CHANNELS:
        assert set(construction.phi(c, 2)) == {k for k in g4 if P.reducible(P.from_key(k), c)}


def test_canonical_keys_ignore_labels():
    # the same diagram under a relabelling of its vertices has one key
    succ, pred, partner = _piece_of_topology(3, od.self_energy_topologies(3)[5].sigma)
    perm = [4, 2, 5, 0, 1, 3]
    inv = {perm[v]: v for v in range(6)}

    def m(w):
        return perm[w] if w >= 0 else w
    relab = tuple(tuple(m(arr[inv[u]]) for u in range(6)) for arr in (succ, pred, partner))
    assert P.canonical(relab) == P.canonical((succ, pred, partner))


def test_vertex_enumerator_equals_brute_force():
    for m in (1, 2, 3):
        assert set(P.enumerate_gamma4(m)) == set(P.brute_gamma4(m))


def test_fully_irreducible_vertices(construction):
    # none at orders 1 and 2; at order 3 the envelope diagrams, irreducible
    # in every channel by the direct two-line cut test
    assert construction.irreducible(1) == {} and construction.irreducible(2) == {}
    env = construction.irreducible(3)
    assert len(env) == 64
    for key in env:
        p = P.from_key(key)
        assert not any(P.reducible(p, c) for c in P.CHANNELS)


def test_order6_equals_the_compilers_enumeration(construction):
    gen = construction.sigma(6)
    assert len(gen) == 31130 and set(gen.values()) == {1}
    ref = {P.canonical(_piece_of_topology(6, d.sigma)) for d in fdgraph.self_energy_diagrams(6)}
    assert set(gen) == ref
