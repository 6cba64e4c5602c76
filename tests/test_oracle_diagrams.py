"""Pins for the brute-force topology enumeration and the routing convention."""
import math

import numpy as np
import pytest

from oracle import diagrams as dg


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_orbit_sizes(n):
    # no automorphisms once the external legs are fixed: every topology is hit
    # by exactly (n-1)! 2^(n-1) permutations with sigma(X) = 0, and together
    # they exhaust the (2n)! - (disconnected) permutations
    tops = dg.all_connected(n)
    mult = {t.multiplicity for t in tops}
    assert mult == {math.factorial(n - 1) * 2 ** (n - 1)}
    assert len(tops) * math.factorial(n - 1) * 2 ** (n - 1) <= math.factorial(2 * n)


def _compositions_product(counts, n):
    # number of chains G0 S G0 S ... G0 of proper pieces with orders summing to n
    total = 0

    def rec(rem, acc):
        nonlocal total
        if rem == 0:
            total += acc
            return
        for k in range(1, rem + 1):
            rec(rem - k, acc * counts[k])
    rec(n, 1)
    return total


def test_dyson_relation():
    # connected Green's-function diagrams are chains of 1PI self-energy pieces
    # (Eq. Dyson); this must hold with and without tadpoles
    N = 4
    conn = {n: dg.all_connected(n) for n in range(1, N + 1)}
    pi_all = {n: sum(t.one_pi for t in conn[n]) for n in conn}
    pi_clean = {n: sum(t.one_pi and t.tadpole_free for t in conn[n]) for n in conn}
    g_clean = {n: sum(t.tadpole_free for t in conn[n]) for n in conn}
    for n in range(1, N + 1):
        assert len(conn[n]) == _compositions_product(pi_all, n)
        assert g_clean[n] == _compositions_product(pi_clean, n)


def test_order1_and_order2_by_hand():
    # order 1: only the exchange (Fock) diagram; order 2: rainbow (Fock
    # insertion), crossed exchange and the bubble with one fermion loop
    t1 = dg.self_energy_topologies(1)
    assert [t.sigma for t in t1] == [(1, 2)]
    t2 = dg.self_energy_topologies(2)
    loops = sorted(t.F for t in t2)
    assert loops == [0, 0, 1]
    signs = sorted(dg.route(t).sign for t in t2)
    assert signs == [-2.0, 1.0, 1.0]


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_routing_conservation_and_irreducibility(n):
    # independent check of the enumerator's filters through the routing: a
    # fermion line that carries no loop momentum is a bridge (not 1PI); an
    # interaction line with zero momentum is a tadpole
    for t in dg.all_connected(n):
        d = dg.route(t)
        assert dg.check_conservation(d) == 0
        g_has_loop = np.any(d.g_mom[:, 1:] != 0, axis=1)
        v_nonzero = np.any(d.v_mom != 0, axis=1)
        assert t.one_pi == bool(np.all(g_has_loop))
        assert t.tadpole_free == bool(np.all(v_nonzero))
        # loop momenta: every k_j appears on exactly one chord as +1 alone
        for j in range(1, n + 1):
            alone = [(row[j] == 1 and np.count_nonzero(row[1:]) == 1 and row[0] == 0)
                     for row in d.g_mom]
            assert sum(alone) >= 1


def test_self_energy_counts_small():
    assert [len(dg.self_energy_topologies(n)) for n in (1, 2, 3)] == [1, 3, 20]
