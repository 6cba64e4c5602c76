"""The construction's diagrams with the construction's own momentum routing,
evaluated by the oracle (the per-sample reference for a tape compiled from
the Dyson-Schwinger / parquet graph): every diagram's sign equals the
oracle's for the same topology, and every diagram equals the oracle's
routing of the same topology sample by sample after the change of loop
variables p = A k + b k_ext (|det A| = 1) that maps one routing onto the
other, for the mu- and Lambda-derivative roots.  (A k-derivative at fixed
loop variables changes with the routing when b != 0; only its integral is
routing-independent.)"""
import numpy as np
import pytest

import parquet_oracle
from oracle import conventions, diagrams as od, integrand as ig
from paper_2403_18840_gb300 import parquet as P


def _key(n, sigma):
    X = 2 * n
    succ = tuple(-1 if sigma[v] == X else sigma[v] for v in range(2 * n))
    pred = [None] * (2 * n)
    for v in range(2 * n):
        if sigma[v] != X:
            pred[sigma[v]] = v
    pred[pred.index(None)] = -1
    return P.canonical((succ, tuple(pred), tuple(v ^ 1 for v in range(2 * n))))


@pytest.fixture(scope="module")
def construction():
    return P.Construction()


@pytest.mark.parametrize("n", [2, 3, 4])
def test_signs_equal_the_oracles(construction, n):
    ref = {_key(n, t.sigma): float((-1) ** (n + t.F) * 2 ** t.F) for t in od.self_energy_topologies(n)}
    for w, d in parquet_oracle.routed_diagrams(n, construction):
        assert ref[_key(n, d.sigma)] == d.sign


def _piece_of(n, d):
    succ = tuple(-1 if w == 2 * n else w for w in d.sigma)
    pred = [None] * (2 * n)
    for v in range(2 * n):
        if succ[v] >= 0:
            pred[succ[v]] = v
    pred[pred.index(None)] = -1
    return succ, tuple(pred), tuple(v ^ 1 for v in range(2 * n))


def _vertex_map(n, dp, do):
    """Vertex correspondence parquet -> oracle through the canonical order."""
    pp, po = _piece_of(n, dp), _piece_of(n, do)
    assert P.canonical(pp) == P.canonical(po)
    op = P._dfs_order(*pp, pp[1].index(-1))
    oo = P._dfs_order(*po, po[1].index(-1))
    return dict(zip(op, oo))


def _loop_change(n, dp, do, vmap):
    """(A, b) with p = A k + b k_ext: the parquet loop momenta p in terms of
    the oracle's k such that every line carries the same momentum."""
    rows, rhs = [], []
    line_o = {(int(s), int(t)): e for e, (s, t) in enumerate(zip(do.g_src, do.g_dst))}
    for e, (s, t) in enumerate(zip(dp.g_src, dp.g_dst)):
        eo = line_o[(vmap[int(s)], vmap[int(t)])]
        rows.append(dp.g_mom[e]), rhs.append(do.g_mom[eo])
    for i in range(n):
        a, b = vmap[2 * i], vmap[2 * i + 1]
        io, sgn = a // 2, (1 if a < b else -1)          # the oracle's line may run the other way
        rows.append(dp.v_mom[i]), rhs.append(sgn * do.v_mom[io])
    R, S = np.array(rows, dtype=float), np.array(rhs, dtype=float)
    # R[:, 1:] (A k + b k_ext) + R[:, 0] k_ext = S[:, 1:] k + S[:, 0] k_ext
    A = np.linalg.lstsq(R[:, 1:], S[:, 1:], rcond=None)[0]
    b = np.linalg.lstsq(R[:, 1:], S[:, 0] - R[:, 0], rcond=None)[0]
    assert np.allclose(R[:, 1:] @ A, S[:, 1:], atol=1e-12) and np.allclose(R[:, 1:] @ b, S[:, 0] - R[:, 0], atol=1e-12)
    assert abs(abs(np.linalg.det(A)) - 1.0) < 1e-12
    return A, b


@pytest.mark.parametrize("n", [2, 3, 4])
def test_each_diagram_equals_the_oracles_under_a_change_of_loop_variables(construction, n):
    # the parquet-routed diagram at p = A k + b k_ext equals the oracle-routed
    # one at k, sample by sample, for every mu- and Lambda-derivative root
    Pm = conventions.ueg_params(1.0, 0.1, 1.0, 1.0)
    oracle = {P.canonical(_piece_of(n, d)): d for d in od.routed_self_energy(n)}
    rng = np.random.default_rng(30 + n)
    N = 64
    kvec = rng.normal(0, 1.5, (n + 1, 3, N))
    kvec[0] = 0.0
    kvec[0, 2] = 1.3                                     # k_ext along z
    tau_o = np.concatenate([np.zeros((1, N)), rng.uniform(0, Pm.beta, (n - 1, N))])
    for w, dp in parquet_oracle.routed_diagrams(n, construction):
        do = oracle[P.canonical(_piece_of(n, dp))]
        vmap = _vertex_map(n, dp, do)
        A, b = _loop_change(n, dp, do, vmap)
        kp = np.concatenate([kvec[:1], np.einsum("ij,jcn->icn", A, kvec[1:]) + b[:, None, None] * kvec[0]])
        tau_p = np.stack([tau_o[vmap[2 * i] // 2] for i in range(n)])
        for (m, l) in ((0, 0), (1, 0), (0, 1), (1, 1)):
            vp = ig.diagram_value(dp, kp, tau_p, Pm, m, l, 0)
            vo = ig.diagram_value(do, kvec, tau_o, Pm, m, l, 0)
            assert np.allclose(vp, vo, rtol=1e-9, atol=1e-12 * np.abs(vo).max()), (m, l)
