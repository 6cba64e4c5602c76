"""The Dyson-Schwinger / parquet graphs compiled into the tape format: the
library's loader accepts the tapes, and executing their arithmetic (a plain
CPU executor of the format, leaves from test functions) gives every root
(n, m, l) per out line as the construction's own Taylor series in (mu,
Lambda) does, with fewer operations than the present compiler's tapes."""
import ctypes
import math

import numpy as np
import pytest

import tape_exec
from paper_2403_18840_gb300 import _lib as L
from paper_2403_18840_gb300 import fdgraph
from paper_2403_18840_gb300 import parquet as P
from paper_2403_18840_gb300 import parquet_graph as PG


@pytest.fixture(scope="module")
def construction():
    return P.Construction()


def _leaf_functions(order, seed, lam=0.6):
    rng = np.random.default_rng(seed)
    var, tau = rng.normal(0, 1, order + 1), rng.uniform(0, 1, order)

    def p2(mom):                                   # even in the momentum (the tape keeps it up to sign)
        return float(np.dot(mom, var[:len(mom)])) ** 2

    def g_leaf(mom, line_dst, line_src, j):
        base = math.exp(-0.3 * p2(mom)) * (1 + 0.5 * math.sin(tau[line_dst] - tau[line_src] + p2(mom)))
        return base * 0.3 ** j / math.factorial(j)

    def v_cq(mom):
        return 1.0 + 0.1 * p2(mom), 0.5 + p2(mom)

    def v_leaf(mom, j):
        c, q2 = v_cq(mom)
        r = 1.0 / (q2 + lam)
        return c * r * (-r) ** j
    return g_leaf, v_leaf, v_cq, lam


def _load_ok_or_nodevice(data):
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(data, len(data))
    st = L.lib().fd_graph_load(buf, len(data), ctypes.byref(h))
    if st == L.FD_OK:
        L.lib().fd_graph_free(h)
    return st in (L.FD_OK, L.FD_ECUDA)


@pytest.mark.parametrize("order,budget", [(3, 96), (4, 96), (4, 8192), (5, 96)])
def test_parquet_tape_executes_every_root(construction, order, budget):
    roots = fdgraph.graph_roots(order)
    tape = PG.parquet_tape(order, roots, budget=budget, construction=construction)
    data = tape.to_bytes()
    assert _load_ok_or_nodevice(data)
    g_leaf, v_leaf, v_cq, lam = _leaf_functions(order, order)
    got = tape_exec.run(data, g_leaf, v_leaf)
    series = {}
    for r, (n, m, l, _) in enumerate(roots):
        if n not in series:
            g0 = lambda mom, x, y, i: g_leaf(mom, y, x, i)
            series[n] = PG.Evaluator(n, PG.BiSeries(g0, v_cq, lam, order - n), construction).root()
        want = {o: s[(m, l)] * math.factorial(m) * math.factorial(l) for o, s in series[n].items() if (m, l) in s}
        scale = max(abs(x) for x in want.values())
        assert set(got[r]) == set(want), (n, m, l)
        for o in want:
            assert abs(got[r][o] - want[o]) < 1e-10 * scale, (n, m, l, o)


def test_parquet_tape_needs_fewer_operations(construction):
    roots = fdgraph.graph_roots(5)
    pq = fdgraph.contraction_ops(PG.parquet_tape(5, roots, construction=construction).to_bytes())
    present = fdgraph.contraction_ops(fdgraph.compile_graph(5, roots).to_bytes())
    assert pq < present / 3
