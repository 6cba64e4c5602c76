"""Test infrastructure: the self-energy diagrams of the Dyson-Schwinger /
parquet construction, each with the momentum routing the construction gives
it, as the oracle's routed diagrams.  The oracle then evaluates them with its
own leaves, derivatives and map (`oracle.integrand.diagram_value`).  This is
the per-sample reference for a tape compiled from the construction, whose
routing differs from the oracle's convention.  Only the line-to-momentum
assignment comes from the construction, and the tests check it for
momentum conservation at every vertex."""
from fractions import Fraction

import numpy as np

from oracle import diagrams as od
from paper_2403_18840_gb300 import parquet_graph as PG


def _loops(n, succ, out_v):
    """Closed fermion loops: succ cycles that do not contain the external path."""
    on_path = set()
    v = 0
    while True:
        on_path.add(v)
        if v == out_v:
            break
        v = succ[v]
    seen, loops = set(on_path), 0
    for s in range(2 * n):
        if s in seen:
            continue
        loops += 1
        v = s
        while v not in seen:
            seen.add(v)
            v = succ[v]
    return loops


def routed_diagrams(n, construction):
    """[(weight, oracle RoutedDiagram)] of Sigma^(n) from the construction."""
    root = PG.Evaluator(n, PG.Expanded(), construction).root()
    out = []
    for out_v, monos in sorted(root.items()):
        for w, mono in monos:
            succ = [None] * (2 * n)
            gl, vl = [], {}
            for leaf in mono:
                if leaf[0] == "G":
                    _, m, x, y = leaf
                    succ[x] = y
                    gl.append((x, y, m))
                else:
                    _, m, a, b = leaf
                    vl[a // 2] = (a, b, m)
            X = 2 * n
            succ[out_v] = X
            F = _loops(n, succ, out_v)
            g_mom = np.zeros((2 * n - 1, n + 1), dtype=np.int64)
            g_src = np.zeros(2 * n - 1, dtype=np.int64)
            g_dst = np.zeros(2 * n - 1, dtype=np.int64)
            g_tau = np.zeros((2 * n - 1, 2), dtype=np.int64)
            for e, (x, y, m) in enumerate(sorted(gl)):
                g_mom[e] = m
                g_src[e], g_dst[e] = x, y
                g_tau[e] = (y // 2, x // 2)
            v_mom = np.zeros((n, n + 1), dtype=np.int64)
            for i in range(n):
                a, b, m = vl[i]
                assert (a, b) == (2 * i, 2 * i + 1)
                v_mom[i] = m
            sign = (-1) ** (n + F) * 2 ** F
            d = od.RoutedDiagram(n=n, sigma=tuple(succ), sign=float(sign), out_vertex=out_v,
                                 g_src=g_src, g_dst=g_dst, g_mom=g_mom, v_mom=v_mom, g_tau=g_tau)
            assert od.check_conservation(d) == 0
            # the graph's weight is the diagram's sign and spin factor times
            # its share: 1, or 2^-k for the 2^k routings of a diagram with k
            # nested pp joins
            share = Fraction(w) / sign
            assert share > 0 and (1 / share).denominator == 1 and ((1 / share).numerator & ((1 / share).numerator - 1)) == 0, \
                (w, sign)
            out.append((float(share), d))
    return out
