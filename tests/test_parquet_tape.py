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
    # order 5, all 15 roots: fewer contraction operations and fewer flops per
    # sample (leaf families included) than the present compiler's tape
    roots = fdgraph.graph_roots(5)
    pq = PG.parquet_tape(5, roots, construction=construction).to_bytes()
    present = fdgraph.compile_graph(5, roots).to_bytes()
    assert fdgraph.contraction_ops(pq) < 0.75 * fdgraph.contraction_ops(present)
    assert fdgraph.tape_work(pq)[0] < 0.8 * fdgraph.tape_work(present)[0]


def _leaf_functions_dk(order, seed, lam=0.6):
    # leaves that depend on the momentum through p^2 = (mom . var)^2, var[0]
    # the external momentum; their k_ext-derivatives in closed form
    rng = np.random.default_rng(seed)
    tau = rng.uniform(0, 1, order)
    var0 = rng.normal(0, 1, order + 1)

    def make(var):
        def p(mom):
            return float(np.dot(mom, var[:len(mom)]))

        def base(p2, dst, src):
            return math.exp(-0.3 * p2) * (1 + 0.5 * math.sin(tau[dst] - tau[src] + p2))

        def dbase(p2, dst, src):
            return -0.3 * base(p2, dst, src) + math.exp(-0.3 * p2) * 0.5 * math.cos(tau[dst] - tau[src] + p2)

        def g_leaf(mom, dst, src, j):
            return base(p(mom) ** 2, dst, src) * 0.3 ** j / math.factorial(j)

        def gd_leaf(mom, dst, src, j):
            return dbase(p(mom) ** 2, dst, src) * 2 * p(mom) * mom[0] * 0.3 ** j / math.factorial(j)

        def v_cq(mom):
            return 1.0 + 0.1 * p(mom) ** 2, 0.5 + p(mom) ** 2

        def v_leaf(mom, j):
            c, q2 = v_cq(mom)
            r = 1.0 / (q2 + lam)
            return c * (-1) ** j * r ** (j + 1)

        def vd_leaf(mom, j):
            c, q2 = v_cq(mom)
            r = 1.0 / (q2 + lam)
            d_dp2 = (-1) ** j * (0.1 * r ** (j + 1) - c * (j + 1) * r ** (j + 2))
            return d_dp2 * 2 * p(mom) * mom[0]
        return g_leaf, gd_leaf, v_leaf, vd_leaf, v_cq
    return make, var0, lam


@pytest.mark.parametrize("order", [3, 4])
def test_parquet_tape_k_derivative_roots(construction, order):
    roots = fdgraph.graph_roots(order, with_dk=True)
    data = PG.parquet_tape(order, roots, construction=construction).to_bytes()
    assert _load_ok_or_nodevice(data)
    make, var0, lam = _leaf_functions_dk(order, 20 + order)
    g_leaf, gd_leaf, v_leaf, vd_leaf, _ = make(var0)
    got = tape_exec.run(data, g_leaf, v_leaf, gd_leaf, vd_leaf)
    h = 1e-5

    def series_at(shift, n):
        var = var0.copy()
        var[0] += shift
        g, _, _, _, v_cq = make(var)
        return PG.Evaluator(n, PG.BiSeries(lambda mom, x, y, i: g(mom, y, x, i), v_cq, lam, order - n),
                            construction).root()
    cache = {}
    for r, (n, m, l, dk) in enumerate(roots):
        f = math.factorial(m) * math.factorial(l)
        if n not in cache:
            cache[n] = (series_at(0.0, n), series_at(h, n), series_at(-h, n))
        s0, sp, sm = cache[n]
        if dk == 0:
            want = {o: s[(m, l)] * f for o, s in s0.items() if (m, l) in s}
        else:
            want = {o: (sp[o][(m, l)] - sm[o][(m, l)]) / (2 * h) * f for o in s0 if (m, l) in s0[o]}
        scale = max(abs(x) for x in want.values()) + 1e-300
        for o in want:
            assert abs(got[r].get(o, 0.0) - want[o]) < (1e-10 if dk == 0 else 1e-6) * scale, (n, m, l, dk, o)


@pytest.mark.parametrize("order,with_dk", [(3, True), (4, False)])
def test_parquet_tape_with_oracle_leaves_equals_the_oracle(construction, order, with_dk):
    # the tape's arithmetic on the oracle's leaf values (Taylor coefficients
    # of G0 in mu and V in Lambda, and their k_ext derivatives) at a sample's
    # momenta and times equals the oracle evaluating the construction's
    # routed diagrams at that sample, root by root and out line by out line
    import parquet_oracle
    from oracle import conventions, integrand as ig
    from oracle.leaves import G0_deriv, V_deriv
    Pm = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    roots = fdgraph.graph_roots(order, with_dk=with_dk)
    data = PG.parquet_tape(order, roots, construction=construction).to_bytes()
    diags = {n: parquet_oracle.routed_diagrams(n, construction) for n in range(1, order + 1)}
    x = np.random.default_rng(40 + order).random((ig.dim_of_order(order), 3))
    # moderate loop momenta (radius coordinates below a quarter of the cutoff):
    # far out the propagators are so small that products of several of them
    # underflow FP64 differently in different multiplication orders
    for j in range(order):
        x[0 if j == 0 else 4 * j - 1] *= 0.25
    kvec, tau, _ = ig.map_hypercube(x, order, Pm)
    for s in range(x.shape[1]):
        def p_of(mom):
            return sum(c * kvec[j, :, s] for j, c in enumerate(mom))

        def g_leaf(mom, dst, src, j):
            p = p_of(mom)
            return float(G0_deriv(np.array([p @ p - Pm.mu]), np.array([tau[dst, s] - tau[src, s]]), Pm.beta, j)[0]) \
                / math.factorial(j)

        def gd_leaf(mom, dst, src, j):
            p = p_of(mom)
            d = G0_deriv(np.array([p @ p - Pm.mu]), np.array([tau[dst, s] - tau[src, s]]), Pm.beta, j + 1)[0]
            return float(-2.0 * mom[0] * p[2] * d) / math.factorial(j)

        def v_leaf(mom, j):
            q = p_of(mom)
            return float(V_deriv(np.array([q @ q]), Pm.Lambda, j)[0]) / math.factorial(j)

        def vd_leaf(mom, j):
            q = p_of(mom)
            return float(2.0 * mom[0] * q[2] * V_deriv(np.array([q @ q]), Pm.Lambda, j + 1)[0]) / math.factorial(j)
        got = tape_exec.run(data, g_leaf, v_leaf, gd_leaf, vd_leaf)
        for r, (n, m, l, dk) in enumerate(roots):
            want, l1 = {}, 0.0
            for w, d in diags[n]:
                val, mag = ig.diagram_value(d, kvec[:n + 1, :, s:s + 1], tau[:n, s:s + 1], Pm, m, l, dk,
                                            return_abs=True)
                line = d.out_vertex // 2
                want[line] = want.get(line, 0.0) + w * val[0]
                l1 += abs(w * d.sign) * mag[0]
            # the terms cancel: compare on the scale of their L1 magnitude
            for line, v in want.items():
                assert abs(got[r].get(line, 0.0) - v) <= 1e-12 * l1, (s, n, m, l, dk, line)


def test_parquet_tape_specialised_source_compiles(construction, tmp_path):
    # the run-time code generator accepts a parquet tape and its kernel
    # source compiles for sm_103a (cross-compiled here)
    import os
    import shutil
    import subprocess
    from paper_2403_18840_gb300 import api
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    tape = PG.parquet_tape(3, fdgraph.graph_roots(3, with_dk=True), construction=construction).to_bytes()
    src, _ = api.jit_source(tape, 0, threads=128, min_blocks=2, max_modules=1)
    f = tmp_path / "m0.cu"
    f.write_text(src)
    csrc = os.path.join(os.path.dirname(os.path.abspath(PG.__file__)), "csrc")
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-cubin",
                        "-I", csrc, "-o", str(tmp_path / "m0.cubin"), str(f)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
