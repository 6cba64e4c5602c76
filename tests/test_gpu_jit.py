"""GPU parity of the specialised (straight-line, run-time compiled) integrand
kernels against the FP64 oracle, and their agreement with the interpreter."""
import numpy as np
import pytest

import parity

import workloads
from oracle import conventions, integrand as oig, philox as ophilox, vegas as ovegas

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_GRAPHS = {}


@pytest.fixture(scope="module")
def api():
    from paper_2403_18840_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def _jit_graph(api, order, with_dk):
    key = (order, with_dk)
    if key not in _GRAPHS:
        G = api.Graph(order, with_dk=with_dk, budget=8192)
        info = G.jit()
        assert info["enabled"] and info["regs"] > 0 and info["modules"] >= 1
        _GRAPHS[key] = G
    return _GRAPHS[key]


def _gparams(api, order, rs=1.0, kk=1.0):
    return api.ueg_params(order, rs, 1.0 / 25.0, 1.0, kk)


def _oracle(order, roots, n, seed, inst=0, kk=1.0, rs=1.0, it=0):
    P = conventions.ueg_params(rs, 1.0 / 25.0, 1.0, kk)
    x = ophilox.uniforms(seed, it, inst, np.arange(n), 4 * order - 1)
    return oig.eval_roots(x, roots, P, with_l1=True)


def _compare(f, ref, mag, label):
    # the interpreter's criterion (tests/parity.py)
    parity.check(parity.rel_error(f, ref, mag), label)


def _run(api, G, order, n, seed, maps=None, points=None, point_w=None, kk=1.0):
    plan = api.EvalPlan([G], [_gparams(api, order, kk=kk)], [0], n, maps=maps, per_sample=True)
    stats = plan.run(seed, 0, points=points, point_w=point_w)
    torch.cuda.synchronize()
    return plan.per_sample[0].cpu().numpy().astype(np.float64), stats[0].cpu().numpy(), plan


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("with_dk", [False, True])
def test_jit_per_sample_parity(api, order, with_dk):
    n = {1: 5000, 2: 3001, 3: 2049, 4: 700}[order]
    G = _jit_graph(api, order, with_dk)
    f, _, _ = _run(api, G, order, n, 17 + order)
    ref, mag = _oracle(order, G.roots, n, 17 + order)
    _compare(f[:len(G.roots)], ref, mag, "jit order %d dk %s" % (order, with_dk))


def test_jit_per_sample_parity_order5(api):
    n = 160
    G = _jit_graph(api, 5, False)
    f, _, _ = _run(api, G, 5, n, 29)
    ref, mag = _oracle(5, G.roots, n, 29)
    _compare(f[:len(G.roots)], ref, mag, "jit order 5")


def test_jit_matches_interpreter(api):
    order, n = 3, 3 * 16384 + 77          # several tiles and a ragged tail
    G = _jit_graph(api, order, True)
    f_jit, st_jit, _ = _run(api, G, order, n, 5)
    G.jit_enable(False)
    try:
        f_int, st_int, _ = _run(api, G, order, n, 5)
    finally:
        G.jit_enable(True)
    scale = np.abs(f_int).max(axis=2, keepdims=True) + 1e-30
    assert np.max(np.abs(f_jit - f_int) / scale) < 1e-4
    # tile partials: means of both paths agree to FP32 summation level
    for r in range(len(G.roots)):
        for c in range(2):
            assert abs(st_jit[r, c, 0] - st_int[r, c, 0]) <= 1e-5 * (np.abs(f_int[r, c]).mean() + 1e-30)
            assert abs(st_jit[r, c, 0] - f_jit[r, c].mean()) <= 1e-6 * (np.abs(f_jit[r, c]).mean() + 1e-30)


def test_jit_bitwise_reproducible(api):
    G = _jit_graph(api, 3, True)
    p = _gparams(api, 3)
    a = api.EvalPlan([G], [p], [0], 40000)
    b = api.EvalPlan([G], [p], [0], 40000)
    a.run(5, 1)
    b.run(5, 1)
    torch.cuda.synchronize()
    assert torch.equal(a.partials, b.partials)


def test_jit_tiny_sample_counts(api):
    G = _jit_graph(api, 2, False)
    for n in (1, 2, 31, 33, 129):
        f, _, _ = _run(api, G, 2, n, 3)
        ref, mag = _oracle(2, G.roots, n, 3)
        err = np.abs(f[:, 0, :] - ref.real) + np.abs(f[:, 1, :] - ref.imag)
        assert np.all(err <= parity.bound(mag))


def _fp32_edges(seed, dim, nb):
    d = workloads.histogram_like(seed, dim, nb)
    e = ovegas.vegas_update(ovegas.uniform_edges(dim, nb), d, 0.7)
    e = e.astype(np.float32).astype(np.float64)
    e[:, 0], e[:, -1] = 0.0, 1.0
    return e

def _root_map_jac(e, y, roots):
    """VEGAS Jacobian of each root's own coordinates (order n: the leading 4n - 1), [R, N]."""
    nb = e.shape[1] - 1
    _, _, i = ovegas.vegas_map(e, y)
    rows = np.arange(e.shape[0])[:, None]
    jd = nb * (e[rows, i + 1] - e[rows, i])               # [D, N]
    return np.stack([np.prod(jd[:4 * r[0] - 1], axis=0) for r in roots])



def test_jit_vegas_map_and_histogram(api):
    order, n, nb = 2, 20000, 64
    G = _jit_graph(api, order, True)
    e = _fp32_edges(31, G.dim, nb)
    hist = {}
    for mode in ("jit", "interp"):
        G.jit_enable(mode == "jit")
        m = api.Vegas(G.dim, nb)
        m.set_edges(e)
        f, _, _ = _run(api, G, order, n, 7, maps=[m])
        hist[mode] = (f, m.hist())
    G.jit_enable(True)
    u = ophilox.uniforms(7, 0, 0, np.arange(n), G.dim)
    x, _, _ = ovegas.vegas_map(e, u)
    jv = _root_map_jac(e, u, G.roots)
    ref, mag = oig.eval_roots(x, G.roots, conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0), with_l1=True)
    _compare(hist["jit"][0][:len(G.roots)], ref * jv, mag * jv, "jit vegas")
    hj, hi = hist["jit"][1], hist["interp"][1]
    assert np.all(hj >= 0) and hj.sum() > 0
    assert np.max(np.abs(hj - hi)) <= 1e-4 * hi.max()


def test_jit_points_on_map(api):
    order, n, nb = 2, 2000, 1024
    G = _jit_graph(api, order, True)
    e = _fp32_edges(21, G.dim, nb)
    m = api.Vegas(G.dim, nb)
    m.set_edges(e)
    y = workloads.uniform_points(22, G.dim, n)
    w = workloads.positive_weights(23, n)
    pts = torch.tensor(y, dtype=torch.float32, device="cuda").contiguous()
    pw = torch.tensor(w, dtype=torch.float32, device="cuda")
    f, _, _ = _run(api, G, order, n, 0, maps=[m], points=pts, point_w=pw)
    y64 = y.astype(np.float32).astype(np.float64)
    x, _, _ = ovegas.vegas_map(e, y64)
    jv = _root_map_jac(e, y64, G.roots) * w[None, :]
    ref, mag = oig.eval_roots(x, G.roots, conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0), with_l1=True)
    _compare(f[:len(G.roots)], ref * jv, mag * jv, "jit points on a map")
    assert np.all(m.hist() == 0.0)


def test_jit_mixed_with_interpreter_in_one_call(api):
    # graph 1 specialised, graphs 0 and 2 interpreted: one call, three launches
    graphs = [api.Graph(1), _jit_graph(api, 2, False), api.Graph(3)]
    specs = [(0, 1, 1.0, 0.5), (1, 2, 2.0, 1.0), (2, 3, 1.0, 2.0), (1, 2, 4.0, 0.0)]
    params = [api.ueg_params(o, rs, 1.0 / 25.0, 1.0, kk) for (_, o, rs, kk) in specs]
    n = 1500
    plan = api.EvalPlan(graphs, params, [g for (g, _, _, _) in specs], n, per_sample=True)
    plan.run(9, 2)
    torch.cuda.synchronize()
    f = plan.per_sample.cpu().numpy().astype(np.float64)
    for j, (gi, o, rs, kk) in enumerate(specs):
        ref, mag = _oracle(o, graphs[gi].roots, n, 9, inst=j, kk=kk, rs=rs, it=2)
        _compare(f[j, :len(graphs[gi].roots)], ref, mag, "mixed inst %d" % j)


def test_jit_captured_iteration(api):
    from paper_2403_18840_gb300 import driver
    graphs = [_jit_graph(api, 2, False), _jit_graph(api, 3, False)]
    params = [api.ueg_params(o, 1.0, 1.0 / 25.0, 1.0, 1.0) for o in (2, 3, 3)]
    a = driver.BatchedIteration(graphs, params, [0, 1, 1], 1 << 16, seed=4, n_bins=64)
    b = driver.BatchedIteration(graphs, params, [0, 1, 1], 1 << 16, seed=4, n_bins=64)
    a.capture()
    ra, rb = [], []
    for _ in range(2):
        ra.append(a.replay().clone())
        rb.append(b.step_direct().clone())
    torch.cuda.synchronize()
    # iteration 0: identical inputs -> bitwise equal; afterwards the grids
    # differ in the last bits (FP64 histogram atomics arrive in any order)
    assert torch.equal(ra[0], rb[0])
    x, y = ra[1].cpu().numpy(), rb[1].cpu().numpy()
    assert np.allclose(x[..., 0], y[..., 0], rtol=1e-3, atol=1e-3 * np.abs(y[..., 0]).max())
    assert int(a.d_iter.item()) == 2


@pytest.mark.parametrize("pair,sv_smem,cross", [(False, False, False), (True, False, False), (False, True, False),
                                                (False, True, True), (True, False, True)])
@pytest.mark.parametrize("order,with_dk,n", [(3, True, 2 * 1024 + 77), (5, False, 160)])
def test_jit_sample_loop_variant(api, order, with_dk, n, pair, sv_smem, cross):
    # spt samples per thread, each compilation unit looping over them (with
    # pair: two samples at a time in packed two-lane arithmetic; with sv_smem:
    # the samples' inputs in shared memory; with cross: units spanning roots);
    # a pass covers 256 x 4 samples, so n spans several passes and a ragged tail
    G = api.Graph(order, with_dk=with_dk, budget=8192)
    info = G.jit(threads=256, min_blocks=1, spt=4, unit_cap=6000, pair=pair, sv_smem=sv_smem, cross_roots=cross,
                 sync_every=1 if cross else 0)
    assert info["enabled"]
    f, st, _ = _run(api, G, order, n, 37)
    ref, mag = _oracle(order, G.roots, n, 37)
    _compare(f[:len(G.roots)], ref, mag, "jit spt 4 pair %s sv_smem %s cross %s order %d" % (pair, sv_smem, cross,
                                                                                              order))
    for r in range(len(G.roots)):
        assert abs(st[r, 0, 0] - f[r, 0].mean()) <= 1e-6 * (np.abs(f[r, 0]).mean() + 1e-30)


def test_jit_packed_pairs_match_scalar_loop(api):
    # several tiles and a ragged tail; the packed code does per lane the
    # operations of the scalar code, up to multiply-add contraction
    order, n = 4, 3 * 16384 + 77
    a = api.Graph(order, with_dk=True, budget=8192)
    a.jit(threads=256, min_blocks=1, spt=4, unit_cap=6000, pair=True)
    b = api.Graph(order, with_dk=True, budget=8192)
    b.jit(threads=256, min_blocks=1, spt=4, unit_cap=6000)
    fa, _, _ = _run(api, a, order, n, 5)
    fb, _, _ = _run(api, b, order, n, 5)
    scale = np.abs(fb).max(axis=2, keepdims=True) + 1e-30
    assert np.max(np.abs(fa - fb) / scale) < 1e-5


def test_jit_sample_loop_matches_one_sample_per_thread(api):
    # several tiles and a ragged tail: the loop variant computes the same FP32 values
    order, n = 3, 3 * 16384 + 77
    a = api.Graph(order, with_dk=True, budget=8192)
    a.jit(threads=256, min_blocks=1, spt=4)
    b = _jit_graph(api, order, True)
    fa, _, _ = _run(api, a, order, n, 5)
    fb, _, _ = _run(api, b, order, n, 5)
    scale = np.abs(fb).max(axis=2, keepdims=True) + 1e-30
    assert np.max(np.abs(fa - fb) / scale) < 1e-5


def test_jit_shared_inputs_bitwise_equal_to_local(api):
    # the inputs' storage changes nothing in the arithmetic: several tiles and a
    # ragged tail, VEGAS map and histogram, bitwise equal outputs and partials
    # (the histogram's FP32 shared-memory atomics arrive in any order: FP32-level)
    order, n, nb = 3, 3 * 16384 + 77, 64
    e = _fp32_edges(8, 4 * order - 1, nb)
    out = []
    for sv in (False, True):
        G = api.Graph(order, with_dk=True, budget=8192)
        G.jit(threads=256, min_blocks=1, spt=4, sv_smem=sv)
        m = api.Vegas(G.dim, nb)
        m.set_edges(e)
        f, st, plan = _run(api, G, order, n, 6, maps=[m])
        out.append((f, plan.partials.cpu().numpy(), m.hist()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.allclose(out[0][2], out[1][2], rtol=1e-5, atol=0)


def test_jit_shared_inputs_too_large_is_rejected(api):
    # 256 threads x 16 samples x 68 bytes (order 2: 8 N + 1 words) exceed a block's shared memory
    G = api.Graph(2, budget=8192)
    with pytest.raises(api.L.FdError):
        G.jit(threads=256, min_blocks=1, spt=16, sv_smem=True)
