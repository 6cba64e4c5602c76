"""The integrand's per-sample device arithmetic (csrc/fd_jit_rt.cuh) compiled
for the host and run on the CPU against the FP64 oracle (Eqs. propagator,
green_ct, interaction_ct, sigma_integration; Sec. IV's spherical map).

The kernels compute the sampler map, the loop momenta and eps = |p|^2 - mu in
double-float arithmetic, so that eps is exact up to its final FP32 rounding
even where it is a small difference near the Fermi surface, and evaluate the
single G line of the order-1 diagram in FP64 (its mu-derivatives vanish at
points the value has no other term to hide).  These tests hold the host build
of that code to the per-sample bound the GPU tests use: every sample within
2e-5 of the oracle's L1 magnitude M(x), at least 99.9 % within 1e-5.  (The
host build evaluates exp with the C library, the kernels with the MUFU
approximation; the GPU tests cover that difference.)"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import workloads
from oracle import conventions, integrand as oig, philox as ophilox, vegas as ovegas
from paper_2403_18840_gb300 import api, fdgraph

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2403_18840_gb300", "csrc")


def _build(tmp_path_factory, name):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp(name) / name)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "native", name + ".cu"), "-o", out], check=True, capture_output=True)
    return out


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    return _build(tmp_path_factory, "integrand_host")


@pytest.fixture(scope="module")
def kin_exe(tmp_path_factory):
    return _build(tmp_path_factory, "kin_host")


def run_host(exe, tmp_path, tape, order, roots, x32, P, edges=None):
    hdr = struct.unpack("<16I", tape[:64])
    n_slots, n_instr, ins_off = hdr[5], hdr[6], hdr[8]
    words = np.frombuffer(tape[ins_off:ins_off + 8 * n_instr], np.uint64)
    rw = np.array([n | (m << 8) | (l << 16) | (dk << 24) for (n, m, l, dk) in roots], np.uint32)
    dim, n = x32.shape
    nb = 0 if edges is None else edges.shape[1] - 1
    src, dst = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(src, "wb") as f:
        np.array([n, dim, order, n_instr, n_slots, len(roots), nb], np.int32).tofile(f)
        np.array([P.kext, P.mu, P.beta, P.Lambda, P.kc], np.float64).tofile(f)
        words.tofile(f)
        rw.tofile(f)
        np.ascontiguousarray(x32, np.float32).tofile(f)
        if nb:
            np.ascontiguousarray(edges, np.float32).tofile(f)
    subprocess.run([exe, src, dst], check=True)
    return np.fromfile(dst, np.float32).reshape(len(roots), 2, n).astype(np.float64)


def _rel(f, ref, mag):
    err = np.abs(f[:, 0] - ref.real) + np.abs(f[:, 1] - ref.imag)
    err = np.maximum(err - 1e-30, 0.0)            # FP32 underflow of values below ~1e-38
    return err / np.maximum(mag, 1e-30)


def _check(rel, label):
    frac = float(np.mean(rel <= 1e-5))
    print("%s: max err/M %.3e, frac <= 1e-5: %.5f" % (label, rel.max(), frac))
    assert rel.max() <= 2e-5, (label, rel.max())
    assert frac >= 0.999, (label, frac)


@pytest.mark.parametrize("order,with_dk,n,seed", [(1, True, 16384, 71), (2, True, 16384, 72),
                                                  (3, True, 8191, 73), (4, True, 1537, 74), (5, False, 1025, 70)])
def test_host_build_per_sample_parity(exe, tmp_path, order, with_dk, n, seed):
    roots = fdgraph.graph_roots(order, with_dk=with_dk)
    tape = api.tape_bytes(order, roots)
    P = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    x = ophilox.uniforms(seed, 0, 0, np.arange(n), 4 * order - 1)
    f = run_host(exe, tmp_path, tape, order, roots, x, P)
    ref, mag = oig.eval_roots(x, roots, P, with_l1=True)
    _check(_rel(f, ref, mag), "host order %d" % order)


def test_host_build_on_a_vegas_grid(exe, tmp_path):
    """Mapped coordinates (FP32 edges, double-float map): the oracle maps the
    same uniforms through the same edges in FP64."""
    order, n = 3, 4099
    dim = 4 * order - 1
    d = workloads.histogram_like(9, dim, 1024)
    e = ovegas.vegas_update(ovegas.uniform_edges(dim, 1024), d, 0.7).astype(np.float32).astype(np.float64)
    e[:, 0], e[:, -1] = 0.0, 1.0
    roots = fdgraph.graph_roots(order, with_dk=True)
    P = conventions.ueg_params(2.0, 1.0 / 25.0, 1.0, 0.5)
    u = ophilox.uniforms(75, 0, 0, np.arange(n), dim)
    f = run_host(exe, tmp_path, api.tape_bytes(order, roots), order, roots, u, P, edges=e)
    xm, J, _ = ovegas.vegas_map(e, u)
    ref, mag = oig.eval_roots(xm, roots, P, with_l1=True)
    nb = e.shape[1] - 1
    _, _, i = ovegas.vegas_map(e, u)
    rows = np.arange(dim)[:, None]
    jd = nb * (e[rows, i + 1] - e[rows, i])
    jr = np.stack([np.prod(jd[:4 * r[0] - 1], axis=0) for r in roots])
    _check(_rel(f, ref * jr, mag * jr), "host order 3 on a VEGAS grid")


def test_loop_momenta_double_float(kin_exe, tmp_path):
    """The kernels' double-float momenta (table-based cos / sin of 2 pi c,
    double-float radius and polar factors) against the oracle's FP64 map.
    A component is a grid part (a multiple of g = 2^-9 at r_s = 1) plus an
    FP32 remainder |lo| <= g / 2, whose rounding is at most 2^-35 ~ 3e-11:
    each component within 1e-10, against ~6e-8 |k| for an FP32 momentum."""
    order, n = 5, 20000
    P = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    x = ophilox.uniforms(76, 0, 0, np.arange(n), 4 * order - 1)
    # the corners of the angles: c at the table nodes and halfway, b near 0 and 1
    x[2, :8] = np.array([0.0, 0.25, 0.5, 0.75, 1.0 / 512, 3.0 / 512, 0.9999999, 2.0 ** -24])
    x[1, 8:12] = np.array([2.0 ** -24, 1.0 - 2.0 ** -24, 0.5, 0.25])
    # points on the cube's faces (a flow's FP32 samples can saturate to 0 or 1)
    x[1, 12], x[1, 13], x[0, 14], x[2, 15], x[0, 16] = 0.0, 1.0, 0.0, 1.0, 1.0
    x = x.astype(np.float32)
    src, dst = str(tmp_path / "k.in"), str(tmp_path / "k.out")
    with open(src, "wb") as f:
        np.array([n, order], np.int32).tofile(f)
        np.array([P.kc], np.float64).tofile(f)
        x.tofile(f)
    subprocess.run([kin_exe, src, dst], check=True)
    k = np.fromfile(dst, np.float64).reshape(order, 3, n)
    assert np.all(np.isfinite(k))
    kref, _, _ = oig.map_hypercube(x.astype(np.float64), order, P)
    err = np.abs(k - kref[1:])
    print("double-float momenta: max err %.2e" % err.max())
    assert err.max() <= 1e-10


def test_host_build_order1_at_the_fermi_surface(exe, tmp_path):
    """The order-1 roots' G families (m <= 4 mu-derivatives, with and without
    the k-derivative) at points where |k_1|^2 - mu lies within 1e-4 .. 1e-2 of
    the Fermi surface (both signs) or anywhere in |eps| <= 1 = 0.27 E_F, where
    the mu-derivatives of the equal-time line cross zero (at beta eps of order
    one).  Each root is a single term there, so its value has to hold 1e-5 of
    itself where it is small: the double-float evaluation of eps, the Fermi
    factor and the Taylor recurrences does (an FP32 family misses the bound
    by orders of magnitude).  The lower end 1e-4 is set by the kinematics:
    the momenta's FP32 remainders carry eps to ~1e-10, and the even
    derivatives vanish linearly at eps = 0."""
    n = 16384
    roots = [(1, m, 0, dk) for m in range(5) for dk in (0, 1)]
    P = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    rng = np.random.default_rng(2024)
    eps = np.where(rng.random(n) < 0.5, 1.0, -1.0) * np.where(
        np.arange(n) % 2 == 0, 10.0 ** rng.uniform(-4.0, -2.0, n), rng.uniform(0.0, 1.0, n))
    x = ophilox.uniforms(77, 0, 0, np.arange(n), 3)
    x[0] = np.sqrt(P.mu + eps) / P.kc
    x = x.astype(np.float32).astype(np.float64)
    f = run_host(exe, tmp_path, api.tape_bytes(1, roots), 1, roots, x, P)
    ref, mag = oig.eval_roots(x, roots, P, with_l1=True)
    _check(_rel(f, ref, mag), "host order 1 at the Fermi surface")


@pytest.fixture(scope="module")
def df_exe(tmp_path_factory):
    return _build(tmp_path_factory, "df_host")


def test_double_float_exp_and_reciprocal(df_exe, tmp_path):
    """The order-1 family's double-float exponential (Cody-Waite reduction
    with ln 2 in three FP32 parts, expm1 by a Taylor series, four squarings)
    and reciprocal (a Newton step) against exact-rational references: exp(y)
    for double-float y in [-103, 0] (the family's arguments -beta |eps| are
    never positive) within 1e-13 relative while exp(y) >= 2^-100 (the low
    half is a normal FP32 number), within the FP32 rounding 2^-24 relative
    or 2^-148 absolute below (0 from -103 on); 1 / d for double-float d in
    [1, 2] within 4e-14 relative (one Newton step: ~2^-46)."""
    from fractions import Fraction
    import math
    rng = np.random.default_rng(5)
    n = 4000
    yv = np.concatenate([-10.0 ** rng.uniform(-9.0, math.log10(103.0), n - 8),
                         [0.0, -1e-30, -0.34657359, -0.34657360, -87.0, -88.0, -103.0, -104.0]])
    yh = yv.astype(np.float32)
    yl = (yv - yh.astype(np.float64)).astype(np.float32)
    dv = 1.0 + rng.random(n)
    dv[:4] = [1.0, 2.0, 1.0 + 2.0 ** -23, 2.0 - 2.0 ** -22]
    dh = dv.astype(np.float32)
    dl = (dv - dh.astype(np.float64)).astype(np.float32)
    src, dst = str(tmp_path / "df.in"), str(tmp_path / "df.out")
    with open(src, "wb") as f:
        np.array([n], np.int32).tofile(f)
        np.stack([yh, yl], 1).astype(np.float32).tofile(f)
        np.stack([dh, dl], 1).astype(np.float32).tofile(f)
    subprocess.run([df_exe, src, dst], check=True)
    out = np.fromfile(dst, np.float32).reshape(2, n, 2).astype(np.float64)
    worst_e = worst_r = 0.0
    for i in range(n):
        y = Fraction(float(yh[i])) + Fraction(float(yl[i]))
        # exp of the exact double-float argument: the FP64 exp of its nearest
        # double times the exp of the tiny remainder (|r| < 2^-53 |y|)
        yd = float(y)
        ref = math.exp(yd) * (1.0 + float(y - Fraction(yd)))
        got = out[0, i, 0] + out[0, i, 1]
        if ref >= 2.0 ** -100:
            worst_e = max(worst_e, abs(got - ref) / ref)
        else:
            assert abs(got - ref) <= max(2.0 ** -24 * ref, 2.0 ** -148), (yd, got, ref)
        d = Fraction(float(dh[i])) + Fraction(float(dl[i]))
        r = float(1 / d)
        worst_r = max(worst_r, abs(out[1, i, 0] + out[1, i, 1] - r) / r)
    print("double-float exp: max rel %.2e; reciprocal: max rel %.2e" % (worst_e, worst_r))
    assert worst_e <= 1e-13 and worst_r <= 4e-14


@pytest.mark.parametrize("order,rs,T,lam,kext,n,seed", [(3, 2.0, 1.0 / 25.0, 1.0, 0.4, 4097, 81),
                                                         (3, 4.0, 1.0 / 25.0, 1.0, 1.6, 4097, 82),
                                                         (5, 4.0, 1.0 / 25.0, 1.0, 2.0, 513, 83),
                                                         (4, 5.0, 1.0 / 40.0, 1.375, 1.0, 1537, 84)])
def test_host_build_at_other_densities(exe, tmp_path, order, rs, T, lam, kext, n, seed):
    """The batched configuration's other densities and external momenta
    (r_s 2 and 4, k up to 2 k_F) and the production point of the effective
    mass (r_s 5, T = T_F / 40, lambda_R = 1.375 k_F: sharper Fermi factors):
    k_F, mu and beta change, and with them the loop momenta's grid and the
    instance split of the parameters."""
    roots = fdgraph.graph_roots(order, with_dk=order < 5)
    P = conventions.ueg_params(rs, T, lam, kext)
    x = ophilox.uniforms(seed, 0, 0, np.arange(n), 4 * order - 1)
    f = run_host(exe, tmp_path, api.tape_bytes(order, roots), order, roots, x, P)
    ref, mag = oig.eval_roots(x, roots, P, with_l1=True)
    _check(_rel(f, ref, mag), "host order %d at r_s %g, T = %.4f T_F, k = %g k_F" % (order, rs, T, kext))
