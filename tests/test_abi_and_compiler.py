"""CPU tests of the product's host logic: exported symbols, tape validation,
graph compiler vs the oracle's enumeration/routing, host post-processing."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

from oracle import diagrams as odg
from oracle import postprocess as opp
from paper_2403_18840_gb300 import _lib as L
from paper_2403_18840_gb300 import fdgraph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "fdcore.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = L.lib()
    names = _declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each
    assert not [n for n in names if n not in L.SIGNATURES]


def _load(data):
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(data, len(data))
    return L.lib().fd_graph_load(buf, len(data), ctypes.byref(h))


def test_tape_validation_rejects_malformed_tapes():
    good = fdgraph.compile_graph(2, fdgraph.graph_roots(2)).to_bytes()
    assert _load(good) in (L.FD_OK, L.FD_ECUDA)
    bad_magic = b"XXXX" + good[4:]
    assert _load(bad_magic) == L.FD_EFORMAT
    assert _load(good[:40]) == L.FD_EFORMAT                      # truncated
    hdr = list(struct.unpack("<16I", good[:64]))
    n_instr, off = hdr[6], hdr[8]
    words = list(struct.unpack("<%dQ" % n_instr, good[off:off + 8 * n_instr]))

    def patched(k, w):
        bad = bytearray(good)
        bad[off + 8 * k:off + 8 * k + 8] = struct.pack("<Q", w)
        return bytes(bad)

    # walk the tape: instruction words vs the u16 FMA words that follow a bundle header
    heads, fmas = [], []
    k = 0
    while k < n_instr:
        heads.append(k)
        if words[k] & 63 == fdgraph.OP_BUNDLE:
            n = (words[k] >> 6) & 15
            fmas.extend(range(k + 1, k + 1 + n))
            k += n
        k += 1
    k_b = next(i for i in heads if words[i] & 63 == fdgraph.OP_BUNDLE)
    k_f = k_b + 1
    w = words[k_f]
    # destination slot beyond the declared slot count
    assert _load(patched(k_f, (w & ~0xFFFF) | 16000)) == L.FD_EFORMAT
    # writing a fixed slot (0.0 and the line times are read-only)
    assert _load(patched(k_f, w & ~0xFFFF)) == L.FD_EFORMAT
    assert _load(patched(k_f, (w & ~0xFFFF) | 2)) == L.FD_EFORMAT
    # an operand slot beyond the declared slot count
    assert _load(patched(k_f, (w & ~(0xFFFF << 48)) | (16000 << 48))) == L.FD_EFORMAT
    # unknown opcode
    assert _load(patched(k_b, (words[k_b] & ~63) | 42)) == L.FD_EFORMAT
    # empty bundle, and a bundle longer than the hardware bundle
    assert _load(patched(k_b, words[k_b] & ~(15 << 6))) == L.FD_EFORMAT
    assert _load(patched(k_b, (words[k_b] & ~(15 << 6)) | (9 << 6))) == L.FD_EFORMAT
    # two results of one bundle in the same slot
    nb = (words[k_b] >> 6) & 15
    if nb >= 2:
        w2 = words[k_f + 1]
        assert _load(patched(k_f + 1, (w2 & ~0xFFFF) | (w & 0xFFFF))) == L.FD_EFORMAT
    # a leaf whose momentum mask names a variable beyond the order, or holds the unused code 2
    k_leaf = next(i for i in heads if words[i] & 63 == fdgraph.OP_GLEAF)
    assert _load(patched(k_leaf, words[k_leaf] | (1 << (20 + 2 * 5)))) == L.FD_EFORMAT
    assert _load(patched(k_leaf, (words[k_leaf] & ~(3 << 20)) | (2 << 20))) == L.FD_EFORMAT
    # a root flushed twice (and therefore another one never)
    k_fl = [i for i in heads if words[i] & 63 == fdgraph.OP_RFLUSH]
    assert _load(patched(k_fl[1], words[k_fl[0]])) == L.FD_EFORMAT
    # missing END
    assert _load(patched(n_instr - 1, words[k_leaf])) == L.FD_EFORMAT
    assert len(L.lib().fd_last_error()) > 0


@pytest.mark.parametrize("n", [1, 2, 3, 4, pytest.param(6, marks=pytest.mark.slow)])
def test_compiler_topologies_match_oracle(n):
    # order 6 (the effective-mass configuration): the oracle's brute force visits
    # 12! contractions (about a minute); the compiler must produce the same
    # 110410 connected and 31130 self-energy topologies
    mine = sorted(d.sigma for d in fdgraph.self_energy_diagrams(n))
    ref = sorted(t.sigma for t in odg.self_energy_topologies(n))
    assert mine == ref
    conn = sorted(fdgraph.generate_connected(n))
    assert conn == sorted(t.sigma for t in odg.all_connected(n))


@pytest.mark.parametrize("n", [2, 3, 4])
def test_compiler_routing_matches_oracle(n):
    ref = {d.sigma: d for d in odg.routed_self_energy(n)}
    for d in fdgraph.self_energy_diagrams(n):
        r = ref[d.sigma]
        assert d.sign == r.sign
        assert d.out_line == r.out_vertex // 2
        got_g = [(list(m), la, lb) for (m, la, lb) in d.g_lines]
        exp_g = [(list(r.g_mom[e]), int(r.g_tau[e][0]), int(r.g_tau[e][1])) for e in range(2 * n - 1)]
        assert got_g == exp_g
        assert [list(m) for m in d.v_lines] == [list(v) for v in r.v_mom]


def test_host_postprocess_matches_oracle():
    rng = np.random.default_rng(3)
    N = 4
    sig, dsig = {}, {}
    for n in range(1, N + 1):
        for m in range(N - n + 1):
            for l in range(N - n - m + 1):
                sig[(n, m, l)] = complex(*rng.normal(size=2) * 0.3 ** n)
                dsig[(n, m, l)] = complex(rng.normal() * 0.3 ** n, 0.0)
    shape = (N + 1,) * 3
    sre, sim, dre = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    for k, v in sig.items():
        sre[k], sim[k] = v.real, v.imag
    for k, v in dsig.items():
        dre[k] = v.real
    outs = [np.zeros(N + 1) for _ in range(4)]
    P = ctypes.POINTER(ctypes.c_double)
    st = L.lib().fd_postprocess(N, sre.ctypes.data_as(P), sim.ctypes.data_as(P), dre.ctypes.data_as(P),
                                1.9, 6.8, 0.7, *[o.ctypes.data_as(P) for o in outs])
    assert st == L.FD_OK
    ref = opp.renormalize(sig, dsig, 1.9, 6.8, 0.7, N)
    for name, o in zip(("dmu", "a", "b", "meff"), outs):
        assert np.allclose(o, ref[name], rtol=1e-12, atol=1e-14), name


def test_compiled_tape_is_consistent():
    tp = fdgraph.compile_graph(3, fdgraph.graph_roots(3, with_dk=True))
    data = tp.to_bytes()
    assert len(data) % 16 == 0
    assert _load_ok_or_nodevice(data)


def _load_ok_or_nodevice(data):
    st = _load(data)
    # validation passes; the upload needs a device (FD_ECUDA on a CPU-only host)
    return st in (L.FD_OK, L.FD_ECUDA)


def test_spline_flow_entry_points_validate_arguments_before_any_device_work():
    # null handles and pointers are rejected on the host with FD_EINVAL and a
    # message, without touching a device (this runs without one)
    lib = L.lib()
    f32 = np.zeros(4, dtype=np.float32)
    p = f32.ctypes.data
    loss = np.zeros(4, dtype=np.float64)
    assert lib.fd_nsf_kl_grad(None, p, p, 4, p, loss.ctypes.data, None) == 1
    assert b"required" in lib.fd_last_error()
    assert lib.fd_nsf_train(None, p, p, 4, 1, 1e-3, None, None) == 1
    assert lib.fd_nsf_get_params(None, f32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 4) == 1
    assert lib.fd_nsf_param_count(None) == 0


@pytest.mark.parametrize("case", [
    "vegas_create_dim", "vegas_create_bins", "vegas_set_edges", "vegas_update", "vegas_update_batch",
    "map_samples", "eval_null_graphs", "eval_no_graphs", "eval_null_graph", "accumulate", "flow_create_dim",
    "flow_create_hidden", "flow_sample", "flow_set_tensor_path", "flow_grad", "flow_train", "mcmc_chains",
    "mcmc_estimate", "nsf_create_small", "nsf_create_large", "nsf_set_tensor_path", "postprocess",
    "wait_polls", "graph_load", "measure_peak"])
def test_entry_points_reject_invalid_arguments_on_the_host(case):
    # every entry point answers a null handle or pointer, or a size out of
    # its documented range, with FD_EINVAL and a message before any device
    # work (this runs without a device)
    lib = L.lib()
    f32 = np.zeros(64, dtype=np.float32)
    p = f32.ctypes.data
    f64 = np.zeros(64, dtype=np.float64)
    pd = f64.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    par = L.fd_params(1.0, 1.0, 1.0, 1.0, 1.0, 6.0, 1, 0)
    gi = (ctypes.c_int32 * 1)(0)
    null_graph = (ctypes.c_void_p * 1)(None)
    calls = {
        "vegas_create_dim": lambda: lib.fd_vegas_create(0, 1024, ctypes.byref(h)),
        "vegas_create_bins": lambda: lib.fd_vegas_create(3, 0, ctypes.byref(h)),
        "vegas_set_edges": lambda: lib.fd_vegas_set_edges(None, pd),
        "vegas_update": lambda: lib.fd_vegas_update(None, 0.5, None),
        "vegas_update_batch": lambda: lib.fd_vegas_update_batch(None, -1, 0.5, None),
        "map_samples": lambda: lib.fd_map_samples(None, 1, 0, 0, 16, 3, None, p, None),   # x is required
        "eval_null_graphs": lambda: lib.fd_integrand_eval(None, 1, ctypes.byref(par), gi, 1, None, None, None,
                                                          1, 0, 16, p, None, None),
        "eval_no_graphs": lambda: lib.fd_integrand_eval(null_graph, 0, ctypes.byref(par), gi, 1, None, None,
                                                        None, 1, 0, 16, p, None, None),
        "eval_null_graph": lambda: lib.fd_integrand_eval(null_graph, 1, ctypes.byref(par), gi, 1, None, None,
                                                         None, 1, 0, 16, p, None, None),
        "accumulate": lambda: lib.fd_accumulate(None, 1, 1, 1, p, None),
        "flow_create_dim": lambda: lib.fd_flow_create(0, 8, 128, 1, ctypes.byref(h)),
        "flow_create_hidden": lambda: lib.fd_flow_create(19, 8, 64, 1, ctypes.byref(h)),
        "flow_sample": lambda: lib.fd_flow_sample(None, 1, 0, 0, 16, p, p, None),
        "flow_set_tensor_path": lambda: lib.fd_flow_set_tensor_path(None, 2),
        "flow_grad": lambda: lib.fd_flow_grad(None, p, p, 16, p, None, None),
        "flow_train": lambda: lib.fd_flow_train(None, p, p, 16, 1, 1e-3, None, None),
        "mcmc_chains": lambda: lib.fd_mcmc_chains(None, 1, 16, 1, 16, 4, 0.5, 1, 0, 0, p, p, None),
        "mcmc_estimate": lambda: lib.fd_mcmc_estimate(None, 1, 16, 4, p, None),
        "nsf_create_small": lambda: lib.fd_nsf_create(1, 8, ctypes.byref(h)),
        "nsf_create_large": lambda: lib.fd_nsf_create(25, 8, ctypes.byref(h)),
        "nsf_set_tensor_path": lambda: lib.fd_nsf_set_tensor_path(None, 0),
        "postprocess": lambda: lib.fd_postprocess(0, pd, pd, pd, 1.0, 1.0, 1.0, pd, pd, pd, pd),
        "wait_polls": lambda: lib.fd_debug_set_wait_polls(1 << 32),
        "graph_load": lambda: lib.fd_graph_load(None, 0, ctypes.byref(h)),
        "measure_peak": lambda: lib.fd_measure_peak(9, pd),
    }
    assert calls[case]() == L.FD_EINVAL
    assert lib.fd_last_error()
    assert h.value is None


def test_last_error_is_per_host_thread():
    # the boundary's error message is thread-local: threads failing different
    # calls at once each read back their own message (no device involved)
    import threading
    lib = L.lib()
    got, barrier = {}, threading.Barrier(8)

    def work(k):
        h = ctypes.c_void_p()
        barrier.wait()
        for _ in range(200):
            if k % 2:
                st = lib.fd_vegas_create(0, 64, ctypes.byref(h))
            else:
                st = lib.fd_vegas_create(3, 0, ctypes.byref(h))
            msg = lib.fd_last_error()
            if st != L.FD_EINVAL or msg != (b"dim out of range" if k % 2 else b"n_bins out of range"):
                got[k] = (st, msg)
                return
        got[k] = "ok"

    ts = [threading.Thread(target=work, args=(k,)) for k in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert all(v == "ok" for v in got.values()) and len(got) == 8, got
