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
    bad_magic = b"XXXX" + good[4:]
    assert _load(bad_magic) == L.FD_EFORMAT
    assert _load(good[:40]) == L.FD_EFORMAT                      # truncated
    hdr = list(struct.unpack("<16I", good[:64]))
    # an instruction pointing past the slot count
    words = list(struct.unpack("<%dQ" % hdr[6], good[hdr[8]:hdr[8] + 8 * hdr[6]]))
    w = words[0]
    w = (w & ~(8191 << 6)) | (8000 << 6)
    bad = bytearray(good)
    bad[hdr[8]:hdr[8] + 8] = struct.pack("<Q", w)
    assert _load(bytes(bad)) == L.FD_EFORMAT
    # unknown opcode
    bad = bytearray(good)
    bad[hdr[8]:hdr[8] + 8] = struct.pack("<Q", (words[0] & ~63) | 42)
    assert _load(bytes(bad)) == L.FD_EFORMAT
    # missing END
    bad = bytearray(good)
    last = hdr[8] + 8 * (hdr[6] - 1)
    bad[last:last + 8] = struct.pack("<Q", words[0])
    assert _load(bytes(bad)) == L.FD_EFORMAT
    assert b"END" in L.lib().fd_last_error() or len(L.lib().fd_last_error()) > 0


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_compiler_topologies_match_oracle(n):
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
