"""CPU checks of the specialised-kernel generator (no device): the generated
source of a small graph compiles for sm_103a, and a large graph splits into
modules whose slice functions are each defined exactly once."""
import os
import re
import shutil
import subprocess

import pytest

from paper_2403_18840_gb300 import api, fdgraph

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2403_18840_gb300", "csrc")


def _tape(order, with_dk):
    return fdgraph.compile_graph(order, fdgraph.graph_roots(order, with_dk=with_dk), budget=8192).to_bytes()


def test_small_graph_is_one_module_with_every_root_flushed():
    tape = _tape(2, True)
    src, n_mod = api.jit_source(tape, 0, threads=128, min_blocks=2, max_modules=8)
    assert n_mod == 1
    roots = fdgraph.graph_roots(2, with_dk=True)
    flushes = re.findall(r"flush<(\d+), (\d+), (\d+)>", src)
    assert sorted(int(r) for r, _, _ in flushes) == list(range(len(roots)))
    for r, n, dk in flushes:
        assert (int(n), int(dk)) == (roots[int(r)][0], 1 if roots[int(r)][3] else 0)
    assert "__launch_bounds__(128, 2)" in src


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")
def test_generated_source_compiles(tmp_path):
    src, _ = api.jit_source(_tape(2, True), 0, threads=128, min_blocks=2, max_modules=1)
    f = tmp_path / "m0.cu"
    f.write_text(src)
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-cubin",
                        "-I", CSRC, "-o", str(tmp_path / "m0.cubin"), str(f)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]


@pytest.mark.parametrize("root_units", [False, True])
def test_large_graph_splits_into_linked_modules(root_units):
    tape = _tape(5, False)
    _, n_mod = api.jit_source(tape, 0, threads=128, min_blocks=2, max_modules=8, root_units=root_units)
    assert 2 <= n_mod <= 8
    unit = "fd_r" if root_units else "fd_s"
    ret = "float2" if root_units else "float"
    defined, declared, slices = [], set(), []
    for m in range(n_mod):
        src, _ = api.jit_source(tape, m, threads=128, min_blocks=2, max_modules=8, root_units=root_units)
        defined += re.findall(r'extern "C" __device__ __noinline__ %s (%s\d+)\(' % (ret, unit), src)
        declared |= set(re.findall(r'extern "C" __device__ %s (%s\d+)\(const FdSV &V' % (ret, unit), src))
        slices += re.findall(r"__device__ __\w+__ float (fd_s\d+)\(const FdSVT<float, \d+> &V, const FdPar &Q\) \{", src)
        assert ("fd_jit_kernel" in src) == (m == 0)
    assert len(defined) == len(set(defined))
    assert declared <= set(defined)
    assert slices and len(slices) == len(set(slices))   # every slice emitted exactly once
    body, _ = api.jit_source(tape, 0, threads=128, min_blocks=2, max_modules=8, root_units=root_units)
    called = set(re.findall(r"= (%s\d+)\(V" % unit, body))
    assert called == set(defined)
    if root_units:
        assert len(defined) == len(fdgraph.graph_roots(5))


@pytest.mark.parametrize("pair,cross", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("unit_cap", [0, 6000, 100000])
def test_sample_loop_units_cover_every_slice_once(unit_cap, pair, cross):
    # spt > 1: units pack consecutive slices of one root (of several roots with
    # cross_roots); every slice emitted once (in packed two-lane arithmetic
    # with pair), every unit called once, every root flushed once per sample
    tape = _tape(5, False)
    kw = dict(threads=256, min_blocks=1, max_modules=8, spt=4, unit_cap=unit_cap, pair=pair, cross_roots=cross)
    _, n_mod = api.jit_source(tape, 0, **kw)
    slices, units = [], []
    vt = "FdF2" if pair else "float"
    for m in range(n_mod):
        src, _ = api.jit_source(tape, m, **kw)
        slices += re.findall(r"__device__ __forceinline__ %s (fd_s\d+)\(const FdSVT<%s, \d+> &V, const FdPar &Q\) \{"
                             % (vt, vt), src)
        if pair:   # every unit defined here packs two samples per pass
            assert src.count("fd_pack(") == len(re.findall(r"__noinline__ void fd_u\d+", src))
        units += re.findall(r"__device__ __noinline__ void (fd_u\d+)\(", src)
    body, _ = api.jit_source(tape, 0, **kw)
    assert slices and len(slices) == len(set(slices))
    assert sorted(re.findall(r"(fd_u\d+)\(V, Q, LC, cs, sn, re, im\)", body)) == sorted(units)
    flushes = re.findall(r"flush(?:_samples)?<(\d+), ", body)
    assert sorted(int(r) for r in flushes) == list(range(len(fdgraph.graph_roots(5))))
    if unit_cap == 0:
        assert len(units) == len(slices)             # one slice per unit
    if unit_cap == 100000:   # one unit per root; across roots, one unit for the whole graph
        assert len(units) == (1 if cross else len(fdgraph.graph_roots(5)))


@pytest.mark.parametrize("kw", [dict(spt=3, pair=True), dict(spt=1, pair=True), dict(spt=4, pair=True, leaf_calls=True),
                                dict(spt=1, sv_smem=True), dict(spt=1, cross_roots=True)])
def test_sample_loop_options_reject_invalid_combinations(kw):
    # packed pairs need an even number of samples per thread and inlined
    # leaves; inputs in shared memory need the sample loop
    with pytest.raises(api.L.FdError):
        api.jit_source(_tape(2, False), 0, threads=256, min_blocks=1, **kw)


@pytest.mark.parametrize("order", [3, 5])
def test_executed_work_model(order):
    # one unit across all roots computes every leaf once: the tape's own work;
    # smaller units recompute leaves, more so when they may not span roots
    data = fdgraph.compile_graph(order, fdgraph.graph_roots(order), budget=8192).to_bytes()
    assert fdgraph.specialised_work(data, True, 10 ** 9, True) == fdgraph.tape_work(data)
    for cap in (6000, 12000):
        per_root = fdgraph.specialised_work(data, True, cap, False)
        cross = fdgraph.specialised_work(data, True, cap, True)
        assert fdgraph.tape_work(data)[0] <= cross[0] <= per_root[0]
        assert fdgraph.tape_work(data)[1] <= cross[1] <= per_root[1]


def test_contraction_ops_below_the_naive_diagram_sum():
    # naive: every diagram a product of 2n - 1 G and n V leaves, then summed
    diagrams = {2: 3, 3: 20, 4: 189}
    ratios = []
    for n, d in diagrams.items():
        ops = fdgraph.contraction_ops(fdgraph.compile_graph(n, [(n, 0, 0, 0)], budget=8192).to_bytes())
        naive = d * (3 * n - 2) + (d - 1)
        assert ops < naive
        ratios.append(naive / ops)
    assert ratios == sorted(ratios)          # the compression grows with the order
    assert fdgraph.contraction_ops(fdgraph.compile_graph(4, [(4, 0, 0, 0)], budget=8192).to_bytes()) == 721


@pytest.mark.parametrize("kw", [dict(spt=2, sv_smem=True, leaf_cache=32), dict(spt=1, leaf_cache=96)])
def test_leaf_cache_stores_each_family_once_and_units_read_it(kw):
    # fd_leaves computes every cached family once per sample and stores its
    # values at distinct offsets [float][sample][thread]; the units read those
    # offsets instead of computing the family (at most leaf_cache floats)
    tape = _tape(4, True)
    T, spt = 256, kw["spt"]
    src, n_mod = api.jit_source(tape, 0, threads=T, min_blocks=1, max_modules=1, unit_cap=6000, **kw)
    assert n_mod == 1
    head = src[src.index("fd_leaves(const FdSV *Vb"):src.index("static __device__ __forceinline__ float fd_s")]
    stores = [int(m) for m in re.findall(r"  L\[(\d+)\] = c\d+\[\d+\];", head)]
    assert stores and len(stores) == len(set(stores)) <= kw["leaf_cache"]
    assert all(s % (T * spt) == 0 for s in stores)
    body = src.replace(head, "")
    loads = set(int(m) for m in re.findall(r"[{ ]L\[(\d+)\]", body))
    assert loads and loads <= set(stores)
    assert "fd_leaves(V, Q, LC);" in src
    assert re.search(r"jit_main_loop<FdBody, 4, 15, \d+, 256, %d, %d, %d, false>" % (spt, T if kw.get("sv_smem") else 1,
                                                                              len(stores)), src)


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")
def test_leaf_cache_source_compiles(tmp_path):
    src, _ = api.jit_source(_tape(3, True), 0, threads=256, min_blocks=1, max_modules=1, spt=2, sv_smem=True,
                            leaf_cache=24)
    f = tmp_path / "lc.cu"
    f.write_text(src)
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-cubin",
                        "-I", CSRC, "-o", str(tmp_path / "lc.cubin"), str(f)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]


@pytest.mark.parametrize("kw", [dict(leaf_cache=-1), dict(leaf_cache=8, spt=2, pair=True),
                                dict(leaf_cache=8, leaf_calls=True)])
def test_leaf_cache_rejects_invalid_options(kw):
    with pytest.raises(api.L.FdError):
        api.jit_source(_tape(2, False), 0, threads=256, min_blocks=1, **kw)


@pytest.mark.parametrize("cap,K", [(6000, 32), (12000, 96), (0, 48)])
def test_work_model_caches_what_the_generator_caches(cap, K):
    # fdgraph.specialised_work's leaf-cache selection (the executed-work model
    # the benchmark reports) picks the same families as the generator
    tape = _tape(4, True)
    src, _ = api.jit_source(tape, 0, threads=256, min_blocks=1, max_modules=1, spt=2, unit_cap=cap, leaf_cache=K)
    head = src[src.index("fd_leaves(const FdSV *Vb"):src.index("static __device__ __forceinline__ float fd_s")]
    stores = len(re.findall(r"  L\[\d+\] = c\d+\[\d+\];", head))
    assert stores == fdgraph.specialised_work(tape, True, cap, leaf_cache=K, return_cache=True)
    assert fdgraph.specialised_work(tape, True, cap, leaf_cache=K)[0] < fdgraph.specialised_work(tape, True, cap)[0]
