"""Autotuner for the integrand launch.

Interpreter: two sets of knobs decide its speed and are tuned per graph and
device by timing real launches:
  * the tape schedule (per-sample slot budget for leaf families and
    temporaries, FMA bundle width, lookahead window of the bundler), which
    trades recomputed leaves against shared-memory occupancy;
  * the CTA shape (threads x samples per thread).
Specialised kernels: CTA size, launch-bounds occupancy (which caps the
registers per thread and so trades spills against resident warps), samples
per thread, the compilation unit's size, where the samples' inputs live and
how many floats per sample of leaf families shared by several units are
computed once into shared memory (the leaf cache) rather than per unit.
Results are cached per (graph, device) in _build/autotune.json.
"""
import json
import os

import torch

from . import api

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
SCHEDULES = [dict(budget=b, bundle=w, window=8 * w) for b in (96, 128, 160) for w in (4, 8)]
SHAPES = [(128, 2), (256, 1), (128, 1), (64, 2)]
# specialised-kernel variants (fd_jit_options; unlisted options at their defaults)
JIT_VARIANTS = [dict(threads=256, min_blocks=1, spt=4, unit_cap=12000, sync_every=1, sv_smem=True),
                dict(threads=256, min_blocks=1, spt=4, unit_cap=12000, sv_smem=True),
                dict(threads=256, min_blocks=1, spt=4, unit_cap=9000, sv_smem=True),
                dict(threads=256, min_blocks=1, spt=4, unit_cap=6000, sv_smem=True),
                dict(threads=256, min_blocks=1, spt=2, unit_cap=12000, sync_every=1, sv_smem=True)]
# Not tried by default, all slower than the best of these at order 5 on GB300:
# leaf caches in shared memory (spt 1, 2, 4 with 24 - 128 cached floats: 15 - 31 %
# slower), the leaf cache in a global L2 scratch (320 floats per sample at spt 3
# and 4: 3.2e8 and 2.7e8 against 4.0e8 samples/s) and 3 samples per thread,
# which leaves room for the tile histogram (3.3e8 - 3.4e8); two CTAs of 256
# threads per SM (128 registers, 2 samples per thread: 2.6e8), three of 128
# threads (3.2e8 - 3.5e8), units of cost 16000 (3.4e8) and samples in packed
# pairs (1.5e8 - 2.0e8 at costs 1500 - 6000: 4 KB of local memory at every cost).
JIT_KEYS = ("threads", "min_blocks", "root_units", "sync_every", "leaf_calls", "spt", "unit_cap", "pair", "sv_smem",
            "cross_roots", "leaf_cache", "lc_global")


def _key(order, roots):
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    return "%s|%d|%s" % (name, order, ",".join("%d%d%d%d" % r for r in roots))


def _load():
    if os.path.exists(CACHE):
        try:
            return json.load(open(CACHE))
        except ValueError:
            return {}
    return {}


def _time(G, params, n, reps=2, n_bins=None):
    """ms per launch of n samples (identity sampler, or a uniform VEGAS grid of n_bins with its histogram)."""
    maps = [api.Vegas(G.dim, n_bins)] if n_bins else None
    plan = api.EvalPlan([G], [params], [0], n, maps=maps)
    plan.run(7, 0)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for it in range(reps):
        plan.run(7, it + 1)
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune(order, roots, params, n_samples=1 << 23, schedules=None, shapes=None, force=False, log=None):
    """Best {'budget','bundle','window','threads','spt','samples_per_s'} for this graph.

    Every candidate is timed once; the three fastest are timed again with more
    repetitions and the best of those is kept (single timings are noisy).
    """
    cache = _load()
    key = _key(order, roots)
    if key in cache and not force:
        return cache[key]
    results = []
    for sch in schedules or SCHEDULES:
        G = api.Graph(order, roots=roots, **sch)
        for (t, p) in shapes or SHAPES:
            G.set_launch(t, p)
            try:
                ms = _time(G, params, n_samples)
            except api.L.FdError:
                continue
            r = dict(sch, threads=t, spt=p, slots=G.n_slots, samples_per_s=n_samples / ms * 1e3)
            results.append(r)
            if log:
                log(r)
    best = None
    for r in sorted(results, key=lambda r: -r["samples_per_s"])[:3]:
        G = api.Graph(order, roots=roots, budget=r["budget"], bundle=r["bundle"], window=r["window"])
        G.set_launch(r["threads"], r["spt"])
        ms = _time(G, params, n_samples, reps=5)
        r = dict(r, samples_per_s=n_samples / ms * 1e3)
        if log:
            log(dict(r, final=True))
        if best is None or r["samples_per_s"] > best["samples_per_s"]:
            best = r
    _store(key, best)
    return best


def _store(key, best):
    cache = _load()
    cache[key] = best
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp%d" % os.getpid()
    json.dump(cache, open(tmp, "w"), indent=1)
    os.replace(tmp, CACHE)


def _jit_graph(order, roots, v):
    G = api.Graph(order, roots=roots, budget=1 << 13)
    G.jit(**{k: v[k] for k in JIT_KEYS if k in v})
    return G


def best_load(order, roots, v, params, copies=4, n_samples=1 << 24, reps=2, n_bins=1024):
    """(graph, ms) of the fastest of `copies` loads of the same specialised kernel,
    timed on the production path (a VEGAS grid of n_bins with its histogram).

    The kernel's speed depends on where the CUDA driver places its code (it runs
    ~26k straight-line instructions per sample out of the instruction cache):
    loads of one image in one process differ by up to ~20 %, each stable for
    the life of the load.  The image comes from the compile cache after the
    first load, so a further load costs a library load and a few launches."""
    loads = []                       # all held until the choice, so each load gets new addresses
    for _ in range(copies):
        G = _jit_graph(order, roots, v)
        loads.append((G, _time(G, params, n_samples, reps, n_bins)))
    return min(loads, key=lambda gm: gm[1])


def tune_jit(order, roots, params, n_samples=1 << 24, variants=None, force=False, log=None, copies=3):
    """Best {'threads','min_blocks','root_units','sync_every','leaf_calls','spt','unit_cap','pair','sv_smem',
    'samples_per_s',...} for the specialised kernel, each variant scored at its best of `copies` loads."""
    key = "jit7|" + _key(order, roots)
    cache = _load()
    if key in cache and not force:
        return cache[key]
    best = None
    for v in variants or JIT_VARIANTS:
        v = dict(v)
        try:
            G, ms = best_load(order, roots, v, params, copies, n_samples)
        except api.L.FdError:
            continue
        r = dict(v, samples_per_s=n_samples / ms * 1e3, **{k: G.jit_info()[k] for k in ("regs", "local_bytes")})
        del G
        if log:
            log(r)
        if best is None or r["samples_per_s"] > best["samples_per_s"]:
            best = r
    if best is None:
        raise RuntimeError("no specialised kernel variant could be compiled")
    _store(key, best)
    return best


def tuned_jit_graph(order, roots, params, copies=4, **kw):
    """Graph with its tuned specialised kernel, the fastest of `copies` loads."""
    best = tune_jit(order, roots, params, **kw)
    G, _ = best_load(order, roots, best, params, copies)
    return G, best


def tuned_graph(order, roots, params, **kw):
    """Graph compiled and configured with the tuned schedule and CTA shape."""
    best = tune(order, roots, params, **kw)
    G = api.Graph(order, roots=roots, budget=best["budget"], bundle=best["bundle"], window=best["window"])
    G.set_launch(best["threads"], best["spt"])
    return G, best
