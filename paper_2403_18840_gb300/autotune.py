"""Autotuner for the integrand launch: tape schedule x CTA shape.

Two sets of knobs decide the interpreter's speed and are tuned per graph and
device by timing real launches:
  * the tape schedule (per-sample slot budget for leaf families and
    temporaries, FMA bundle width, lookahead window of the bundler), which
    trades recomputed leaves against shared-memory occupancy;
  * the CTA shape (threads x samples per thread).
Results are cached per (graph, device) in _build/autotune.json.
"""
import json
import os

import torch

from . import api

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
SCHEDULES = [dict(budget=b, bundle=w, window=8 * w) for b in (96, 128, 160) for w in (4, 8)]
SHAPES = [(128, 2), (256, 1), (128, 1), (64, 2)]


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


def _time(G, params, n, reps=2):
    plan = api.EvalPlan([G], [params], [0], n)
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
    cache[key] = best
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp%d" % os.getpid()
    json.dump(cache, open(tmp, "w"), indent=1)
    os.replace(tmp, CACHE)
    return best


def tuned_graph(order, roots, params, **kw):
    """Graph compiled and configured with the tuned schedule and CTA shape."""
    best = tune(order, roots, params, **kw)
    G = api.Graph(order, roots=roots, budget=best["budget"], bundle=best["bundle"], window=best["window"])
    G.set_launch(best["threads"], best["spt"])
    return G, best
