"""Effective mass order by order (Sec. VI.A, Eq. eff_mass_ratio; App. B):
the counterterm-renormalised self-energy and its k-derivative at the Fermi
surface from GPU runs, through the host post-process, with statistical
errors.

For every total order N = 1..N_max one graph carries all roots (n, m, l) with
n + m + l = N and their k-derivatives (Sigma^(n,m,l)(k_F, i w0) and
d Sigma^(n,m,l) / dk).  Its specialised kernel evaluates it on a VEGAS grid
adapted to the graph (the histogram follows the sum of |f| over the value
roots); the highest order may instead take an affine coupling flow on the
grid's coordinates as its proposal (trained on the same |f|, App. A), the
configuration's "flow proposal".  Each iteration is one call of n samples;
the estimate of a root is the mean of the iterations' means and its error
the standard error of those means.  The estimates of all orders go through
the library's post-process (`api.postprocess`: mu counterterms,
a = (1 / 2 k_F) d Re Sigma / dk, b = Im Sigma / w0, m*/m as the xi-series
of (1 - b) / (1 + a)) and the errors through `analysis.meff_with_errors`.

    python -m paper_2403_18840_gb300.meff_run [--rs 1 2] [--max-order 6]
        [--samples 24] [--iters 20] [--adapt 8] [--flow-steps 0] [--parquet-from 6]

(--samples is log2 of the samples per iteration.)  Prints one JSON line per
r_s with the partial sums m*/m(N) and their errors, the per-order seconds
and the kernels' samples/s.
"""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import analysis, api, driver, fdgraph
from . import parquet as _parquet
from . import parquet_graph as _pg

# specialised-kernel variants for the effective-mass graphs (samples per
# thread, their inputs in shared memory, a leaf cache; no tuning per graph).
# The order-6 parquet graph shares its leaf families across many units, so
# its kernel computes 2048 floats of them once per sample into a global (L2)
# scratch: 1.0e7 against 5.9e6 samples/s with the small cache on GB300
# (4096 floats: 1.1e7, but a 15-minute compile).  One sample per thread;
# the unit cost cap hardly matters there, as its largest root-accumulate
# slices (up to 18k FMAs over 1 100 leaf families) are units by themselves.
JIT_VARIANT = dict(threads=256, min_blocks=1, spt=2, unit_cap=12000, sync_every=1, sv_smem=True, leaf_cache=24)
JIT_VARIANT_PARQUET = dict(threads=256, min_blocks=1, spt=1, unit_cap=4000, leaf_cache=2048, lc_global=True)


def _kf(rs):
    return (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs


_CONSTRUCTION = []


def _tape(N, roots, parquet):
    """The order-N tape: enumerated diagrams with hash-consed Horner factorisation,
    or (parquet) the Dyson-Schwinger / parquet evaluation graph (Sec. II.B-C),
    which needs ~2x fewer operations at order 6 with the k-derivative roots."""
    if not parquet:
        return api.tape_bytes(N, roots, budget=1 << 13)
    if not _CONSTRUCTION:
        _CONSTRUCTION.append(_parquet.Construction())
    return _pg.parquet_tape(N, roots, budget=1 << 13, construction=_CONSTRUCTION[0]).to_bytes()


def run_order(N, rs, T_over_TF, lam_over_kF, n, iters, adapt, seed, flow_steps=0, jit=None, parquet=False):
    """Estimates {(n, m, l): complex} of Sigma and d Sigma / dk at k_F for the
    order-N graph, their errors, and timings."""
    roots = fdgraph.graph_roots(N, with_dk=True)
    t0 = time.perf_counter()
    G = api.Graph(N, roots=roots, tape=_tape(N, roots, parquet))
    G.jit(**(jit or (JIT_VARIANT_PARQUET if parquet else JIT_VARIANT)))
    t_compile = time.perf_counter() - t0
    p = api.ueg_params(N, rs, T_over_TF, lam_over_kF, 1.0)
    V = api.Vegas(G.dim, 1024)
    driver.adapt_vegas(G, p, V, min(n, 1 << 22), adapt, seed=seed)
    F = None
    if flow_steps > 0:
        F = api.Flow(G.dim, 8, 128, seed=seed)
        driver.train_flow(G, p, F, V, steps=flow_steps, batch=1 << 18, lr=1e-3, seed=seed + 1, vegas_steps=100,
                          evals_per_batch=4, defensive=0.1)
    plan = api.EvalPlan([G], [p], [0], n, maps=[V])
    means = []
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for it in range(iters):
        if F is None:
            st = plan.run(seed + 17, 1000 + it)
        else:
            x, w, _ = F.sample_defensive(seed + 17, 1000 + it, 3, n, 0.1)
            st = plan.run(seed + 17, 1000 + it, points=x, point_w=w)
        means.append(st[0, :, :, 0].cpu().numpy())          # [R][re, im]
    torch.cuda.synchronize()
    t_eval = time.perf_counter() - t1
    api.device_status()
    m = np.mean(means, axis=0)
    e = np.std(means, axis=0, ddof=1) / math.sqrt(iters) if iters > 1 else np.zeros_like(m)
    sig, sig_e, dsig, dsig_e = {}, {}, {}, {}
    for r, (nn, mm, ll, dk) in enumerate(roots):
        key = (nn, mm, ll)
        if dk:
            dsig[key], dsig_e[key] = complex(m[r, 0], m[r, 1]), complex(e[r, 0], e[r, 1])
        else:
            sig[key], sig_e[key] = complex(m[r, 0], m[r, 1]), complex(e[r, 0], e[r, 1])
    info = {"order": N, "roots": len(roots), "dim": G.dim, "tape": "parquet" if parquet else "enumerated",
            "compile_s": t_compile, "eval_s": t_eval,
            "samples_per_s": n * iters / t_eval, "proposal": "flow" if F is not None else "vegas",
            "jit": G.jit_info()}
    return sig, sig_e, dsig, dsig_e, info


def run(rs, max_order, n, iters, adapt, T_over_TF=1.0 / 25.0, lam_over_kF=1.0, seed=4, flow_steps=0, parquet_from=99):
    sig, sig_e, dsig, dsig_e, infos = {}, {}, {}, {}, []
    for N in range(1, max_order + 1):
        s, se, d, de, info = run_order(N, rs, T_over_TF, lam_over_kF, n, iters, adapt, seed + N,
                                       flow_steps=flow_steps if N == max_order else 0, parquet=N >= parquet_from)
        sig.update(s)
        sig_e.update(se)
        dsig.update(d)
        dsig_e.update(de)
        infos.append(info)
    kF = _kf(rs)
    beta = 1.0 / (T_over_TF * kF * kF)
    Lam = (lam_over_kF * kF) ** 2
    meff, err = analysis.meff_with_errors(max_order, sig, sig_e, dsig, dsig_e, kF, beta, Lam)
    pp = api.postprocess(max_order, sig, dsig, kF, beta, Lam)
    est, trunc = analysis.truncation_estimate(meff[1:]) if max_order >= 3 else (float(meff[-1]), None)
    return {"rs": rs, "T_over_TF": T_over_TF, "lam_over_kF": lam_over_kF, "samples_per_iter": n, "iters": iters,
            "meff": [float(v) for v in meff[1:]], "meff_err": [float(v) for v in err[1:]],
            "estimate": {"meff": est, "stat": float(err[-1]), "truncation": trunc,
                         "rule": "highest-order partial sum; truncation = largest deviation of the last three"},
            "dmu": [float(v) for v in pp["dmu"][1:]], "a": [float(v) for v in pp["a"][1:]],
            "b": [float(v) for v in pp["b"][1:]], "orders": infos}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rs", type=float, nargs="+", default=[1.0, 2.0])
    ap.add_argument("--max-order", type=int, default=6)
    ap.add_argument("--samples", type=int, default=24, help="log2 of the samples per iteration")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--adapt", type=int, default=8)
    ap.add_argument("--flow-steps", type=int, default=0, help="> 0: the highest order with a trained flow proposal")
    ap.add_argument("--parquet-from", type=int, default=6, help="orders from this one use the parquet tape")
    args = ap.parse_args()
    for rs in args.rs:
        out = run(rs, args.max_order, 1 << args.samples, args.iters, args.adapt, flow_steps=args.flow_steps,
                  parquet_from=args.parquet_from)
        print(json.dumps(out, default=float), flush=True)


if __name__ == "__main__":
    main()
