"""Efficiency of VEGAS-MCMC and NF-MCMC relative to VEGAS importance sampling,
order by order (Sec. V, Fig. benchmark_MC): Re Sigma^(n)(k_F, i w0) of the
single-root order-n graph of the uniform electron gas (r_s = 1, lambda = k_F,
T/T_F = 1/32), n = 1..5.

Per order: the graph's tuned specialised kernel, a VEGAS grid adapted over
12 x 2^22 samples, an affine coupling flow on the grid's coordinates trained
on |f|; then VEGAS and flow importance sampling (`driver.compare`) and the
chains with either proposal (`driver.mcmc_compare`: alpha from a scan, the
efficiency from an independent draw).  With --spline the paper's own flow
(App. A: rational-quadratic spline couplings, 8 bins, a residual conditioner
of width 32, uniform base) is trained the same way with the temperature
annealing of App. A (the target at 4 T at first, lowered to T over the first
half of the steps) and compared in both roles against VEGAS and the affine
flow.  The figure of merit is
1 / (variance x seconds); ratios are taken against VEGAS importance sampling
with its pooled and its median batch variance.

    python -m paper_2403_18840_gb300.mcmc_benchmark [--orders 1 2 3 4 5] [--flow-steps 1000] [--spline]

prints one JSON line per order and a summary line.
"""
import argparse
import json
import time

from . import api, autotune, driver


def run_order(order, flow_steps, batch=1 << 20, n_compare=1 << 24, n_chains=1 << 12, n_steps=1 << 12,
              alphas=(0.1, 0.3, 0.5, 0.7, 0.9), T_over_TF=1.0 / 32.0, seed=41, spline=False):
    t0 = time.perf_counter()
    params = api.ueg_params(order, 1.0, T_over_TF, 1.0, 1.0)
    G, _ = autotune.tuned_jit_graph(order, [(order, 0, 0, 0)], params)
    V = api.Vegas(G.dim, 1024)
    driver.adapt_vegas(G, params, V, 1 << 22, 12, seed=seed)
    F = api.Flow(G.dim, 8, 128, seed=seed)
    driver.train_flow(G, params, F, V, steps=flow_steps, batch=batch, lr=1e-3, seed=seed, vegas_steps=100,
                      evals_per_batch=4, defensive=0.1)
    cmp = driver.compare(G, params, V, F, n_compare, seed=seed + 7, batches=8, defensive=0.1)
    mc = driver.mcmc_compare(G, params, V, F, n_chains, n_steps, alphas, seed=seed + 31)
    ref_pooled = cmp["vegas"]["samples_per_s"] / cmp["vegas"]["var_per_sample"]
    ref_median = cmp["vegas"]["samples_per_s"] / cmp["vegas"]["var_median"]
    out = {"order": order, "dim": G.dim, "T_over_TF": T_over_TF,
           "vegas": {k: cmp["vegas"][k] for k in ("mean", "err", "samples_per_s")},
           "flow_is": {k: cmp["flow"][k] for k in ("mean", "err", "samples_per_s")},
           "flow_is_over_vegas": {"pooled": cmp["flow_over_vegas"], "median": cmp["flow_over_vegas_median"]}}
    for name in ("vegas_mcmc", "nf_mcmc"):
        m = mc[name]
        out[name] = {k: m[k] for k in ("alpha", "mean", "err", "accepted", "seconds")}
        out[name + "_over_vegas"] = {"pooled": m["merit"] / ref_pooled, "median": m["merit"] / ref_median}
    out["nf_over_vegas_mcmc"] = mc["nf_mcmc"]["merit"] / mc["vegas_mcmc"]["merit"]
    if spline:
        S = api.SplineFlow(G.dim, 8)
        driver.train_flow(G, params, S, V, steps=flow_steps, batch=batch, lr=1e-3, seed=seed + 1,
                          vegas_steps=100, evals_per_batch=4, anneal=(4.0, flow_steps // 2))
        cs = driver.compare(G, params, V, S, n_compare, seed=seed + 7, batches=8)
        ms = driver.mcmc_compare(G, params, V, S, n_chains, n_steps, alphas, seed=seed + 31)
        m = ms["nf_mcmc"]
        out["spline_is"] = {k: cs["flow"][k] for k in ("mean", "err", "samples_per_s")}
        out["spline_is_over_vegas"] = {"pooled": cs["flow_over_vegas"], "median": cs["flow_over_vegas_median"]}
        out["nf_mcmc_spline"] = {k: m[k] for k in ("alpha", "mean", "err", "accepted", "seconds")}
        out["nf_mcmc_spline_over_vegas"] = {"pooled": m["merit"] / ref_pooled, "median": m["merit"] / ref_median}
        out["nf_mcmc_spline_over_affine"] = m["merit"] / mc["nf_mcmc"]["merit"]
    out["seconds_total"] = time.perf_counter() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--orders", type=int, nargs="+", default=[1, 2, 3, 4, 5])
    ap.add_argument("--flow-steps", type=int, default=1000)
    ap.add_argument("--chains", type=int, default=1 << 12)
    ap.add_argument("--steps", type=int, default=1 << 12)
    ap.add_argument("--spline", action="store_true", help="also the spline flow (App. A) in both roles")
    args = ap.parse_args()
    rows = []
    for n in args.orders:
        r = run_order(n, args.flow_steps, n_chains=args.chains, n_steps=args.steps, spline=args.spline)
        rows.append(r)
        print(json.dumps(r), flush=True)
    print(json.dumps({"summary": [{"order": r["order"],
                                   "vegas_mcmc_over_vegas_median": r["vegas_mcmc_over_vegas"]["median"],
                                   "nf_mcmc_over_vegas_median": r["nf_mcmc_over_vegas"]["median"],
                                   "nf_over_vegas_mcmc": r["nf_over_vegas_mcmc"],
                                   "nf_mcmc_spline_over_vegas_median":
                                       r.get("nf_mcmc_spline_over_vegas", {}).get("median"),
                                   "nf_mcmc_spline_over_affine": r.get("nf_mcmc_spline_over_affine")}
                                  for r in rows]}), flush=True)


if __name__ == "__main__":
    main()
