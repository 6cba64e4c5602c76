"""Production protocol of the effective mass (App. B): at each temperature a
scan over the screening parameter lambda_R, the choice of the lambda_R whose
last partial sums of m*/m vary least (`analysis.choose_screening`: its
estimate and a systematic uncertainty from the variation among it and its
neighbours), and the linear extrapolation of those estimates to T = 0
(`analysis.extrapolate_linear_T`), each temperature weighted by its
statistical and systematic uncertainties added in quadrature.

Every (lambda_R, T) point is one `meff_run.run`: all orders up to N_max on the
GPU (the parquet tape from the order given, a trained flow proposal at the
highest order when asked), the post-process and its statistical errors.

    python -m paper_2403_18840_gb300.production_run --rs 5 \
        --lam 1.0 1.25 1.375 1.5 --T 0.025 0.03333 0.05 \
        [--max-order 6] [--samples 26] [--iters 50] [--adapt 8] [--flow-steps 2000]

(--lam in units of k_F, --T in units of T_F, --samples is log2 of the
samples per iteration.)  Prints one JSON line per (lambda_R, T) point as it
finishes and a final line with the choice at each temperature and the T = 0
extrapolation.
"""
import argparse
import json
import math

from . import analysis


def protocol(runner, lams, temps, last=3):
    """runner(lam_over_kF, T_over_TF) -> {"meff": partial sums for N = 1..N_max,
    "meff_err": their statistical errors, ...}.  Returns the scan and choice
    at every temperature and the T = 0 extrapolation (None with fewer than two
    distinct temperatures)."""
    per_T = []
    for T in temps:
        scan, errs = {}, {}
        for lam in lams:
            out = runner(lam, T)
            scan[lam] = [float(v) for v in out["meff"]]
            errs[lam] = [float(v) for v in out["meff_err"]]
        lam_star, est, sys_err = analysis.choose_screening(scan, last)
        per_T.append({"T_over_TF": T, "lam_over_kF": lam_star, "estimate": est,
                      "stat": errs[lam_star][-1], "sys": sys_err,
                      "scan": {repr(lam): scan[lam] for lam in lams},
                      "scan_err": {repr(lam): errs[lam] for lam in lams}})
    ext = None
    if len({p["T_over_TF"] for p in per_T}) >= 2:
        t = [p["T_over_TF"] for p in per_T]
        y = [p["estimate"] for p in per_T]
        dy = [math.hypot(p["stat"], p["sys"]) for p in per_T]
        fit = analysis.extrapolate_linear_T(t, y, dy)
        ext = {"meff_T0": fit["y0"], "err_T0": fit["dy0"], "alpha": fit["alpha"], "dalpha": fit["dalpha"],
               "chi2_dof": fit["chi2_dof"]}
    return {"per_T": per_T, "T0": ext}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rs", type=float, default=5.0)
    ap.add_argument("--lam", type=float, nargs="+", default=[1.0, 1.25, 1.375, 1.5])
    ap.add_argument("--T", type=float, nargs="+", default=[1.0 / 40.0, 1.0 / 30.0, 1.0 / 20.0])
    ap.add_argument("--max-order", type=int, default=6)
    ap.add_argument("--samples", type=int, default=26, help="log2 of the samples per iteration")
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--adapt", type=int, default=8)
    ap.add_argument("--flow-steps", type=int, default=0, help="> 0: the highest order with a trained flow proposal")
    ap.add_argument("--parquet-from", type=int, default=6, help="orders from this one use the parquet tape")
    args = ap.parse_args()
    from . import meff_run

    def runner(lam, T):
        out = meff_run.run(args.rs, args.max_order, 1 << args.samples, args.iters, args.adapt, T_over_TF=T,
                           lam_over_kF=lam, flow_steps=args.flow_steps, parquet_from=args.parquet_from)
        print(json.dumps(out, default=float), flush=True)
        return out

    res = protocol(runner, args.lam, args.T)
    res["rs"] = args.rs
    print(json.dumps(res, default=float), flush=True)


if __name__ == "__main__":
    main()
