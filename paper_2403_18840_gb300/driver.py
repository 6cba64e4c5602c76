"""Monte Carlo drivers: VEGAS adaptation, flow training and sampler comparison.

The integral is I_f = int dx f(x) over the unit hypercube (Sec. IV).  VEGAS
adapts its separable map from the histogram the integrand kernel accumulates;
the learned proposal (Appendix A) is trained by forward KL on samples that the
method itself generates: points drawn from the current sampler q_s carry the
weight |f(x)| / q_s(x), which the integrand kernel returns directly when it is
given the sampler's 1/q as point weights.  The comparison is at equal error
bars: efficiency 1 / (per-sample variance x time per sample).

With `on_vegas` the flow lives in the input coordinates y of the adapted VEGAS
map: x = map(y), and the proposal density is q_flow(y) / J_map(y).  The flow
starts as the identity, so the proposal starts as VEGAS itself and training
adds the correlations between coordinates that a separable grid cannot hold;
its target is |f(map(y))| J_map(y), which the kernel returns when it is given
the map together with the points.
"""
import math

import numpy as np
import torch

from . import api


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def adapt_vegas(G, params, vegas, n, iters, seed, alpha=0.5, first_iter=0):
    """`iters` VEGAS iterations of n samples; returns the per-iteration stats
    [iters][R][2][2] (root, Re/Im, mean/variance of the mean), which
    `analysis.combine_iterations(stats[..., 0], stats[..., 1])` combines with
    inverse-variance weights."""
    plan = api.EvalPlan([G], [params], [0], n, maps=[vegas])
    out = []
    for it in range(iters):
        vegas.clear()
        st = plan.run(seed, first_iter + it)
        vegas.update(alpha)
        out.append(st[0].clone())
    torch.cuda.synchronize()
    return torch.stack(out).cpu().numpy()


def _flow_draw(flow, seed, it, inst, n, defensive):
    """Proposals (x, 1/q) of an affine flow (optionally with its defensive
    uniform share) or a spline flow."""
    if defensive > 0:
        x, w, _ = flow.sample_defensive(seed, it, inst, n, defensive)
        return x, w
    return flow.draw(seed, it, inst, n)


def train_flow(G, params, flow, vegas, steps, batch, lr, seed, vegas_steps=50, evals_per_batch=1, log=None,
               on_vegas=True, defensive=0.0, anneal=None):
    """Forward-KL training of `flow` (affine or spline) on |f|; the first
    `vegas_steps` batches come from VEGAS.

    Every batch is drawn from the current sampler, evaluated by the integrand
    kernel (points mode, weights 1/q), and used for `evals_per_batch` Adam steps.
    anneal = (factor, n_steps): App. A's annealing in the temperature, the
    training target taken at factor x T at the first step and lowered
    geometrically to T over the first n_steps steps (a smoother integrand
    first).  Returns the list of losses.
    """
    plan = api.EvalPlan([G], [params], [0], batch, maps=[vegas] if on_vegas else None)
    tw = torch.empty(batch, dtype=torch.float32, device="cuda")
    beta0 = plan._p[0].beta
    losses = []
    k = 0
    while k < steps:
        if k < vegas_steps:
            # VEGAS draws: uniform in the map's input space, or mapped points
            x, w = api.map_samples(None if on_vegas else vegas, seed, 1000 + k, 1, batch, G.dim)
        else:
            x, w = _flow_draw(flow, seed, 1000 + k, 2, batch, defensive)
        if anneal is not None:
            factor, n_anneal = anneal
            plan._p[0].beta = beta0 / factor ** max(0.0, 1.0 - k / n_anneal)
        # target |f| / q_s per sample, formed by the integrand kernel
        plan.run_target(seed, 1000 + k, tw, points=x, point_w=w)
        m = min(evals_per_batch, steps - k)
        step_losses = flow.train(x, tw, m, lr).tolist()
        losses.extend(step_losses)
        k += m
        if not all(math.isfinite(v) for v in step_losses):
            raise FloatingPointError("flow training diverged at step %d" % k)
        if log and k % 100 < m:
            log(k, losses[-1])
    return losses


def mcmc(G, params, vegas, flow, n_chains, n_steps, alpha, seed, it, n_therm=0, chains=None, n_sel=1, plan=None):
    """One call of NF-MCMC (flow given: proposals from the flow on the VEGAS
    grid's coordinates) or VEGAS-MCMC (flow None: proposals from the VEGAS map),
    Sec. V: n_chains x n_steps proposals drawn from q and evaluated by the
    integrand kernel (their weights f/q per root and Re/Im), then n_steps
    Metropolis-Hastings steps of every chain (target alpha q + (1 - alpha)|f|,
    |f| from the first n_sel weight rows).  Pass the returned chains (and plan)
    back in to continue the same chains.  Returns (chains, plan, estimates
    [n_out + 1][2] on the device: (I, variance) per weight row, then the
    accepted fraction)."""
    n = n_chains * n_steps
    if plan is None:
        plan = api.EvalPlan([G], [params], [0], n, maps=[vegas] if vegas is not None else None, per_sample=True)
    if flow is None:
        plan.run(seed, it)
    else:
        x, w = flow.draw(seed, it, 3, n)
        plan.run(seed, it, points=x, point_w=w)
    weights = plan.per_sample[0].reshape(-1, n)[:2 * len(G.roots)]
    if chains is None:
        chains = api.Chains(weights.shape[0], n_chains, n_sel=n_sel, alpha=alpha)
    out = chains.run(weights, n_steps, seed, it, n_therm)
    return chains, plan, out


def mcmc_compare(G, params, vegas, flow, n_chains, n_steps, alphas, seed, n_therm=None):
    """Efficiency of VEGAS-MCMC and NF-MCMC (Sec. V) for Re of root 0.

    Per sampler: alpha is chosen on one draw of proposals (the smallest
    variance of the estimate over `alphas`, the same weights reused, the first
    n_therm steps of each chain discarded; default a quarter), then an
    independent draw with that alpha thermalises a fresh set of chains (one
    whole call discarded) and a continuation of the same chains is timed end
    to end (proposals, integrand, chains, estimate).  The chains must be long
    enough to equilibrate: with heavy-tailed weights short chains stick in
    high-weight states and give biased estimates with too small error bars.
    Returns per sampler: alpha, estimate and error, accepted fraction,
    seconds of the timed call, and the figure of merit 1 / (variance x
    seconds) of the timed call (thermalisation not charged)."""
    n = n_chains * n_steps
    if n_therm is None:
        n_therm = n_steps // 4
    res = {}
    for name, fl in (("vegas_mcmc", None), ("nf_mcmc", flow)):
        _, plan, _ = mcmc(G, params, vegas, fl, n_chains, n_steps, alphas[0], seed, 1000, n_therm)
        w = plan.per_sample[0].reshape(-1, n)[:2]
        scan = []
        for a in alphas:
            out = api.Chains(2, n_chains, n_sel=1, alpha=a).run(w, n_steps, seed, 1000, n_therm).cpu().numpy()
            scan.append((float(out[0, 1]), a))
        a = min(scan)[1]
        ch, plan, _ = mcmc(G, params, vegas, fl, n_chains, n_steps, a, seed + 1, 2000, n_steps)
        torch.cuda.synchronize()
        s, e = _events()
        s.record()
        _, _, out = mcmc(G, params, vegas, fl, n_chains, n_steps, a, seed + 1, 2001, 0, chains=ch, plan=plan)
        e.record()
        torch.cuda.synchronize()
        t = s.elapsed_time(e) / 1e3
        out = out.cpu().numpy()
        res[name] = {"alpha": a, "alpha_scan": {str(b): v for v, b in sorted(scan, key=lambda x: x[1])},
                     "mean": float(out[0, 0]), "err": float(math.sqrt(out[0, 1])), "accepted": float(out[2, 0]),
                     "seconds": t, "proposals": n, "chains": n_chains, "steps": n_steps,
                     "merit": 1.0 / (float(out[0, 1]) * t)}
    return res


def measure_sampler(G, params, n, seed, it, vegas=None, flow=None, reps=3, defensive=0.0):
    """Per-sample variance of every root and seconds per sample for one sampler.

    VEGAS: the map is applied inside the integrand kernel.  Flow: the sampling
    kernel writes points and 1/q, the integrand kernel reads them (and applies
    `vegas` on top when it is given).
    Returns (stats [R][2][2] of the last rep, seconds per sample).
    """
    if flow is None:
        plan = api.EvalPlan([G], [params], [0], n, maps=[vegas] if vegas is not None else None)
        plan.run(seed, it)
        torch.cuda.synchronize()
        s, e = _events()
        s.record()
        for r in range(reps):
            st = plan.run(seed, it + 1 + r)
        e.record()
        torch.cuda.synchronize()
        return st[0].cpu().numpy(), s.elapsed_time(e) / 1e3 / reps / n
    plan = api.EvalPlan([G], [params], [0], n, maps=[vegas] if vegas is not None else None)
    x, w = _flow_draw(flow, seed, it, 3, n, defensive)
    plan.run(seed, it, points=x, point_w=w)
    torch.cuda.synchronize()
    s, e = _events()
    s.record()
    for r in range(reps):
        x, w = _flow_draw(flow, seed, it + 1 + r, 3, n, defensive)
        st = plan.run(seed, it + 1 + r, points=x, point_w=w)
    e.record()
    torch.cuda.synchronize()
    return st[0].cpu().numpy(), s.elapsed_time(e) / 1e3 / reps / n


def kish_ess(G, params, n, seed, it, root=0, vegas=None, flow=None, defensive=0.0):
    """Kish effective sample size fraction (sum |wf|)^2 / (n sum (wf)^2) of the
    real part of `root` over one batch of n weighted samples of a sampler
    (VEGAS map, or the flow's points with 1/q on top of `vegas`), from the
    integrand's per-sample values."""
    plan = api.EvalPlan([G], [params], [0], n, maps=[vegas] if vegas is not None else None, per_sample=True)
    if flow is None:
        plan.run(seed, it)
    else:
        x, w = _flow_draw(flow, seed, it, 3, n, defensive)
        plan.run(seed, it, points=x, point_w=w)
    return kish_fraction(plan.per_sample[0, root, 0])


def kish_fraction(f):
    """(sum |f|)^2 / (n sum f^2) of the n weighted values f (a tensor), in
    FP64; 0 when every value is 0."""
    f = f.double()
    a1, a2 = float(f.abs().sum().item()), float((f * f).sum().item())
    return a1 * a1 / (f.numel() * a2) if a2 > 0 else 0.0


def bootstrap_ratio(num, den, stat, resamples=4000, seed=0, level=0.95):
    """Percentile bootstrap interval of stat(num) / stat(den), the batches of
    the two samplers resampled independently with replacement."""
    rng = np.random.default_rng(seed)
    num, den = np.asarray(num, dtype=np.float64), np.asarray(den, dtype=np.float64)
    a = stat(num[rng.integers(0, num.size, (resamples, num.size))], axis=1)
    b = stat(den[rng.integers(0, den.size, (resamples, den.size))], axis=1)
    q = (1.0 - level) / 2.0
    r = a / b
    return [float(np.quantile(r, q)), float(np.quantile(r, 1.0 - q))]


def compare(G, params, vegas, flow, n, seed, root=0, batches=4, on_vegas=True, defensive=0.0):
    """Variance-adjusted efficiency of flow vs VEGAS for the real part of `root`.

    Each sampler draws `batches` independent batches of n samples.  The
    per-sample variance is estimated from all samples together (the mean of
    the batch estimates) and, as a robust companion, by the median of the
    batch estimates: the order-5 integrand is heavy-tailed, so a single rare
    sample can dominate a batch's estimate.  The batch means give the combined
    estimate and its error.  Both time-adjusted ratios come with a 95 %
    percentile-bootstrap interval over the batches (ci95).
    """
    res = {}
    flow_kw = dict(flow=flow, vegas=vegas if on_vegas else None, defensive=defensive)
    for name, kw, it0 in (("vegas", dict(vegas=vegas), 50000), ("flow", flow_kw, 60000)):
        means, vars_, secs = [], [], []
        for b in range(batches):
            st, sec = measure_sampler(G, params, n, seed, it0 + 10 * b, reps=1, **kw)
            means.append(st[root, 0, 0])
            vars_.append(st[root, 0, 1] * n)
            secs.append(sec)
        v = float(np.mean(vars_))
        t = float(np.mean(secs))
        m = float(np.mean(means))
        err = float(math.sqrt(v / (n * batches)))
        res[name] = {"mean": m, "err": err, "var_per_sample": v, "var_median": float(np.median(vars_)),
                     "var_batches": [float(x) for x in vars_], "batch_means": [float(x) for x in means],
                     "samples_per_s": 1.0 / t}
    res["vegas"]["eff_samples_per_s"] = res["vegas"]["samples_per_s"]
    res["flow"]["eff_samples_per_s"] = res["flow"]["samples_per_s"] * res["vegas"]["var_per_sample"] / \
        res["flow"]["var_per_sample"]
    res["flow_over_vegas"] = res["flow"]["eff_samples_per_s"] / res["vegas"]["eff_samples_per_s"]
    res["flow_over_vegas_median"] = (res["flow"]["samples_per_s"] / res["vegas"]["samples_per_s"] *
                                     res["vegas"]["var_median"] / res["flow"]["var_median"])
    res["means_agree_sigma"] = abs(res["flow"]["mean"] - res["vegas"]["mean"]) / math.sqrt(
        res["flow"]["err"] ** 2 + res["vegas"]["err"] ** 2)
    speed = res["flow"]["samples_per_s"] / res["vegas"]["samples_per_s"]
    vv, fv = res["vegas"]["var_batches"], res["flow"]["var_batches"]
    res["ci95"] = {"flow_over_vegas": [speed * x for x in bootstrap_ratio(vv, fv, np.mean)],
                   "flow_over_vegas_median": [speed * x for x in bootstrap_ratio(vv, fv, np.median)],
                   "variance_gain_median": bootstrap_ratio(vv, fv, np.median),
                   "variance_gain_pooled": bootstrap_ratio(vv, fv, np.mean),
                   "batches": batches, "samples_per_batch": n, "resamples": 4000}
    res["defensive_share"] = defensive
    # Kish effective sample size fraction of one batch of each sampler
    res["kish_ess_fraction"] = {"vegas": kish_ess(G, params, n, seed, 70000, root, vegas=vegas),
                                "flow": kish_ess(G, params, n, seed, 70000, root, **flow_kw),
                                "samples": n}
    return res


class BatchedIteration:
    """One persistent launch over many instances of uneven graph order, captured
    as a CUDA graph per iteration: integrand (with VEGAS histograms), fixed-order
    reduction, batched VEGAS update and the device-side iteration counter."""

    def __init__(self, graphs, params, graph_of_inst, n_per_inst, seed, n_bins=1024, alpha=0.5):
        self.graphs = list(graphs)
        self.params = list(params)
        self.gi = list(graph_of_inst)
        self.n = int(n_per_inst)
        self.seed = seed
        self.alpha = alpha
        self.maps = [api.Vegas(self.graphs[g].dim, n_bins) for g in self.gi]
        self.plan = api.EvalPlan(self.graphs, self.params, self.gi, self.n, maps=self.maps)
        self._maps_arr = (api.ctypes.c_void_p * len(self.maps))(*[m.handle for m in self.maps])
        self.d_iter = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.graph = None
        self.stream = None

    def _enqueue(self, stream):
        lib = api.L.lib()
        sp = api._stream_ptr(stream)
        api.L.check(lib.fd_integrand_eval_iter_dev(self.plan._g, len(self.graphs), self.plan._p, self.plan._gi,
                                                   self.plan.n_inst, self.plan._m, self.seed, 0,
                                                   api._ptr(self.d_iter), self.n, api._ptr(self.plan.partials), sp))
        api.L.check(lib.fd_accumulate(api._ptr(self.plan.partials), self.plan.n_inst, self.plan.r_max, self.n,
                                      api._ptr(self.plan.stats), sp))
        api.L.check(lib.fd_vegas_update_batch(self._maps_arr, len(self.maps), self.alpha, sp))
        api.L.check(lib.fd_counter_add(api._ptr(self.d_iter), 1, sp))

    def step_direct(self, stream=None):
        self._enqueue(stream or torch.cuda.current_stream())
        return self.plan.stats

    def capture(self):
        self.stream = torch.cuda.Stream()
        api.device_status()                       # make sure per-device state exists before capture
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._enqueue(self.stream)
        return self.graph

    def replay(self):
        self.graph.replay()
        return self.plan.stats
