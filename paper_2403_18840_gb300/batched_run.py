"""Batched persistent evaluation of many uneven graph instances: orders 1-5 x
r_s in {1, 2, 4} x 16 external momenta in [0, 2 k_F] (240 instances over 5
graphs, dimension up to 19), 2^22 samples per instance per iteration, a
VEGAS grid per instance (Sec. V.B: the graphs are compiled once and
evaluated in batches).

Every graph runs its specialised kernel (one variant for all orders: 4
samples per thread with their inputs in shared memory, units of cost
<= 12000); one iteration -- every instance's integrand with its histogram,
the fixed-order reduction, the batched VEGAS update and the device-side
iteration counter -- is captured as a CUDA graph (`driver.BatchedIteration`)
and replayed.

    python -m paper_2403_18840_gb300.batched_run [--iters 5] [--warmup 2] [--samples 22]

(--samples is log2 of the samples per instance.)  Prints one JSON line: the
iterations' seconds (CUDA events) and samples/s over all instances.
"""
import argparse
import json
import time

import torch

from . import api, driver, fdgraph

ORDERS = (5, 4, 3, 2, 1)
RS = (1.0, 2.0, 4.0)
KEXT = tuple(2.0 * j / 15.0 for j in range(16))
T_OVER_TF, LAM_OVER_KF = 1.0 / 25.0, 1.0
VARIANT = dict(threads=256, min_blocks=1, spt=4, unit_cap=12000, sv_smem=True)


def build(n_per_inst, seed):
    graphs, gi, params = [], [], []
    for g, order in enumerate(ORDERS):
        G = api.Graph(order, roots=fdgraph.graph_roots(order), budget=1 << 13)
        G.jit(**VARIANT)
        graphs.append(G)
        for rs in RS:
            for k in KEXT:
                gi.append(g)
                params.append(api.ueg_params(order, rs, T_OVER_TF, LAM_OVER_KF, k))
    return driver.BatchedIteration(graphs, params, gi, n_per_inst, seed=seed), len(gi)


def run(iters, warmup, n_per_inst, seed=3):
    t0 = time.perf_counter()
    it, n_inst = build(n_per_inst, seed)
    it.capture()
    for _ in range(warmup):
        it.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        it.replay()
    e1.record()
    torch.cuda.synchronize()
    api.device_status()
    ms = e0.elapsed_time(e1) / iters
    return {"workload": "batched240_orders1to5", "instances": n_inst, "samples_per_instance": n_per_inst,
            "iterations": iters, "ms_per_iteration": ms,
            "samples_per_s": n_inst * n_per_inst / ms * 1e3, "kernel_variant": VARIANT,
            "setup_s": time.perf_counter() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--samples", type=int, default=22, help="log2 of the samples per instance")
    a = ap.parse_args()
    print(json.dumps(run(a.iters, a.warmup, 1 << a.samples)), flush=True)


if __name__ == "__main__":
    main()
