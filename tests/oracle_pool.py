"""The oracle's per-sample roots evaluated in worker processes (test
infrastructure): the sample range is cut into chunks, each chunk evaluated
by oracle.integrand.eval_roots on its own Philox points.  Workers start with
the spawn method, so a pool may be opened after the parent has used CUDA."""
import multiprocessing as mp
import os

import numpy as np


def _chunk(args):
    order, roots, prm, seed, iteration, lo, hi = args
    from oracle import conventions, integrand, philox
    P = conventions.ueg_params(*prm)
    x = philox.uniforms(seed, iteration, 0, np.arange(lo, hi), 4 * order - 1)
    return integrand.eval_roots(x, roots, P, with_l1=True)


def eval_roots(order, roots, seed, n, prm=(1.0, 1.0 / 25.0, 1.0, 1.0), iteration=0, workers=None):
    """(values [R, n] complex, L1 magnitudes [R, n]) at the Philox points
    0..n-1 of (seed, iteration, stream 0); prm = (r_s, T/T_F, lambda/k_F, k/k_F)."""
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    pieces = max(1, min(n // 256, 4 * workers))
    edges = np.linspace(0, n, pieces + 1).astype(int)
    jobs = [(order, list(roots), tuple(prm), seed, iteration, int(a), int(b))
            for a, b in zip(edges[:-1], edges[1:]) if b > a]
    if workers == 1 or len(jobs) == 1:
        parts = [_chunk(j) for j in jobs]
    else:
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_chunk, jobs)
    return np.concatenate([p[0] for p in parts], axis=1), np.concatenate([p[1] for p in parts], axis=1)
