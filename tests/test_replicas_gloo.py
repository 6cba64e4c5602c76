"""The multi-rank (replica) host logic on two gloo ranks on the CPU: distinct
Philox seeds per rank, maximum-over-ranks timing, and the combination of the
ranks' estimates equal to the estimate over all their samples together."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2
N = 5000


def _samples(rank):
    from paper_2403_18840_gb300 import replicas
    rng = np.random.default_rng(replicas.rank_seed(7, rank))
    # the last row: a large offset with a small spread (sum f^2 - N mean^2
    # would cancel ~16 digits)
    return (rng.standard_normal((4, N)) * np.array([[1.0], [0.1], [5.0], [1e-3]])
            + np.array([[0.5], [-2.0], [0.0], [1e8]]) + rank * np.array([[0.0], [0.0], [0.0], [1e-3]]))


def _stats(f):
    """Mean and variance of the mean, two-pass."""
    n = f.shape[-1]
    mean = f.mean(axis=-1)
    var = np.sum((f - mean[..., None]) ** 2, axis=-1) / (n - 1) / n
    return mean, var


def _worker(rank, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        from paper_2403_18840_gb300 import replicas
        mean, var = _stats(_samples(rank))
        m_all, v_all = replicas.combine_estimates(tdist, mean, var, N)
        t_max = replicas.max_over_ranks(tdist, 1.0 + rank)
        out[rank] = (m_all, v_all, t_max, replicas.rank_seed(7, rank))
    finally:
        tdist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_combine_like_one_pool():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(_free_port(), out), nprocs=WORLD, join=True, start_method="spawn")
        res = dict(out)
    pooled = np.concatenate([_samples(r) for r in range(WORLD)], axis=-1)
    ref_mean, ref_var = _stats(pooled)
    for r in range(WORLD):
        m_all, v_all, t_max, seed = res[r]
        assert np.allclose(m_all, ref_mean, rtol=1e-12, atol=1e-15)
        assert np.allclose(v_all[:3], ref_var[:3], rtol=1e-9, atol=1e-18)
        # offset 1e8, spread 1e-3: the pooled mean carries FP64's 1e-16 relative
        # rounding, 1e-8 absolute, ~1e-5 of the spread, and the variance that
        # much relatively; subtracting sums of squares would lose every digit
        assert abs(v_all[3] / ref_var[3] - 1.0) < 1e-4
        assert t_max == float(WORLD)                 # slowest rank's time
    assert res[0][3] != res[1][3]                    # independent streams
