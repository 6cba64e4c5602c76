"""Independent replicas across ranks (one process per GPU).

Monte Carlo samples are independent, so the path shards without exchanging
anything while it samples: rank k draws its own Philox stream (the seed offset
by the rank), adapts its own VEGAS grid and evaluates its own samples.  Two
small host-side exchanges remain, both outside the sampling: the timing of a
benchmark (the maximum over ranks of the timed region), and, when one answer
is wanted, the combination of the ranks' estimates into the estimate over all
their samples.
"""
import torch

SEED_STRIDE = 1000003


def rank_seed(seed, rank):
    """Philox seed of rank `rank`: distinct streams for distinct ranks."""
    return int(seed) + SEED_STRIDE * int(rank)


def max_over_ranks(dist, value, device="cpu"):
    """Largest `value` over the ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_estimates(dist, mean, var, n, device="cpu"):
    """Pool the ranks' estimates of the same quantities.

    mean, var: arrays (any shape) of a rank's mean and variance of the mean
    over its n samples, as fd_accumulate returns them (var = sum (f - mean)^2
    / ((n - 1) n)).  Returns the mean and the variance of the mean over all
    ranks' samples together (n times the number of ranks).  Pairwise
    combination (Chan, Golub and LeVeque): the pooled mean first, then the
    ranks' sums of squared deviations plus n (mean_r - mean)^2, so no large
    sums of squares are subtracted from each other.
    """
    m = torch.as_tensor(mean, dtype=torch.float64, device=device)
    v = torch.as_tensor(var, dtype=torch.float64, device=device)
    s = m * n
    world = 1 if dist is None else dist.get_world_size()
    if dist is not None:
        dist.all_reduce(s)
    N = n * world
    mean_all = s / N
    d = m - mean_all
    q = v * n * (n - 1) + n * d * d                    # this rank's sum of (f - mean_all)^2
    if dist is not None:
        dist.all_reduce(q)
    var_all = torch.clamp(q / (N - 1), min=0.0) / N
    return mean_all.cpu().numpy(), var_all.cpu().numpy()
