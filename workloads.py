"""Seeded synthetic workloads shared by the GPU path, its tests, the bench and the oracle.

This module holds descriptions only (dimensionless physics parameters, sample
counts, seeds) and seeded random inputs; none of the method's arithmetic lives
here.  Each consumer derives physical parameters (k_F, beta, Lambda, ...) with
its own code.

The workloads mirror the paper's uniform-electron-gas calculations
(Sec. VI.A: r_s, T/T_F, screening lambda, external momentum), at the sizes of
the benchmark configurations (the order-1 exchange case to the order-6
effective mass).  No dataset is involved: the
paper's inputs are synthetic by nature.
"""
import numpy as np

# Order-1 exchange (Fock) self-energy: r_s = 1, lambda = 0.5 k_F, T = 0.04 T_F,
# cutoff 6 k_F, 8 external momenta k_j = 3 k_F j / 7, 2^20 samples, seed 0.
FOCK_ORDER1 = dict(
    name="fock_order1_rs1", order=1, rs=1.0, T_over_TF=0.04, lam_over_kF=0.5,
    kext_over_kF=[3.0 * j / 7.0 for j in range(8)], kc_over_kF=6.0,
    n_samples=1 << 20, seed=0, sampler="identity")

# Orders 1-4 counterterm-renormalised Sigma(k, i w0): r_s = 1, lambda = k_F,
# beta = 25 / E_F, k in {0, k_F, 2 k_F}, VEGAS 1024 bins/dim, 2^24 samples/iter.
ORDERS_1_4 = dict(
    name="orders1to4_rs1", orders=[1, 2, 3, 4], rs=1.0, T_over_TF=1.0 / 25.0,
    lam_over_kF=1.0, kext_over_kF=[0.0, 1.0, 2.0], kc_over_kF=6.0, n_bins=1024,
    n_samples=1 << 24, n_iters=10, n_warm=3, seed=1, sampler="vegas")

# Batched persistent launch: orders 1-5 x r_s in {1,2,4} x 16 k in [0, 2 k_F]
# (240 instances over 5 graphs), 2^22 samples per instance per iteration.
BATCHED_240 = dict(
    name="batched240_orders1to5", orders=[1, 2, 3, 4, 5], rs=[1.0, 2.0, 4.0],
    T_over_TF=1.0 / 25.0, lam_over_kF=1.0,
    kext_over_kF=[2.0 * j / 15.0 for j in range(16)], kc_over_kF=6.0, n_bins=1024,
    n_per_instance=1 << 22, seed=3, sampler="vegas")

# Learned proposal at order 5, r_s = 1 (D = 19): 8 affine coupling layers,
# MLP hidden 128, trained 2000 steps on 2^20-sample batches, compared with
# VEGAS at 2^24 samples; as the proposal of Metropolis-Hastings chains
# (NF-MCMC, and VEGAS-MCMC with the grid): 2^12 chains x 2^12 steps, the
# mixing parameter from a scan.
FLOW_ORDER5 = dict(
    name="flow_order5_rs1", order=5, rs=1.0, T_over_TF=1.0 / 25.0, lam_over_kF=1.0,
    kext_over_kF=1.0, kc_over_kF=6.0, n_layers=8, hidden=128, train_steps=2000,
    batch=1 << 20, n_compare=1 << 24, n_bins=1024, seed=2,
    mcmc_chains=1 << 12, mcmc_steps=1 << 12, mcmc_alphas=(0.1, 0.3, 0.5, 0.7, 0.9))

# Order-6 effective mass: r_s in {1, 2}, D = 23, 2^26 samples x 50 iterations.
ORDER6_MEFF = dict(
    name="order6_meff", order=6, rs=[1.0, 2.0], T_over_TF=1.0 / 25.0, lam_over_kF=1.0,
    kext_over_kF=1.0, kc_over_kF=6.0, n_samples=1 << 26, n_iters=50, seed=4)

# The integrand-throughput workload of the benchmark: one order-5 graph at
# r_s = 1, k = k_F, VEGAS sampler, 2^24 samples per step.
BENCH_ORDER5 = dict(
    name="order5_rs1_kF_vegas", order=5, rs=1.0, T_over_TF=1.0 / 25.0,
    lam_over_kF=1.0, kext_over_kF=1.0, kc_over_kF=6.0, n_bins=1024,
    n_samples=1 << 24, seed=5)


def small_params(seed, n, scale=0.05):
    """Seeded FP32 parameter vector (normal, small): an untrained network's weights."""
    return (np.random.default_rng(seed).standard_normal(n) * scale).astype(np.float32)


def uniform_points(seed, dim, n, lo=1e-6, hi=1.0 - 1e-6):
    """Seeded points in (lo, hi)^dim as FP32-representable values, shape [dim, n]."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=(dim, n)).astype(np.float32)
    return x.astype(np.float64)


def normal_blob(seed, n, scale):
    """Seeded N(0, scale^2) values, FP32-representable, shape [n]."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) * scale).astype(np.float32).astype(np.float64)


def positive_weights(seed, n):
    """Seeded positive weights (log-normal), FP32-representable, shape [n]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.standard_normal(n)).astype(np.float32).astype(np.float64)


def histogram_like(seed, dim, n_bins):
    """Seeded non-negative bin contents with a peak and empty bins, shape [dim, n_bins]."""
    rng = np.random.default_rng(seed)
    y = (np.arange(n_bins) + 0.5) / n_bins
    out = np.empty((dim, n_bins))
    for k in range(dim):
        c = rng.uniform(0.1, 0.9)
        w = rng.uniform(0.01, 0.2)
        out[k] = np.exp(-0.5 * ((y - c) / w) ** 2) * rng.uniform(0.5, 2.0, n_bins)
        out[k, rng.integers(0, n_bins, n_bins // 20)] = 0.0
    return out
