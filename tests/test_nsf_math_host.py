"""The spline flow's per-sample device code (csrc/fd_nsf_math.cuh: the spline,
its inverse, its closed-form partials, one coupling layer's conditioner,
inverse and reverse-mode backward) compiled for the host and run on the CPU
against the FP64 oracle (App. A): the density at given points and the
gradient of the forward-KL loss.  The GPU kernels call the same functions;
their own parity (staging, warp sums, atomics) is in test_gpu_spline_flow."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads
from oracle import spline_flow as osf

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2403_18840_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("nsfhost") / "nsf_math_host")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "native", "nsf_math_host.cu"),
                    "-o", out], check=True, capture_output=True)
    return out


def _run(exe, tmp_path, flow, x32, w32):
    dim, n = x32.shape[1], x32.shape[0]
    src, dst = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(src, "wb") as f:
        np.array([dim, len(flow.layers), n], np.int32).tofile(f)
        flow.flat().astype(np.float32).tofile(f)
        np.ascontiguousarray(x32.T).tofile(f)
        w32.tofile(f)
    subprocess.run([exe, src, dst], check=True)
    raw = open(dst, "rb").read()
    npar = flow.flat().size
    loss = np.frombuffer(raw, np.float64, 1)[0]
    grad = np.frombuffer(raw, np.float64, npar, 8)
    z = np.frombuffer(raw, np.float32, dim * n, 8 + 8 * npar).reshape(dim, n)
    lq = np.frombuffer(raw, np.float32, n, 8 + 8 * npar + 4 * dim * n)
    return loss, grad, z.astype(np.float64), lq.astype(np.float64)


def _fp32_flow(dim, n_layers, seed, **kw):
    flow = osf.SplineFlow(dim, n_layers, seed=seed, **kw)
    flow.set_flat(flow.flat().astype(np.float32).astype(np.float64))
    return flow


@pytest.mark.parametrize("dim,n_layers,n,seed", [(5, 4, 300, 41), (6, 3, 200, 42), (19, 2, 64, 43), (2, 1, 50, 44)])
def test_host_build_matches_oracle(exe, tmp_path, dim, n_layers, n, seed):
    flow = _fp32_flow(dim, n_layers, seed, scale=0.8)
    z0 = workloads.uniform_points(seed, dim, n)
    x_ref, _ = flow.forward(z0.T)
    x32 = x_ref.astype(np.float32)
    w32 = np.exp(-4.0 * ((x32.astype(np.float64) - 0.4) ** 2).sum(axis=1)).astype(np.float32)
    loss, grad, z, lq = _run(exe, tmp_path, flow, x32, w32)
    x64, w64 = x32.astype(np.float64), w32.astype(np.float64)
    lq_ref, z_ref = flow.log_density(x64)
    # the inverse pass in FP32 (the density test's inverse bounds)
    assert np.quantile(np.abs(z - z_ref.T), 0.99) < 5e-5 and np.abs(z - z_ref.T).max() < 5e-4
    assert np.quantile(np.abs(lq - lq_ref), 0.99) < 1e-3 and np.abs(lq - lq_ref).max() < 1e-2
    gr = flow.kl_grad(x64, w64, analytic=True)
    assert abs(loss - flow.kl_loss(x64, w64)) < 1e-5 * (1.0 + abs(loss))
    scale = np.abs(gr).max()
    assert np.abs(grad - gr).max() < 1e-4 * scale
    assert np.linalg.norm(grad - gr) < 5e-5 * np.linalg.norm(gr)


def test_host_build_identity_flow(exe, tmp_path):
    # zero parameters: every spline is the identity, log q = 0, and the
    # gradient of the loss is the oracle's at the identity
    flow = _fp32_flow(4, 2, 1, zero=True)
    x32 = workloads.uniform_points(3, 4, 100).T.astype(np.float32)
    w32 = np.linspace(0.1, 1.0, 100).astype(np.float32)
    loss, grad, z, lq = _run(exe, tmp_path, flow, x32, w32)
    assert np.abs(z - x32.T).max() < 1e-6 and np.abs(lq).max() < 1e-5 and abs(loss) < 1e-5
    gr = flow.kl_grad(x32.astype(np.float64), w32.astype(np.float64), analytic=True)
    assert np.abs(grad - gr).max() < 1e-4 * max(np.abs(gr).max(), 1e-6)
