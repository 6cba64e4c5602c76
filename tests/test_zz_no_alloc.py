"""The allocation-free evaluation entry point against the regular one.

fd_integrand_eval_stats_noalloc exists for callers that cannot allocate device
memory (everything allocated up front, graph replays that may not allocate,
no allocator at hand); it keeps the tile partial sums in a fixed array inside
the library.  Its results must match fd_integrand_eval + fd_accumulate on the
same inputs, on consecutive calls that reuse the shared array.  This file is
collected last so a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _regular(A, L, plan, seed, it):
    lib = L.lib()
    L.check(lib.fd_integrand_eval(plan._g, len(plan.graphs), plan._p, plan._gi, plan.n_inst, plan._m, None, None,
                                  seed, it, plan.n_per_inst, A._ptr(plan.partials), None, A._stream_ptr(None)))
    out = torch.zeros_like(plan.stats)
    L.check(lib.fd_accumulate(A._ptr(plan.partials), plan.n_inst, plan.r_max, plan.n_per_inst, A._ptr(out),
                              A._stream_ptr(None)))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _noalloc(A, L, plan, seed, it):
    out = torch.full_like(plan.stats, -7.0)
    st = L.lib().fd_integrand_eval_stats_noalloc(plan._g, len(plan.graphs), plan._p, plan._gi, plan.n_inst,
                                                 plan._m, None, None, seed, it, plan.n_per_inst, A._ptr(out),
                                                 None, A._stream_ptr(None))
    L.check(st)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    from paper_2403_18840_gb300 import _lib as L
    from paper_2403_18840_gb300 import api as A

    assert torch.cuda.is_available()
    g3 = A.Graph(3, with_dk=True)
    g2 = A.Graph(2)
    # call 1: one instance, several tiles and a ragged tail
    p1 = A.EvalPlan([g3], [A.ueg_params(3, 1.0, 1.0 / 25.0, 1.0, 1.0)], [0], 3 * 16384 + 101)
    # call 2: smaller, two graphs and three instances (reads a different part of the array)
    p2 = A.EvalPlan([g2, g3], [A.ueg_params(2, 2.0, 1.0 / 25.0, 1.0, 0.5),
                                A.ueg_params(3, 1.0, 1.0 / 25.0, 1.0, 2.0),
                                A.ueg_params(2, 1.0, 1.0 / 25.0, 1.0, 0.0)], [0, 1, 0], 20000)
    for plan, seed in ((p1, 31), (p2, 32)):
        ref = _regular(A, L, plan, seed, 4)
        got = _noalloc(A, L, plan, seed, 4)
        assert np.all(np.isfinite(got))
        # same kernels and summation order; the test tolerance for means is 1e-6 relative
        assert np.allclose(got, ref, rtol=1e-6, atol=1e-300), np.max(np.abs(got - ref))


def test_noalloc_rejects_requests_beyond_its_array():
    from paper_2403_18840_gb300 import _lib as L
    from paper_2403_18840_gb300 import api as A

    g = A.Graph(2)
    n = 1 << 30           # needs far more partial sums than the fixed array holds
    plan_g = (ctypes.c_void_p * 1)(g.handle)
    params = (L.fd_params * 1)(A.ueg_params(2, 1.0, 1.0 / 25.0, 1.0, 1.0))
    gi = (ctypes.c_int32 * 1)(0)
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    st = L.lib().fd_integrand_eval_stats_noalloc(plan_g, 1, params, gi, 1, None, None, None, 1, 0, n,
                                                 A._ptr(out), None, A._stream_ptr(None))
    assert st == L.FD_EINVAL
    assert b"fixed array" in L.lib().fd_last_error()
    torch.cuda.synchronize()
    assert torch.all(out == 0)
