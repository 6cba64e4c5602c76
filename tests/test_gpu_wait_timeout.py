"""Failure detection without a fault: the tape interpreter's bounded mbarrier
waits.  A test hook makes every tape wait give up at its first poll; the
kernel then records the timeout, waits (at the full limit) for the bulk
copies it has in flight and returns early.  The host sees FD_ETIMEOUT from
fd_device_status after a launch that ended in bounded time, the record is
cleared, and the context stays usable: the next evaluation at the default
limit matches the oracle."""
import time

import numpy as np
import pytest

import parity
from oracle import conventions, integrand as oig, philox as ophilox

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_2403_18840_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def test_tape_wait_gives_up_and_reports(api):
    order, n, seed = 3, 70000, 91           # several tiles and both tape buffers in use
    G = api.Graph(order, with_dk=True)
    plan = api.EvalPlan([G], [api.ueg_params(order, 1.0, 1.0 / 25.0, 1.0, 1.0)], [0], n, per_sample=True)
    api.device_status()                      # no earlier record
    api.set_wait_polls(0)
    try:
        t0 = time.perf_counter()
        plan.run(seed, 0)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    finally:
        api.set_wait_polls(-1)
    with pytest.raises(api.L.FdError) as e:
        api.device_status()
    assert e.value.status == api.L.FD_ETIMEOUT
    print("timed-out launch returned in %.3f s" % dt)
    assert dt < 10.0
    api.device_status()                      # the record was cleared
    # the same context evaluates correctly at the default limit
    plan.run(seed, 0)
    torch.cuda.synchronize()
    api.device_status()
    f = plan.per_sample[0].cpu().numpy().astype(np.float64)[:len(G.roots), :, :2048]
    P = conventions.ueg_params(1.0, 1.0 / 25.0, 1.0, 1.0)
    x = ophilox.uniforms(seed, 0, 0, np.arange(2048), 4 * order - 1)
    ref, mag = oig.eval_roots(x, G.roots, P, with_l1=True)
    parity.check(parity.rel_error(f, ref, mag), "after the timeout")


def test_wait_polls_argument_checked(api):
    with pytest.raises(api.L.FdError):
        api.L.check(api.L.lib().fd_debug_set_wait_polls(1 << 33))
    api.set_wait_polls(-1)
