"""The failure contract of the library, exercised without faulting the GPU:
host waits on the device are bounded (a host function that sleeps on the
context's stream stands in for a device that does not answer), and a
particle count whose buffers cannot fit in device memory is refused with
ENOMEM before anything is allocated or launched.  In both cases the
context stays usable."""
import time

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def _model():
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    m = workloads.plummer(4096, seed=21)
    g = TreeGravity(G=1.0, theta=0.4, eps=0.01)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    return m, g


def test_a_wait_past_the_limit_returns_etimeout_and_the_context_recovers():
    from paper_1412_0659_gb300 import capi
    m, g = _model()
    acc0, pot0 = (x.clone() for x in g.forces())
    torch.cuda.synchronize()
    try:
        capi.bonsai_set_wait_timeout(0.3)
        capi.tree_debug_hold_stream(g.ctx, 2.0)
        t0 = time.perf_counter()
        with pytest.raises(capi.BonsaiError) as ex:
            g.forces()
        waited = time.perf_counter() - t0
        assert ex.value.code == capi.BONSAI_ETIMEOUT
        assert 0.25 < waited < 1.5, waited
    finally:
        capi.bonsai_set_wait_timeout(600.0)
    time.sleep(2.0)  # the held stream drains; the queued walk completes
    acc1, pot1 = g.forces()
    torch.cuda.synchronize()
    assert torch.equal(acc1, acc0) and torch.equal(pot1, pot0)
    g.close()


def test_bad_wait_limits_are_rejected():
    from paper_1412_0659_gb300 import capi
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(capi.BonsaiError) as ex:
            capi.bonsai_set_wait_timeout(bad)
        assert ex.value.code == capi.BONSAI_EINVAL


def test_n_over_the_memory_budget_is_enomem_and_the_context_recovers():
    """n = 2^31 - 1 needs ~430 GB of particle buffers, more than the GPU
    holds: tree_build refuses it before allocating or launching anything
    (the small pos/mass buffers passed are never read), then builds a real
    model in the same context."""
    from paper_1412_0659_gb300 import capi
    m, g = _model()
    free0, _ = torch.cuda.mem_get_info()
    pos = torch.zeros(3, 8, dtype=torch.float64, device="cuda")
    mass = torch.ones(8, dtype=torch.float64, device="cuda")
    rc = capi.load().tree_build(g.ctx, capi._ptr(pos), capi._ptr(mass), (1 << 31) - 1)
    assert rc == capi.BONSAI_ENOMEM
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)  # nothing was allocated on the way
    with pytest.raises(capi.BonsaiError) as ex:
        g.forces()
    assert ex.value.code == capi.BONSAI_ESTATE  # the old tree is gone, no half-built one
    g.build(torch.from_numpy(m.pos).cuda(), torch.from_numpy(m.mass).cuda())
    acc, pot = g.forces()
    torch.cuda.synchronize()
    assert torch.isfinite(acc).all() and torch.isfinite(pot).all()
    g.close()
