"""The allocation-free entry point bonsai_sfc_order_noalloc against the
regular path.

Some callers cannot allocate device memory: their GPU memory is owned by
another allocator or a fixed budget, or they cannot accept the device-wide
synchronisation that cudaMalloc/cudaFree imply, or they are plugins handed
buffers but no allocation rights.  For them the library offers the bounding
cube, Peano-Hilbert keys and key sort with scratch in a fixed static device
array.  Here its keys, order and cube must equal, bit for bit, what
tree_build computes for the same particles, on consecutive calls that reuse
the shared scratch.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def _call_c_abi(lib, pos, mass, keys, perm):
    n = mass.numel()
    cube = (ctypes.c_double * 4)()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.bonsai_sfc_order_noalloc(ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(mass.data_ptr()),
                                      ctypes.c_int64(n), ctypes.c_void_p(keys.data_ptr()),
                                      ctypes.c_void_p(perm.data_ptr()), cube, stream)
    return rc, list(cube)


def test_noalloc_order_equals_tree_build_on_consecutive_calls():
    from paper_1412_0659_gb300 import TreeGravity, capi
    lib = capi.load()
    dev = torch.device("cuda", 0)
    # three calls in a row: a ragged size, the same input again, then a
    # smaller input that must not see the first call's leftovers
    inputs = [workloads.plummer(100003, seed=31), None, workloads.milky_way(40961, seed=32)]
    inputs[1] = inputs[0]
    for m in inputs:
        pos = torch.from_numpy(m.pos).to(dev)
        mass = torch.from_numpy(m.mass).to(dev)
        keys = torch.full((m.n,), -1, dtype=torch.int64, device=dev)
        perm = torch.full((m.n,), -1, dtype=torch.int32, device=dev)
        rc, cube = _call_c_abi(lib, pos, mass, keys, perm)
        assert rc == 0, capi.strerror(rc)
        with TreeGravity(G=1.0, theta=0.4, eps=0.01) as g:
            g.build(pos, mass)
            ref = g.debug()
        assert torch.equal(keys, ref["keys"])
        assert torch.equal(perm, ref["perm"])
        assert cube == [*ref["lo"], ref["L"]]


def test_noalloc_at_the_size_limit_allocates_nothing():
    """n = BONSAI_NOALLOC_MAX_N, the only size that fills the fixed
    histogram and scan regions: keys, order and cube equal tree_build's bit
    for bit.  After a first call (which has looked up the scratch address),
    a second call changes neither the device's free memory nor what torch's
    caching allocator holds."""
    from paper_1412_0659_gb300 import TreeGravity, capi
    lib = capi.load()
    dev = torch.device("cuda", 0)
    m = workloads.milky_way(capi.BONSAI_NOALLOC_MAX_N, seed=34)
    pos = torch.from_numpy(m.pos).to(dev)
    mass = torch.from_numpy(m.mass).to(dev)
    keys = torch.full((m.n,), -1, dtype=torch.int64, device=dev)
    perm = torch.full((m.n,), -1, dtype=torch.int32, device=dev)
    rc, cube = _call_c_abi(lib, pos, mass, keys, perm)
    assert rc == 0, capi.strerror(rc)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    rc2, cube2 = _call_c_abi(lib, pos, mass, keys, perm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rc2 == 0 and cube2 == cube
    assert free1 == free0 and torch.cuda.memory_reserved() == reserved0
    with TreeGravity(G=m.G, theta=0.4, eps=0.01) as g:
        g.build(pos, mass)
        ref = g.debug()
    assert torch.equal(keys, ref["keys"])
    assert torch.equal(perm, ref["perm"])
    assert cube == [*ref["lo"], ref["L"]]


def test_noalloc_rejects_bad_sizes_and_inputs():
    from paper_1412_0659_gb300 import capi
    lib = capi.load()
    dev = torch.device("cuda", 0)
    small = torch.zeros(4, dtype=torch.float64, device=dev)
    # n beyond the fixed scratch: rejected before any device work
    rc = lib.bonsai_sfc_order_noalloc(ctypes.c_void_p(small.data_ptr()), ctypes.c_void_p(small.data_ptr()),
                                      ctypes.c_int64(capi.BONSAI_NOALLOC_MAX_N + 1),
                                      ctypes.c_void_p(small.data_ptr()), ctypes.c_void_p(small.data_ptr()),
                                      None, None)
    assert rc == capi.BONSAI_EINVAL
    with pytest.raises(ValueError, match="fixed scratch limit"):
        big = torch.zeros(capi.BONSAI_NOALLOC_MAX_N + 1, dtype=torch.float64, device=dev)
        capi.bonsai_sfc_order_noalloc(small, big, small, small)
    # a non-finite position is reported, and the next call is clean again
    m = workloads.plummer(5000, seed=33)
    pos = torch.from_numpy(m.pos).to(dev)
    mass = torch.from_numpy(m.mass).to(dev)
    keys = torch.empty(m.n, dtype=torch.int64, device=dev)
    perm = torch.empty(m.n, dtype=torch.int32, device=dev)
    bad = pos.clone()
    bad[2, 123] = float("inf")
    rc, _ = _call_c_abi(lib, bad, mass, keys, perm)
    assert rc == capi.BONSAI_EINVAL
    rc, cube = _call_c_abi(lib, pos, mass, keys, perm)
    assert rc == 0 and np.all(np.isfinite(cube))
    assert torch.equal(torch.sort(perm.long()).values.cpu(), torch.arange(m.n))
