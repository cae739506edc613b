"""Failure detection without faulting the GPU: every failure here is made on
the host (an allocator that refuses, a wait given too little time, a NaN
planted in the input elsewhere) and must come back as a status code with the
context still usable."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1507_02509_gb300 import KBCError, Lattice, capi, flows, use_torch_allocator  # noqa: E402
from tests.gpu_helpers import random_field  # noqa: E402

pytestmark = pytest.mark.gpu


def test_allocation_failure_is_reported_and_cleaned_up():
    capi.load()
    calls = {"n": 0}

    def alloc(nbytes, stream, user):
        calls["n"] += 1
        return None  # refuse every request

    def release(p, stream, user):
        raise AssertionError("nothing was allocated")

    hooks = (capi.ALLOC_FN(alloc), capi.FREE_FN(release))
    capi.kbc_set_allocator(hooks[0], hooks[1], None)
    try:
        with pytest.raises(KBCError) as e:
            capi.kbc_create(256, 8, capi.KBC_B, 0.9, capi.KBC_F32_DEV)
        assert e.value.status == capi.KBC_ERR_NOMEM
        assert calls["n"] >= 1
    finally:
        capi.kbc_set_allocator(capi.ALLOC_FN(0), capi.FREE_FN(0), None)
        import paper_1507_02509_gb300 as pkg

        pkg._torch_hooks = None
    # the context is still usable
    lat = Lattice(256, 8, variant="B", beta=0.9, dtype="f32")
    lat.set_populations(random_field(256, 8, 1))
    lat.step(3)
    lat.sync()
    lat.close()


def test_bounded_host_wait_times_out_and_recovers():
    """kbc_sync with a 1 ms limit while ~0.3 s of steps are queued returns
    KBC_ERR_TIMEOUT; a later sync without a short limit succeeds."""
    n = 8192
    rho, ux, uy = flows.taylor_green(n, u0=0.03, modes=4)
    lat = Lattice(n, n, variant="B", beta=0.99, dtype="f32")
    lat.init(rho, ux, uy)
    lat.sync()
    lat.step(400)
    with pytest.raises(KBCError) as e:
        capi.kbc_sync(lat.h, 0.001)
    assert e.value.status == capi.KBC_ERR_TIMEOUT
    lat.sync()
    lat.close()


def test_library_memory_comes_from_the_torch_caching_allocator():
    import gc

    use_torch_allocator()
    gc.collect()  # tensors of earlier tests left in reference cycles are freed now, not mid-test
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    lat = Lattice(1024, 512, variant="B", beta=0.95, dtype="f32")
    during = torch.cuda.memory_allocated()
    assert during - before >= 2 * 9 * 1024 * 512 * 4  # the A-B population pair
    lat.close()
    assert torch.cuda.memory_allocated() == before


def test_bound_stream_is_honoured():
    """Work is issued on the stream given to kbc_set_stream: an event recorded
    on that stream after kbc_step completes only after the steps."""
    s = torch.cuda.Stream()
    n = 4096
    rho, ux, uy = flows.taylor_green(n, u0=0.03, modes=2)
    with torch.cuda.stream(s):
        lat = Lattice(n, n, variant="B", beta=0.99, dtype="f32")
        lat.init(rho, ux, uy)
        lat.step(50)
        ev = torch.cuda.Event()
        ev.record(s)
    ev.synchronize()
    # everything the handle queued has finished: a zero-timeout query agrees
    assert capi.load().kbc_sync(lat.h, ctypes.c_double(1e-3)) == capi.KBC_OK
    lat.close()
