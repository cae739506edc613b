"""kbc_diagnostics_noalloc: diagnostics without any device allocation.

Some callers cannot allocate device memory: their device memory is owned by
another allocator (a framework's caching pool or a fixed arena), or they run
a timed loop that must not hit the implicit synchronisation of
cudaMalloc/cudaFree.  This entry point serves them: it keeps its scratch in a
static device array and takes the caller's own FP64 population field.

The test calls it through the C ABI twice in a row on the same field and
checks both results against kbc_diagnostics of a handle holding the same
populations (same per-node arithmetic, different reduction split, so the
sums agree to rounding: 1e-12 relative).  It lives in its own file, collected
last, and passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1507_02509_gb300 import KBCError, Lattice, capi  # noqa: E402
from tests.gpu_helpers import random_field  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["B", "lbgk", "C"])
def test_noalloc_diagnostics_match_handle_diagnostics(variant):
    assert torch.cuda.is_available()
    capi.load()
    nx, ny, beta = 384, 37, 0.96
    g = random_field(nx, ny, 123)
    vid = {"B": capi.KBC_B, "lbgk": capi.KBC_LBGK, "C": capi.KBC_C}[variant]

    lat = Lattice(nx, ny, variant=variant, beta=beta, dtype="f64")
    lat.set_populations(g)
    ref = np.array(list(lat.diagnostics().values()))
    lat.close()

    f_dev = torch.as_tensor(g, device="cuda").contiguous()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for _ in range(2):  # two calls in a row share the static scratch
        out = np.full(capi.KBC_DIAG_N, np.nan)
        capi.kbc_diagnostics_noalloc(nx, ny, vid, beta, f_dev, out, stream)
        outs.append(out)
    for out in outs:
        assert np.allclose(out, ref, rtol=1e-12, atol=1e-15), (out, ref)
    assert np.array_equal(outs[0], outs[1])

    # device output works too
    out_dev = torch.full((capi.KBC_DIAG_N,), float("nan"), dtype=torch.float64, device="cuda")
    capi.kbc_diagnostics_noalloc(nx, ny, vid, beta, f_dev, out_dev, stream)
    assert np.allclose(out_dev.cpu().numpy(), ref, rtol=1e-12, atol=1e-15)


def test_noalloc_rejects_oversize_and_host_fields():
    capi.load()
    g = np.ones((9, 4, 4))
    out = np.zeros(capi.KBC_DIAG_N)
    with pytest.raises(KBCError) as e:  # host field: staging would allocate
        capi.kbc_diagnostics_noalloc(4, 4, capi.KBC_B, 0.9, g, out)
    assert e.value.status == capi.KBC_ERR_ARG and "device memory" in str(e.value)
    f_dev = torch.ones((9, 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(KBCError) as e:  # beyond 2^28 nodes
        capi.kbc_diagnostics_noalloc(32768, 16385, capi.KBC_B, 0.9, f_dev, out)
    assert e.value.status == capi.KBC_ERR_ARG and "2^28" in str(e.value)
