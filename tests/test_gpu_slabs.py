"""y-slab handles on one GPU: halo format, decomposed runs against the
periodic handle (bit for bit) and the oracle, and the calls a slab refuses.

A grid split into slabs that exchange halos before every step must give the
periodic handle's bits: the kernels, the node arithmetic and every pulled
value are the same; only the source of the rows across a slab face changes
(the ghost row instead of the periodic wrap).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1507_02509_gb300 import KBCError, Lattice, capi, flows, slabs  # noqa: E402
from tests.gpu_helpers import (max_rel_velocity_error, oracle_sensitivity,  # noqa: E402
                               random_field, representable, weights)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    capi.load()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_halo_format(dtype):
    """kbc_halo_send writes [3][nx] stored deviations of the face's row and
    populations; kbc_halo_recv puts them into the ghost row that the next
    step pulls (checked by sending a slab's own halos back to itself and
    comparing one step with the periodic handle)."""
    nx, ny = 256, 5
    g = representable(random_field(nx, ny, 3), dtype)
    lat = Lattice(nx, ny, variant="B", beta=0.95, dtype=dtype, slab=True)
    lat.set_populations(g)
    nb = lat.halo_bytes
    assert nb == 3 * nx * (8 if dtype == "f64" else 4)
    W = weights()
    npd = np.float64 if dtype == "f64" else np.float32
    for face, row in ((0, 0), (1, ny - 1)):
        buf = np.zeros(nb, dtype=np.uint8)
        capi.kbc_halo_send(lat.h, face, 0, buf)
        pops = list(slabs.SEND_POPS[face])
        got = buf.view(npd).reshape(3, nx).astype(np.float64) + W[pops][:, None]
        assert np.array_equal(got, g[pops, row]), face
    # a single slab fed its own halos is the periodic grid
    lo = torch.empty(nb, dtype=torch.uint8, device="cuda")
    hi = torch.empty_like(lo)
    capi.kbc_halo_send(lat.h, 0, 0, lo)
    capi.kbc_halo_send(lat.h, 1, 0, hi)
    capi.kbc_halo_recv(lat.h, 0, 0, hi)
    capi.kbc_halo_recv(lat.h, 1, 0, lo)
    lat.step(1)
    got = lat.populations().cpu().numpy()
    lat.close()
    ref = Lattice(nx, ny, variant="B", beta=0.95, dtype=dtype)
    ref.set_populations(g)
    ref.step(1)
    want = ref.populations().cpu().numpy()
    ref.close()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype,kernel,nx", [("f64", "rows", 128), ("f32", "rows", 256),
                                             ("f32", "bulk", 512), ("f16", "bulk", 512),
                                             ("f16", "rows", 256), ("f32", "nodes", 37),
                                             ("f64", "nodes", 19)])
@pytest.mark.parametrize("variant", ["lbgk", "B", "C"])
def test_slab_group_matches_periodic_handle_bit_for_bit(variant, dtype, kernel, nx):
    """Three slabs (uneven rows) advancing 24 steps with halo exchanges give
    exactly the bits of one periodic handle (FP32 guard pass at its default,
    which re-evaluates nodes pulled across the faces too)."""
    ny, steps, beta = 23, 24, 0.96
    rho, ux, uy = flows.turbulence(64, k0=4, urms=0.05, seed=13, kcut=16)
    rho = np.resize(rho, (ny, nx))
    ux, uy = np.resize(ux, (ny, nx)), np.resize(uy, (ny, nx))
    grp = slabs.SlabGroup(nx, ny, 3, variant=variant, beta=beta, dtype=dtype)
    for s in grp.slabs:
        s.set_kernel(kernel)
    grp.init(rho, ux, uy).step(steps)
    got = grp.populations().cpu().numpy()
    grp.sync()
    grp.close()
    lat = Lattice(nx, ny, variant=variant, beta=beta, dtype=dtype)
    lat.set_kernel(kernel)
    lat.init(rho, ux, uy).step(steps)
    want = lat.populations().cpu().numpy()
    lat.sync()
    lat.close()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("parts", [1, 2, 4])
def test_slab_group_matches_oracle(parts):
    """The 64^2 vortex (u0 = 0.04, nu = 0.01), KBC B in FP64 split into
    y-slabs: 200 steps against the oracle on the whole periodic field, to the
    same bound as the undecomposed run (max(1e-12, 3 x the oracle's 1-ulp
    sensitivity))."""
    n, nu, steps = 64, 0.01, 200
    beta = 1.0 / (6 * nu + 1)
    rho, ux, uy = flows.taylor_green(n, u0=0.04)
    grp = slabs.SlabGroup(n, n, parts, variant="B", beta=beta, dtype="f64")
    grp.init(rho, ux, uy).step(steps)
    _, vx, vy = (t.cpu().numpy() for t in grp.moments())
    grp.sync()
    grp.close()
    g0 = O.init_feq(rho, ux, uy)
    _, rx, ry = O.macro(O.step(g0, O.B, beta, steps, nthreads=8))
    err = max_rel_velocity_error((vx, vy), (rx, ry))
    floor = oracle_sensitivity(g0, O.B, beta, steps, nthreads=8, ref_uv=(rx, ry))
    assert err < max(1e-12, 3 * floor), (err, floor)
    k = 2 * math.pi / n
    amp = np.sum(vx * ux) / np.sum(ux * ux)
    assert amp == pytest.approx(math.exp(-2 * nu * k * k * steps), rel=2e-2)


def test_distributed_slab_single_rank_is_periodic():
    """DistributedSlab with one rank (no process group) exchanges with itself
    and reproduces the periodic handle bit for bit."""
    nx, ny, beta = 256, 16, 0.97
    g = representable(random_field(nx, ny, 21), "f32")
    r, ux, uy = O.macro(g)
    d = slabs.DistributedSlab(nx, ny, 0, 1, variant="B", beta=beta, dtype="f32")
    d.init(r, ux, uy).step(10)
    got = d.lat.populations().cpu().numpy()
    d.close()
    lat = Lattice(nx, ny, variant="B", beta=beta, dtype="f32")
    lat.init(r, ux, uy).step(10)
    want = lat.populations().cpu().numpy()
    lat.close()
    assert np.array_equal(got, want)


def test_slab_refusals():
    lat = Lattice(128, 8, variant="B", beta=0.9, dtype="f32", slab=True)
    lat.init(np.ones((8, 128)), np.zeros((8, 128)), np.zeros((8, 128)))
    buf = torch.empty(lat.halo_bytes, dtype=torch.uint8, device="cuda")
    for call in (lambda: lat.step(2), lambda: lat.diagnostics(), lambda: lat.diagnostics_ext(),
                 lambda: capi.kbc_halo_send(lat.h, 2, 0, buf),
                 lambda: lat.init(np.ones((8, 128)), np.zeros((8, 128)), np.zeros((8, 128)),
                                  grad=True)):
        with pytest.raises(KBCError) as e:
            call()
        assert e.value.status == capi.KBC_ERR_ARG
    lat.step(1)
    lat.sync()
    lat.close()
    plain = Lattice(128, 8, variant="B", beta=0.9, dtype="f32")
    with pytest.raises(KBCError) as e:
        capi.kbc_halo_send(plain.h, 0, 0, buf)
    assert e.value.status == capi.KBC_ERR_ARG
    plain.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["lbgk", "B"])
def test_slab_group_global_diagnostics(variant, dtype):
    """Global diagnostics of a grid split into 3 slabs (full halos, one
    partial set per slab, merged) equal the periodic handle's after 10 steps
    (1e-12; the reduction splits differ) and the oracle's on the same stored
    populations; one partial set of a plain handle merged alone equals
    kbc_diagnostics."""
    nx, ny, beta = 256, 37, 0.95
    g = representable(random_field(nx, ny, 29), dtype)
    grp = slabs.SlabGroup(nx, ny, 3, variant=variant, beta=beta, dtype=dtype)
    grp.set_populations(g).step(10)
    got = grp.diagnostics()
    f = grp.populations().cpu().numpy()
    grp.close()
    lat = Lattice(nx, ny, variant=variant, beta=beta, dtype=dtype)
    lat.set_populations(g)
    lat.step(10)
    want = lat.diagnostics()
    alone = slabs.merge_diagnostics([lat.diagnostics_partial()])
    lat.close()
    ref = dict(zip(O.DIAG_NAMES, O.diagnostics(f, O.VARIANTS[variant], beta)))
    for name in O.DIAG_NAMES:
        assert got[name] == pytest.approx(want[name], rel=1e-12, abs=1e-15), name
        assert got[name] == pytest.approx(ref[name], rel=1e-11, abs=1e-15), name
        assert alone[name] == pytest.approx(want[name], rel=1e-15, abs=0), name


def test_slab_partial_diagnostics_need_current_full_halos():
    """kbc_diagnostics_partial on a slab refuses (KBC_ERR_STATE) until both
    ghost rows hold full halos of the current state; a step or a 3-population
    halo makes them stale again."""
    nx, ny = 128, 6
    lat = Lattice(nx, ny, variant="B", beta=0.9, dtype="f32", slab=True)
    lat.set_populations(representable(random_field(nx, ny, 5), "f32"))
    full = torch.empty(lat.full_halo_bytes, dtype=torch.uint8, device="cuda")
    part = torch.empty(lat.halo_bytes, dtype=torch.uint8, device="cuda")

    def refused():
        with pytest.raises(KBCError) as e:
            lat.diagnostics_partial()
        return e.value.status == capi.KBC_ERR_STATE

    assert refused()
    capi.kbc_halo_send(lat.h, 0, 1, full)
    capi.kbc_halo_recv(lat.h, 1, 1, full)
    assert refused()  # one face only
    capi.kbc_halo_send(lat.h, 1, 1, full)
    capi.kbc_halo_recv(lat.h, 0, 1, full)
    assert lat.diagnostics_partial()[3] == nx * ny
    capi.kbc_halo_send(lat.h, 1, 0, part)
    capi.kbc_halo_recv(lat.h, 0, 0, part)
    assert refused()
    for face in (0, 1):
        capi.kbc_halo_send(lat.h, 1 - face, 1, full)
        capi.kbc_halo_recv(lat.h, face, 1, full)
    lat.step(1)
    assert refused()
    lat.close()
