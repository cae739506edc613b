"""y-slab decomposition on CPU processes (gloo): the host-side partition and
halo exchange of ``slabs.py``, with the oracle as each rank's step.

Each rank holds its rows of a 64 x 32 FP64 field plus a ghost row below and
above.  Before every step the ranks exchange the [3][nx] halos in the
library's format (face 0 sends populations 0, 1, 2 of the bottom row, face 1
populations 6, 7, 8 of the top row; the ghost rows receive them as in
kbc_halo_recv) through ``slabs.exchange`` on CPU tensors; each rank then
steps its padded field with the oracle and keeps the interior rows, which
depend only on themselves and on the received ghost populations.  After 50
steps the gathered field must equal the oracle run on the whole periodic
field bit for bit: the pull of Eq. Egeneral crosses the slab faces exactly
as it crosses the periodic boundary.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _initial(nx, ny, seed):
    import oracle as O

    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.02 * rng.standard_normal((ny, nx))
    ux = 0.06 * (2 * rng.random((ny, nx)) - 1)
    uy = 0.06 * (2 * rng.random((ny, nx)) - 1)
    g = O.init_feq(rho, ux, uy)
    return g * (1.0 + 0.02 * rng.standard_normal(g.shape))


def _advance_slab(rank, world, nx, ny, steps, variant, beta, seed, group=None):
    """This rank's interior rows after `steps` exchanged steps."""
    import oracle as O
    from paper_1507_02509_gb300 import slabs

    g = _initial(nx, ny, seed)
    y0, rows = slabs.partition(ny, world)[rank]
    W = O.weights().reshape(9, 1)
    loc = np.empty((9, rows + 2, nx))
    loc[:, 1:rows + 1] = g[:, y0:y0 + rows]
    send_lo = torch.empty((3, nx), dtype=torch.float64)
    send_hi, recv_lo, recv_hi = (torch.empty_like(send_lo) for _ in range(3))
    lo_send, hi_send = list(slabs.SEND_POPS[0]), list(slabs.SEND_POPS[1])
    lo_recv, hi_recv = list(slabs.RECV_POPS[0]), list(slabs.RECV_POPS[1])
    for _ in range(steps):
        send_lo.copy_(torch.from_numpy(loc[lo_send, 1]))
        send_hi.copy_(torch.from_numpy(loc[hi_send, rows]))
        slabs.exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world, group)
        loc[:, 0] = W            # ghost populations nobody pulls: f = W
        loc[:, rows + 1] = W
        loc[lo_recv, 0] = recv_lo.numpy()
        loc[hi_recv, rows + 1] = recv_hi.numpy()
        out = O.step(loc, variant, beta, 1)
        loc[:, 1:rows + 1] = out[:, 1:rows + 1]
    return y0, rows, loc[:, 1:rows + 1].copy()


def _worker(rank, world, port, q, args):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + _advance_slab(rank, world, *args))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("variant", [0, 2])
def test_slab_ranks_reproduce_the_periodic_field_bit_for_bit(world, variant):
    import oracle as O

    nx, ny, steps, beta, seed = 64, 32, 50, 0.93, 5
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    args = (nx, ny, steps, variant, beta, seed)
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, args)) for r in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.empty((9, ny, nx))
    for _, y0, rows, f in parts:
        got[:, y0:y0 + rows] = f
    ref = O.step(_initial(nx, ny, seed), variant, beta, steps)
    assert np.array_equal(got, ref)


def test_single_slab_is_its_own_neighbour():
    """world = 1: the exchange swaps the slab's own faces (no process group)."""
    import oracle as O

    nx, ny, steps, beta, seed = 16, 12, 20, 0.9, 3
    _, _, f = _advance_slab(0, 1, nx, ny, steps, O.B, beta, seed)
    assert np.array_equal(f, O.step(_initial(nx, ny, seed), O.B, beta, steps))


def test_partition_and_neighbours():
    from paper_1507_02509_gb300 import slabs

    assert slabs.partition(32, 3) == [(0, 11), (11, 11), (22, 10)]
    assert slabs.partition(8, 8) == [(k, 1) for k in range(8)]
    assert slabs.partition(5, 1) == [(0, 5)]
    with pytest.raises(ValueError):
        slabs.partition(3, 4)
    assert slabs.neighbours(0, 4) == (3, 1)
    assert slabs.neighbours(3, 4) == (2, 0)
    assert slabs.neighbours(0, 1) == (0, 0)
    # a face sends the populations moving across it; the opposite ghost row of
    # the neighbour receives exactly those
    va = [i % 3 - 1 for i in range(9)]
    vb = [i // 3 - 1 for i in range(9)]
    assert all(vb[i] == -1 for i in slabs.SEND_POPS[0])
    assert all(vb[i] == +1 for i in slabs.SEND_POPS[1])
    assert slabs.RECV_POPS[0] == slabs.SEND_POPS[1]
    assert slabs.RECV_POPS[1] == slabs.SEND_POPS[0]
    assert sorted(va[i] for i in slabs.SEND_POPS[0]) == [-1, 0, 1]


def _node_parts(g, variant, beta, rows):
    """One partial diagnostics set (the layout of kbc_diagnostics_partial)
    per row range, computed with numpy from the oracle's per-node values of
    the whole field: sums, node count, mean and sum of squared deviations of
    |u|^2/2 and of w^2/2 (w by periodic central differences), gamma sum, min
    and max of the next step's collision."""
    import oracle as O

    rho, ux, uy = O.macro(g)
    ke = 0.5 * (ux * ux + uy * uy)
    w = 0.5 * (np.roll(uy, -1, 1) - np.roll(uy, 1, 1)) - 0.5 * (np.roll(ux, -1, 0) - np.roll(ux, 1, 0))
    zz = 0.5 * w * w
    _, gam = O.step(g, variant, beta, 1, want_gamma=True)
    parts = []
    for y0, r in rows:
        sl = slice(y0, y0 + r)
        k, z, gm = ke[sl].ravel(), zz[sl].ravel(), gam[sl].ravel()
        parts.append([rho[sl].sum(), (rho * ux)[sl].sum(), (rho * uy)[sl].sum(), k.size,
                      k.mean(), ((k - k.mean()) ** 2).sum(), z.mean(), ((z - z.mean()) ** 2).sum(),
                      gm.sum(), gm.min(), gm.max()])
    return np.array(parts)


def _diag_worker(rank, world, port, q, args):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    from paper_1507_02509_gb300 import slabs

    nx, ny, variant, beta, seed = args
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rows = slabs.partition(ny, world)
        mine = _node_parts(_initial(nx, ny, seed), variant, beta, rows)[rank]
        parts = slabs.gather_parts(torch.tensor(mine), rank, world)
        d = slabs.merge_diagnostics(np.stack([p.numpy() for p in parts]))
        q.put((rank, [d[k] for k in sorted(d)], sorted(d)))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_slab_ranks_merge_global_diagnostics():
    """Each gloo rank holds the partial diagnostics of its slab; after one
    all-gather every rank merges them (kbc_diagnostics_merge, a host routine
    of the library) into the oracle's diagnostics of the whole field."""
    import oracle as O

    nx, ny, variant, beta, seed, world = 40, 33, O.B, 0.94, 9, 3
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_diag_worker, args=(r, world, port, q, (nx, ny, variant, beta, seed)))
             for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = O.diagnostics(_initial(nx, ny, seed), variant, beta)
    names = got[0][2]
    want = dict(zip(O.DIAG_NAMES, ref))
    for _, vals, _ in got:
        assert vals == got[0][1]  # every rank merges the same sets in the same order
        for name, v in zip(names, vals):
            assert v == pytest.approx(want[name], rel=1e-12, abs=1e-15), name


def test_merge_combines_partial_sets_in_order():
    """kbc_diagnostics_merge against the direct mean / std / min / max of the
    concatenated samples, for uneven splits including a single node."""
    from paper_1507_02509_gb300 import capi

    capi.load()
    rng = np.random.default_rng(4)
    k = 1e-3 + 1e-4 * rng.standard_normal(1000)
    z = 2e-6 * rng.random(1000)
    gm = 1.0 + 0.3 * rng.standard_normal(1000)
    cuts = [0, 1, 250, 251, 700, 1000]
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        kk, zz, gg = k[a:b], z[a:b], gm[a:b]
        parts.append([a + 0.5, 2 * a, -a, b - a, kk.mean(), ((kk - kk.mean()) ** 2).sum(),
                      zz.mean(), ((zz - zz.mean()) ** 2).sum(), gg.sum(), gg.min(), gg.max()])
    parts = np.ascontiguousarray(parts, dtype=np.float64)
    out = np.zeros(capi.KBC_DIAG_N)
    capi.kbc_diagnostics_merge(len(parts), parts, out)
    want = [parts[:, 0].sum(), parts[:, 1].sum(), parts[:, 2].sum(), k.mean(), z.mean(),
            gm.mean(), gm.min(), gm.max(), k.std(), z.std()]
    assert np.allclose(out, want, rtol=1e-13, atol=0)
    with pytest.raises(capi.KBCError):
        capi.kbc_diagnostics_merge(0, parts, out)
