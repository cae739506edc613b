"""y-slab decomposition of a doubly periodic D2Q9 grid.

The pull of Eq. Egeneral reaches one row up and one row down, so a grid of
NY rows splits into horizontal slabs that exchange one row per face before
every step: each slab sends the three populations of its bottom row that
move down (b = -1, i = 0, 1, 2) to the slab below, and the three of its top
row that move up (b = +1, i = 6, 7, 8) to the slab above, both taken
periodically in y.  x stays periodic inside every slab.

The device side is the library's y-slab handle (kbc_create_slab,
kbc_halo_send, kbc_halo_recv): halos are [3][nx] arrays in the storage
encoding, or [9][nx] (full rows) before global diagnostics, which each slab
computes as a partial set (kbc_diagnostics_partial) and the library
combines in a fixed order (kbc_diagnostics_merge) -- across ranks after one
all-gather of the sets.  This module holds the host-side bookkeeping around
it: the row partition, the neighbour ranks, the exchange over
torch.distributed (NCCL between GPUs, gloo between CPU processes; one
process per slab), and a group of slabs advanced in one process (several
handles on one device).  No lattice Boltzmann arithmetic happens here.
"""
from __future__ import annotations

# populations a face sends, and those its ghost row receives (index order
# i = 3(b+1) + (a+1) of v_i = (a, b)); face 0 is the lower face, 1 the upper
SEND_POPS = {0: (0, 1, 2), 1: (6, 7, 8)}
RECV_POPS = {0: (6, 7, 8), 1: (0, 1, 2)}


def partition(ny: int, parts: int) -> list[tuple[int, int]]:
    """(y0, rows) of each slab: rows as even as possible, the first
    ny % parts slabs one row longer; every slab has at least one row."""
    if parts < 1 or ny < parts:
        raise ValueError(f"cannot split {ny} rows into {parts} slabs")
    base, extra = divmod(ny, parts)
    out, y0 = [], 0
    for k in range(parts):
        rows = base + (1 if k < extra else 0)
        out.append((y0, rows))
        y0 += rows
    return out


def neighbours(rank: int, world: int) -> tuple[int, int]:
    """(lower, upper) slab of slab `rank` on the periodic y axis."""
    return (rank - 1) % world, (rank + 1) % world


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None):
    """One halo exchange between the slabs of a process group.

    send_lo / send_hi: this slab's outgoing halos of faces 0 and 1;
    recv_lo / recv_hi: filled with the lower neighbour's face-1 halo and the
    upper neighbour's face-0 halo.  Tensors of equal size (CUDA tensors for
    NCCL, CPU tensors for gloo).  Messages going down carry tag 0 and those
    going up tag 1; NCCL, which ignores tags, pairs them by their order,
    which is the same on every rank.  A single slab is its own neighbour.
    """
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    import torch.distributed as dist

    lower, upper = neighbours(rank, world)
    ops = [dist.P2POp(dist.isend, send_lo, lower, group, 0),
           dist.P2POp(dist.irecv, recv_hi, upper, group, 0),
           dist.P2POp(dist.isend, send_hi, upper, group, 1),
           dist.P2POp(dist.irecv, recv_lo, lower, group, 1)]
    for w in dist.batch_isend_irecv(ops):
        w.wait()


def _halo_buffers(lat, count: int, full: bool = False):
    import torch

    nb = lat.full_halo_bytes if full else lat.halo_bytes
    return [torch.empty(nb, dtype=torch.uint8, device=lat.device) for _ in range(count)]


def merge_diagnostics(parts):
    """The KBC_DIAG_N global diagnostics from partial sets [n][KBC_DIAG_PART_N]
    (in slab order), combined by the library (kbc_diagnostics_merge)."""
    import numpy as np

    from . import DIAG_NAMES, capi

    parts = np.ascontiguousarray(np.asarray(parts, dtype=np.float64))
    out = np.zeros(capi.KBC_DIAG_N)
    capi.kbc_diagnostics_merge(parts.shape[0], parts, out)
    return dict(zip(DIAG_NAMES, out.tolist()))


class SlabGroup:
    """All slabs of one nx x ny periodic grid in this process (on the current
    device): `parts` y-slab handles that exchange halos through device
    buffers before every step, all on one stream.  The field it advances is
    the same as one periodic handle's, bit for bit (same kernels, same
    inputs)."""

    def __init__(self, nx: int, ny: int, parts: int, **lattice_kw):
        from . import Lattice

        self.nx, self.ny = int(nx), int(ny)
        self.rows = partition(self.ny, parts)
        self.slabs = [Lattice(self.nx, r, slab=True, **lattice_kw) for _, r in self.rows]
        self._send = [_halo_buffers(s, 2) for s in self.slabs]

    def close(self):
        for s in self.slabs:
            s.close()

    def init(self, rho, ux, uy):
        """Equilibrium initialisation from full-grid [ny][nx] fields."""
        for (y0, r), s in zip(self.rows, self.slabs):
            s.init(rho[y0:y0 + r], ux[y0:y0 + r], uy[y0:y0 + r])
        return self

    def set_populations(self, f):
        for (y0, r), s in zip(self.rows, self.slabs):
            s.set_populations(f[:, y0:y0 + r])
        return self

    def exchange(self):
        """Fill every ghost row from the neighbouring slabs' boundary rows."""
        from . import capi

        world = len(self.slabs)
        for k, s in enumerate(self.slabs):
            s._bind_stream()
            capi.kbc_halo_send(s.h, 0, 0, self._send[k][0])
            capi.kbc_halo_send(s.h, 1, 0, self._send[k][1])
        for k, s in enumerate(self.slabs):
            lower, upper = neighbours(k, world)
            capi.kbc_halo_recv(s.h, 0, 0, self._send[lower][1])
            capi.kbc_halo_recv(s.h, 1, 0, self._send[upper][0])

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.exchange()
            for s in self.slabs:
                s.step(1)
        return self

    def diagnostics(self) -> dict:
        """Global diagnostics of the grid (those of kbc_diagnostics): full
        halos into every ghost row, one partial set per slab, combined."""
        from . import capi

        world = len(self.slabs)
        full = [_halo_buffers(s, 2, full=True) for s in self.slabs]
        for k, s in enumerate(self.slabs):
            s._bind_stream()
            capi.kbc_halo_send(s.h, 0, 1, full[k][0])
            capi.kbc_halo_send(s.h, 1, 1, full[k][1])
        for k, s in enumerate(self.slabs):
            lower, upper = neighbours(k, world)
            capi.kbc_halo_recv(s.h, 0, 1, full[lower][1])
            capi.kbc_halo_recv(s.h, 1, 1, full[upper][0])
        return merge_diagnostics([s.diagnostics_partial() for s in self.slabs])

    def populations(self):
        """f[9][ny][nx] of the whole grid (float64 CUDA tensor)."""
        import torch

        return torch.cat([s.populations() for s in self.slabs], dim=1)

    def moments(self):
        import torch

        parts = [s.moments() for s in self.slabs]
        return tuple(torch.cat([p[k] for p in parts], dim=0) for k in range(3))

    def sync(self):
        for s in self.slabs:
            s.sync()


class DistributedSlab:
    """This rank's slab of an nx x ny periodic grid split over the ranks of a
    torch.distributed group (one process, and one device, per slab).  Each
    step sends both faces, exchanges halos with the neighbouring ranks and
    advances one step."""

    def __init__(self, nx: int, ny: int, rank: int, world: int, group=None, **lattice_kw):
        from . import Lattice

        self.nx, self.ny = int(nx), int(ny)
        self.rank, self.world, self.group = int(rank), int(world), group
        self.y0, self.rows = partition(self.ny, self.world)[self.rank]
        self.lat = Lattice(self.nx, self.rows, slab=True, **lattice_kw)
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = _halo_buffers(self.lat, 4)

    def close(self):
        self.lat.close()

    def init(self, rho, ux, uy):
        """Equilibrium initialisation from this slab's rows of full-grid fields."""
        sl = slice(self.y0, self.y0 + self.rows)
        self.lat.init(rho[sl], ux[sl], uy[sl])
        return self

    def step(self, n: int = 1):
        from . import capi

        for _ in range(int(n)):
            self.lat._bind_stream()
            capi.kbc_halo_send(self.lat.h, 0, 0, self.send_lo)
            capi.kbc_halo_send(self.lat.h, 1, 0, self.send_hi)
            exchange(self.send_lo, self.send_hi, self.recv_lo, self.recv_hi, self.rank,
                     self.world, self.group)
            capi.kbc_halo_recv(self.lat.h, 0, 0, self.recv_lo)
            capi.kbc_halo_recv(self.lat.h, 1, 0, self.recv_hi)
            self.lat.step(1)
        return self

    def diagnostics(self) -> dict:
        """Global diagnostics of the split grid on every rank: full halos
        exchanged with the neighbours, this slab's partial set, an all-gather
        of the sets over the group and the library's merge in rank order."""
        import numpy as np
        import torch

        from . import capi

        lo, hi, rlo, rhi = _halo_buffers(self.lat, 4, full=True)
        self.lat._bind_stream()
        capi.kbc_halo_send(self.lat.h, 0, 1, lo)
        capi.kbc_halo_send(self.lat.h, 1, 1, hi)
        exchange(lo, hi, rlo, rhi, self.rank, self.world, self.group)
        capi.kbc_halo_recv(self.lat.h, 0, 1, rlo)
        capi.kbc_halo_recv(self.lat.h, 1, 1, rhi)
        part = torch.as_tensor(self.lat.diagnostics_partial(), device=self.lat.device)
        parts = gather_parts(part, self.rank, self.world, self.group)
        return merge_diagnostics(np.stack([p.cpu().numpy() for p in parts]))


def gather_parts(part, rank: int, world: int, group=None):
    """Every rank's partial diagnostics set, in rank order (an all-gather over
    the group; a single rank keeps its own)."""
    if world == 1:
        return [part]
    import torch
    import torch.distributed as dist

    out = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(out, part, group=group)
    return out
