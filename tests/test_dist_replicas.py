"""Multi-process path of bench.py on CPU: two gloo ranks act as replicas.

Each rank times its own work; the job's time is the maximum over ranks
after a barrier and its throughput counts the node updates of every rank.
The reference arm prints only on rank 0.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench

    r = bench.Ranks()
    assert (r.world, r.rank) == (world, rank)
    r.init("gloo")
    r.barrier()
    t = 1.5 + rank  # rank 1 is the slow one
    tmax = r.max(t, "cpu")
    value = bench.job_mlups(r.world, 1024 * 1024, 100, tmax)
    r.barrier()
    r.close()
    q.put((rank, tmax, value))


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(world))
    for rank, tmax, value in out:
        assert tmax == 2.5
        assert value == pytest.approx(2 * 1024 * 1024 * 100 / 2.5 / 1e6)


def test_single_process_defaults():
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    r = bench.Ranks()
    assert (r.world, r.rank, r.local) == (1, 0, 0)
    r.init("gloo")  # no process group for one rank
    assert r.max(3.0, "cpu") == 3.0
    r.close()
