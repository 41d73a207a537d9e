"""The multi-rank aggregation of bench.py (replicas, weak scaling) on CPU with gloo, 2 ranks.

Each rank reports its own time and HSAW count; the job's figures are the slowest rank's
time and the sum of the counts."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed, hits = bench.reduce_over_ranks(dist, torch, "cpu", 1.5 + rank, 1000 * (rank + 1))
    q.put((rank, elapsed, hits))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, elapsed, hits in out:
        assert elapsed == 2.5 and hits == 3000.0
