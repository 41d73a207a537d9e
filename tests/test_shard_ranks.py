"""The ordered cut across attempt-range shards (paper_1702_05854_gb300.shard) on CPU ranks.

Two and three gloo ranks each examine the attempt chunks c = rank (mod world), exchange
per-chunk hit counts, cut at the N-th hit and gather the kept hits in chunk order.  Each
rank's hits come from a CPU stand-in for its GPU (the oracle's per-attempt outcomes of the
chunk), and the merged stream must equal the first N hits of the single-rank oracle stream
(Alg. 3): same attempt ids in the same order, same walk lengths.
"""
import os
import socket

import numpy as np
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


def _oracle_query():
    import oracle
    import synth
    d = synth.workload_c1()
    g = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    return g, oracle.Query(g, d["sources"], seed=synth.SEED_WALKS)


def _rank(rank, world, port, q, n_hits, chunk, per_rank, first):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1702_05854_gb300 import shard
    g, oq = _oracle_query()
    seen = []

    def sample_chunk(a0, count):  # CPU stand-in for this rank's GPU: hits of [a0, a0 + count)
        seen.append(a0)
        out, ln = oq.classify(a0, count)
        idx = np.nonzero(out == oracle.HIT)[0]
        return (a0 + idx).astype(np.uint64), ln[idx].astype(np.uint32)

    aid, ln = shard.ordered_cut(sample_chunk, n_hits, chunk, per_rank, first_attempt=first)
    owned_ok = all(((a - first) // chunk) % world == rank for a in seen)
    q.put((rank, aid, ln, owned_ok))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_hits,chunk,per_rank,first", [(2, 2500, 16384, 4, 0), (3, 1777, 10000, 2, 1000),
                                                              (2, 1, 4096, 1, 5)])
def test_ordered_cut_equals_single_rank_stream(world, n_hits, chunk, per_rank, first):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, n_hits, chunk, per_rank, first))
             for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    _, oq = _oracle_query()
    W = oracle.Stream(oq, first_aid=first).extend(n_hits).export()
    want_len = np.diff(W.node_off).astype(np.uint32)
    for rank, aid, ln, owned_ok in out:
        assert owned_ok  # each rank examined only its own chunks
        assert np.array_equal(aid, W.aid) and np.array_equal(ln, want_len)


def test_locate_cut():
    from paper_1702_05854_gb300.shard import locate_cut
    c = np.array([0, 3, 0, 2, 5])
    assert locate_cut(c, 1) == (1, 1) and locate_cut(c, 3) == (1, 3) and locate_cut(c, 4) == (3, 1)
    assert locate_cut(c, 10) == (4, 5) and locate_cut(c, 11) is None and locate_cut(np.zeros(0), 1) is None
