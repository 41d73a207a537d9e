"""The ordered cut (paper_1702_05854_gb300.shard) with the GPU chunk sampler on one rank.

With one rank the cut runs every round's chunks through the allocation-free library call;
the kept hits must be the first N hits of the oracle's stream (Alg. 3)."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hs = pytest.importorskip("paper_1702_05854_gb300")


def test_gpu_chunks_ordered_cut_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.distributed as dist
    from paper_1702_05854_gb300 import shard
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        d = synth.workload_c1()
        g = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
        bits = np.zeros((d["n"] + 31) // 32, np.uint32)
        for v in d["sources"]:
            bits[v >> 5] |= np.uint32(1 << (int(v) & 31))
        bits_dev = torch.from_numpy(bits.view(np.int32)).cuda()
        chunk = 1 << 16
        sample = shard.gpu_chunk_sampler(g, bits_dev, synth.SEED_WALKS, chunk)
        aid, ln = shard.ordered_cut(sample, 3000, chunk, 3, first_attempt=777)
    finally:
        dist.destroy_process_group()
    og = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    W = oracle.Stream(oracle.Query(og, d["sources"], seed=synth.SEED_WALKS), first_aid=777).extend(3000).export()
    assert np.array_equal(aid, W.aid)
    assert np.array_equal(ln, np.diff(W.node_off).astype(np.uint32))
