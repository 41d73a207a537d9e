"""Ordered cut of the HSAW stream across ranks (attempt-range sharding).

The stream R_1, R_2, ... (Alg. 3) is the hits of attempts 0, 1, 2, ... in attempt order, and
attempts are independent, so G ranks can examine disjoint attempt ranges at once: attempts
are grouped in chunks of `chunk` consecutive ids, and rank g examines the chunks c with
c = g (mod G).  One exchange per round fixes the global order: an all-gather of the hit
count of every chunk.  With those counts every rank knows where the N-th hit falls (chunk
c*, position r*), keeps its hits of chunks before c* (and the first r* of c* if it owns
c*), and the kept hits are gathered in chunk order.  The result is exactly the first N
hits of the single-rank stream, with the attempt count A = 1 + the N-th hit's attempt id.

The per-chunk sampler is passed in: on a GPU it is a library call that returns the hits of
an attempt range (for example ``hsaw_sample_hits_static``); any function with the same
contract (ordered attempt ids and walk lengths of the range's hits) works, which is how the
multi-rank logic is tested on CPU ranks.
"""
from __future__ import annotations

from typing import Callable, Tuple

import numpy as np

ChunkSampler = Callable[[int, int], Tuple[np.ndarray, np.ndarray]]


def owned_chunks(round_first_chunk: int, chunks_per_rank: int, rank: int, world: int):
    """Chunk ids rank `rank` examines in a round that starts at chunk `round_first_chunk`."""
    return [round_first_chunk + i * world + rank for i in range(chunks_per_rank)]


def locate_cut(counts: np.ndarray, need: int):
    """(chunk index, hits taken from it) of the `need`-th hit (need >= 1) in chunk order, or
    None when the chunks hold fewer than `need` hits."""
    c = np.cumsum(counts.astype(np.int64))
    if c.size == 0 or c[-1] < need:
        return None
    i = int(np.searchsorted(c, need))  # first chunk whose running total reaches need
    before = int(c[i - 1]) if i > 0 else 0
    return i, need - before


def ordered_cut(sample_chunk: ChunkSampler, n_hits: int, chunk: int, chunks_per_rank: int, group=None,
                first_attempt: int = 0, max_rounds: int = 1 << 20):
    """The first n_hits hits (attempt ids uint64, walk lengths uint32) of the stream, drawn
    by all ranks of `group` (torch.distributed) over attempt chunks c = rank (mod world).
    Every rank returns the same arrays.  Exchanges per round: an all-gather of per-chunk hit
    counts, then an all-gather of the kept hits."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    kept_aid, kept_len = [], []
    have = 0
    next_chunk = 0
    for _ in range(max_rounds):
        mine = owned_chunks(next_chunk, chunks_per_rank, rank, world)
        hits = [sample_chunk(first_attempt + c * chunk, chunk) for c in mine]
        counts = torch.tensor([h[0].shape[0] for h in hits], dtype=torch.int64)
        everyone = [torch.zeros_like(counts) for _ in range(world)]
        dist.all_gather(everyone, counts, group=group)
        # chunk order of the round: chunk next_chunk + i * world + g is entry (i, g)
        per_chunk = torch.stack(everyone, dim=1).reshape(-1).numpy()
        cut = locate_cut(per_chunk, n_hits - have)
        take = np.zeros(per_chunk.shape[0], np.int64)
        if cut is None:
            take[:] = per_chunk
        else:
            ci, r = cut
            take[:ci] = per_chunk[:ci]
            take[ci] = r
        # my kept hits, in my chunk order; gathered and laid out in global chunk order
        my_take = [int(take[i * world + rank]) for i in range(chunks_per_rank)]
        aid = np.concatenate([h[0][:t] for h, t in zip(hits, my_take)]).astype(np.uint64)
        ln = np.concatenate([h[1][:t] for h, t in zip(hits, my_take)]).astype(np.uint32)
        sizes = [int(sum(take[i * world + g] for i in range(chunks_per_rank))) for g in range(world)]
        width = max(sizes) if sizes else 0
        buf = torch.zeros((width, 2), dtype=torch.int64)
        if aid.size:
            buf[:aid.size, 0] = torch.from_numpy(aid.view(np.int64))
            buf[:aid.size, 1] = torch.from_numpy(ln.astype(np.int64))
        bufs = [torch.zeros_like(buf) for _ in range(world)]
        dist.all_gather(bufs, buf, group=group)
        parts = [b[:sizes[g]].numpy() for g, b in enumerate(bufs)]
        # interleave back to chunk order: rank g's hits of its i-th chunk come after chunk (i, g-1)
        offs = [0] * world
        for i in range(chunks_per_rank):
            for g in range(world):
                t = int(take[i * world + g])
                if t:
                    seg = parts[g][offs[g]:offs[g] + t]
                    kept_aid.append(seg[:, 0].view(np.uint64).copy())
                    kept_len.append(seg[:, 1].astype(np.uint32))
                    offs[g] += t
        have += int(take.sum())
        if cut is not None:
            break
        next_chunk += chunks_per_rank * world
    else:
        raise RuntimeError("ordered_cut: attempt rounds exhausted before enough hits")
    aid = np.concatenate(kept_aid) if kept_aid else np.zeros(0, np.uint64)
    ln = np.concatenate(kept_len) if kept_len else np.zeros(0, np.uint32)
    return aid, ln


def gpu_chunk_sampler(graph, suspect_bits, seed: int, chunk: int):
    """A ChunkSampler over the allocation-free library call (p == 1, no removed elements):
    the hits of attempts [first, first + chunk) on this rank's GPU."""
    import torch

    from . import hsaw_sample_hits_static

    aid_out = torch.empty(chunk, dtype=torch.int64, device="cuda")
    len_out = torch.empty(chunk, dtype=torch.int32, device="cuda")

    def sample(first: int, count: int):
        n = hsaw_sample_hits_static(graph, suspect_bits, seed, first, count, aid_out, len_out)
        return aid_out[:n].cpu().numpy().view(np.uint64), len_out[:n].cpu().numpy().view(np.uint32)

    return sample
