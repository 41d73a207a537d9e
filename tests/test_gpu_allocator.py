"""Scratch device memory from a caller's allocator (hsaw_set_allocator), here torch's
caching allocator: a fixed-N and a stopping-rule solve give the same result as with CUDA's
pool, every block handed out comes back, the allocator cannot change while the library
holds scratch (a live walks handle), and an allocator with no memory fails the call with
HSAW_E_NOMEM instead of faulting."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hs = pytest.importorskip("paper_1702_05854_gb300")

E_INVALID, E_NOMEM = -1, -4


@pytest.fixture(scope="module")
def c1():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = synth.workload_c1()
    g = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    return d, g


class CountingTorchAllocator:
    """torch's caching allocator, with the blocks the library holds."""

    def __init__(self):
        self.live, self.allocs, self.releases = {}, 0, 0

    def alloc(self, nbytes, stream):
        p = torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
        self.allocs += 1
        self.live[p] = nbytes
        return p

    def release(self, ptr, stream):
        self.releases += 1
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)

    def __enter__(self):
        hs.hsaw_set_allocator(self.alloc, self.release)
        return self

    def __exit__(self, *exc):
        torch.cuda.synchronize()
        hs.hsaw_set_allocator()


def _same(a, b):
    return a == b or (isinstance(a, float) and a != a and b != b)


@pytest.mark.parametrize("sampling", ["fixed", "stop"])
def test_torch_allocator_gives_the_same_solve(c1, sampling):
    d, g = c1
    kw = dict(sources=d["sources"], mode=hs.HSAW_EDGE, k=50, seed=synth.SEED_WALKS)
    q = hs.Query(n_hsaw=20_000, **kw) if sampling == "fixed" else hs.Query(sampling=hs.HSAW_STOP_RULE, eps=0.2, **kw)
    ids0, gains0, r0 = hs.hsaw_solve(g, q)
    with CountingTorchAllocator() as a:
        ids1, gains1, r1 = hs.hsaw_solve(g, q)
        torch.cuda.synchronize()
        assert a.allocs > 0 and a.allocs == a.releases and not a.live
    assert np.array_equal(ids0, ids1) and np.array_equal(gains0, gains1)
    assert r0.keys() == r1.keys() and all(_same(r0[k], r1[k]) for k in r0)


def test_allocator_change_refused_while_scratch_is_held(c1):
    d, g = c1
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_EDGE, k=10, n_hsaw=1000, seed=synth.SEED_WALKS)
    with CountingTorchAllocator() as a:
        w = hs.hsaw_sample(g, q, 0, 500)
        assert a.live  # the walks handle holds its stream buffers
        with pytest.raises(hs.HsawError) as e:
            hs.hsaw_set_allocator()
        assert e.value.status == E_INVALID
        w.close()
        assert not a.live and a.allocs == a.releases
    hs.hsaw_set_allocator()  # nothing held: accepted


def test_allocator_without_memory_reports_nomem(c1):
    d, g = c1
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_EDGE, k=10, n_hsaw=1000, seed=synth.SEED_WALKS)
    hs.hsaw_set_allocator(lambda n, s: 0, lambda p, s: None)
    try:
        with pytest.raises(hs.HsawError) as e:
            hs.hsaw_solve(g, q)
        assert e.value.status == E_NOMEM
    finally:
        hs.hsaw_set_allocator()  # refused if the failed call kept a block
    ids, gains, r = hs.hsaw_solve(g, q)  # the pool serves again
    assert r["hits"] == 1000
