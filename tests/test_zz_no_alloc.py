"""The allocation-free sampler entry point agrees with the allocating one.

hsaw_sample_hits_static serves callers that must not allocate device memory while they
run (a framework that owns every device allocation through its own pool, or a loop that
cannot afford cudaMalloc's device-wide synchronisation).  Its scratch is a static device
array shared by every call, so this test makes two calls in a row on the same array and
checks each against hsaw_sample, the entry point that allocates its own workspace.
The file is named to run last: if it fails, every other test has already run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hs = pytest.importorskip("paper_1702_05854_gb300")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = synth.workload_c1()
    g = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    bits = np.zeros((d["n"] + 31) // 32, np.uint32)
    for v in d["sources"]:
        bits[v >> 5] |= np.uint32(1 << (int(v) & 31))
    bits_dev = torch.from_numpy(bits.view(np.int32)).cuda()
    return d, g, bits_dev


def reference_hits(g, d, first, count, seed):
    """Hits in [first, first + count) from the allocating entry point."""
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_EDGE, k=1, seed=seed)
    need = 64
    while True:
        w = hs.hsaw_sample(g, q, first, need)
        aid, off, _, _ = w.export()
        if aid.size and int(aid[-1]) >= first + count:
            break
        need *= 2
    lens = np.diff(off).astype(np.uint32)
    sel = aid < first + count
    return aid[sel], lens[sel]


def test_static_sampler_matches_allocating_sampler(setup):
    d, g, bits = setup
    seed = synth.SEED_WALKS
    cap = hs.HSAW_STATIC_MAX_ATTEMPTS
    aid_out = torch.empty(cap, dtype=torch.int64, device="cuda")
    len_out = torch.empty(cap, dtype=torch.int32, device="cuda")
    ranges = [(0, cap), (cap, cap - 777)]  # two calls in a row on the shared scratch, one ragged
    for first, count in ranges:
        n = hs.hsaw_sample_hits_static(g, bits, seed, first, count, aid_out, len_out)
        got_aid = aid_out[:n].cpu().numpy().view(np.uint64)
        got_len = len_out[:n].cpu().numpy().view(np.uint32)
        ref_aid, ref_len = reference_hits(g, d, first, count, seed)
        assert n > 100
        assert np.array_equal(got_aid, ref_aid)
        assert np.array_equal(got_len, ref_len)


def test_static_sampler_rejects_oversized_range(setup):
    d, g, bits = setup
    aid_out = torch.empty(16, dtype=torch.int64, device="cuda")
    len_out = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(hs.HsawError) as e:
        hs.hsaw_sample_hits_static(g, bits, 4, 0, hs.HSAW_STATIC_MAX_ATTEMPTS + 1, aid_out, len_out)
    assert e.value.status == -1
    with pytest.raises(hs.HsawError) as e:  # more hits than the output holds
        hs.hsaw_sample_hits_static(g, bits, 4, 0, 100_000, aid_out, len_out)
    assert e.value.status == -1
