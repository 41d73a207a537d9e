"""Edge lookup, residual-graph spread estimates and allocation-failure handling (GPU).

hsaw_estimate_spread is checked against the oracle bit for bit (same integer counts)
and against brute-force live-edge enumeration on tiny graphs (within 4 standard errors).
Allocation failures are injected on the host (a test hook that makes the n-th device
allocation report out-of-memory); no GPU fault is involved.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tinygraphs import random_tiny

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hs = pytest.importorskip("paper_1702_05854_gb300")


@pytest.fixture(scope="module")
def c1():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = synth.workload_c1()
    return d, hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"]), oracle.Graph(d["n"], d["src"], d["dst"],
                                                                                        d["w"])


def test_graph_edge_lookup(c1):
    d, g, og = c1
    rp, s, dd, thr, ii = og.arrays()
    for e in list(np.random.default_rng(1).integers(0, d["m"], 50)) + [0, d["m"] - 1]:
        assert hs.hsaw_graph_edge(g, int(e)) == (int(s[e]), int(dd[e]), int(ii[e]))
    with pytest.raises(hs.HsawError) as ex:
        hs.hsaw_graph_edge(g, d["m"])
    assert ex.value.status == -3


def test_estimate_spread_matches_oracle(c1):
    d, g, og = c1
    rng = np.random.default_rng(3)
    for mode, M in ((hs.HSAW_EDGE, d["m"]), (hs.HSAW_NODE, d["n"])):
        removed = np.sort(rng.choice(M, size=300, replace=False))
        q = hs.Query(sources=d["sources"], mode=mode, k=1, n_hsaw=4000, seed=17)
        sp, se = hs.hsaw_estimate_spread(g, q, removed)
        mask = np.zeros(M, np.uint8)
        mask[removed] = 1
        kw = dict(edge_removed=mask) if mode == hs.HSAW_EDGE else dict(node_removed=mask)
        st = oracle.Stream(oracle.Query(og, d["sources"], seed=17, **kw)).extend(4000)
        W = st.export()
        A = int(W.aid[3999]) + 1
        assert sp == pytest.approx(d["n"] * 4000 / A, rel=1e-12)
        f = 4000 / A
        assert se == pytest.approx(d["n"] * math.sqrt(f * (1 - f) / A), rel=1e-12)
        # removing nothing gives a larger spread than removing 300 elements
        sp0, _ = hs.hsaw_estimate_spread(g, q)
        assert sp0 > sp


@pytest.mark.parametrize("gseed", range(6))
def test_estimate_spread_matches_bruteforce(gseed):
    n, src, dst, w = random_tiny(800 + gseed, n=7, m=12)
    g, og = hs.hsaw_graph_from_edges(n, src, dst, w), oracle.Graph(n, src, dst, w)
    S = np.array([gseed % n, (gseed + 2) % n], np.int32)
    node_mode = gseed % 2 == 1
    M = n if node_mode else len(src)
    T = np.array([gseed % M, (3 * gseed + 1) % M], np.int64)
    T = np.unique(T)
    mask = np.zeros(M, np.uint8)
    mask[T] = 1
    kw = dict(node_removed=mask) if node_mode else dict(edge_removed=mask)
    exact = oracle.bruteforce_spread(og, S, **kw)
    q = hs.Query(sources=S, mode=hs.HSAW_NODE if node_mode else hs.HSAW_EDGE, k=1, n_hsaw=50_000, seed=gseed)
    sp, se = hs.hsaw_estimate_spread(g, q, T)
    assert abs(sp - exact) <= 4 * se + 1e-9, (sp, exact, se)


def test_allocation_failures_are_reported_and_recovered(c1):
    d, g, og = c1
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_EDGE, k=10, sampling=hs.HSAW_STOP_RULE, eps=0.2, seed=4)
    ref = hs.hsaw_solve(g, q)
    seen_nomem = 0
    try:
        for k in range(1, 80, 3):
            hs.hsaw_debug_fail_alloc_after(k)
            try:
                ids, gains, r = hs.hsaw_solve(g, q)
                assert np.array_equal(ids, ref[0]) and np.array_equal(gains, ref[1])
            except hs.HsawError as e:
                assert e.status == -4
                seen_nomem += 1
            hs.hsaw_debug_fail_alloc_after(0)
            ids, gains, r = hs.hsaw_solve(g, q)  # the library is still usable
            assert np.array_equal(ids, ref[0]) and np.array_equal(gains, ref[1])
        # graph ingest too
        hs.hsaw_debug_fail_alloc_after(2)
        with pytest.raises(hs.HsawError) as e:
            hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
        assert e.value.status == -4
    finally:
        hs.hsaw_debug_fail_alloc_after(0)
    assert seen_nomem > 5
    g2 = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    assert np.array_equal(hs.hsaw_solve(g2, q)[0], ref[0])


def test_profile_counters_reset_and_results_unchanged(c1):
    d, g, og = c1
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_EDGE, k=10, sampling=hs.HSAW_STOP_RULE, eps=0.2, seed=4)
    hs.hsaw_profile_enable(False)
    ref = hs.hsaw_solve(g, q)
    for _ in range(3):  # repeated enables recycle the timing events
        hs.hsaw_profile_enable(True)
        got = hs.hsaw_solve(g, q)
        p = hs.hsaw_profile_read()
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        assert p["kernel_launches"] > 0 and p["sampler_launches"] >= 1 and p["sampler_ms"] > 0
        assert p["sampler_steps"] == got[2]["steps"]
        assert all(p["phase_ms"][k] > 0 for k in ("sampling", "counting", "greedy", "coverage"))
    hs.hsaw_profile_enable(False)
    p = hs.hsaw_profile_read()
    assert p["kernel_launches"] == 0 and p["sampler_launches"] == 0 and p["phase_ms"]["greedy"] == 0


def test_walks_export_device_equals_host(c1):
    """Device export into caller-owned torch tensors gives the host export's arrays."""
    d, g = c1[0], c1[1]
    w = hs.hsaw_sample(g, hs.Query(sources=d["sources"], k=1, seed=4), 100, 3000)
    aid, off, nodes, edges = w.export()
    daid, doff, dnodes, dedges = w.export_device()
    assert np.array_equal(daid.cpu().numpy().view(np.uint64), aid) and np.array_equal(doff.cpu().numpy(), off)
    assert np.array_equal(dnodes.cpu().numpy(), nodes) and np.array_equal(dedges.cpu().numpy(), edges)
