"""Batched and served solves give exactly the results of each instance solved alone.

Also host-side failure handling of the server: rejection by memory admission,
cancellation of queued and running queries, per-instance error statuses in a batch.
None of these tests faults, traps or hangs the GPU: failures are made on the host.
"""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hs = pytest.importorskip("paper_1702_05854_gb300")


def small_instances(count, seed=0):
    """Chung-Lu graphs of uneven size with eSI/nSI, fixed-N and stopping-rule queries."""
    rng = np.random.default_rng(seed)
    graphs, queries = [], []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(1000), np.log(30000))))
        deg = int(rng.integers(8, 33))
        src, dst = synth.chung_lu_graph(n, n * deg, 2.1, seed=100 + i)
        w = synth.wc_weights(n, dst)
        g = hs.hsaw_graph_from_edges(n, src, dst, w)
        ns = int(min(n, np.exp(rng.uniform(0, np.log(300)))))
        S = synth.sources(n, ns, seed=200 + i)
        mode = hs.HSAW_EDGE if i % 2 == 0 else hs.HSAW_NODE
        M = n * deg if mode == hs.HSAW_EDGE else n
        k = int(min(M, rng.integers(10, 200)))
        if i % 3 == 2:
            q = hs.Query(sources=S, mode=mode, k=k, sampling=hs.HSAW_STOP_RULE, eps=0.2, seed=4 + i)
        else:
            q = hs.Query(sources=S, mode=mode, k=k, n_hsaw=int(rng.integers(2000, 40000)), seed=4 + i)
        graphs.append(g)
        queries.append(q)
    return graphs, queries


@pytest.fixture(scope="module")
def inst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return small_instances(12)


def same(a, b):
    ids, gains, r = a
    ids2, gains2, r2 = b
    assert np.array_equal(ids, ids2) and np.array_equal(gains, gains2)
    for f in ("rounds_t", "hits", "attempts", "cov_R", "cov_Rprime", "hits_Rprime", "attempts_Rprime",
              "spread_base_est", "spread_reduction_est"):
        assert r[f] == r2[f], f


@pytest.mark.parametrize("way", ["joint", "threads"])
def test_batch_matches_serial(inst, monkeypatch, way):
    """joint: the fixed-N instances sampled together by multi-instance sampler launches;
    threads: every instance solved whole on the worker threads."""
    graphs, queries = inst
    alone = [hs.hsaw_solve(g, q) for g, q in zip(graphs, queries)]
    monkeypatch.setenv("HSAW_BATCH", way)
    for conc in (1, 4, 12):
        out = hs.hsaw_solve_batch(graphs, queries, concurrency=conc)
        for (st, ids, gains, r), a in zip(out, alone):
            assert st == 0
            same((ids, gains, r), a)


@pytest.mark.parametrize("way", ["joint", "threads"])
def test_batch_with_probabilities_and_budgets(inst, monkeypatch, way):
    """Probabilistic suspects, a candidate mask, an instance whose attempt budget runs out
    (HSAW_E_TIMEOUT for it alone) and one with too few candidates (HSAW_E_INVALID)."""
    monkeypatch.setenv("HSAW_BATCH", way)
    graphs, queries = inst
    g0, g1 = graphs[0], graphs[1]
    q = queries[0]
    p = synth.probabilities(len(q.sources))
    M = g1.m
    cm = (np.arange(M) % 2 == 0).astype(np.uint8)
    qs = [hs.Query(sources=q.sources, p_fixed=p, mode=hs.HSAW_NODE, k=7, n_hsaw=5000, seed=11),
          hs.Query(sources=queries[1].sources, mode=hs.HSAW_EDGE, k=9, n_hsaw=7000, seed=12, candidate_mask=cm),
          hs.Query(sources=q.sources[:1], mode=hs.HSAW_NODE, k=3, n_hsaw=10 ** 6, seed=13, max_attempts=1 << 20),
          hs.Query(sources=q.sources, mode=hs.HSAW_NODE, k=g0.n + 1, n_hsaw=100, seed=14)]
    gs = [g0, g1, g0, g0]
    out = hs.hsaw_solve_batch(gs, qs, concurrency=3)
    assert [o[0] for o in out] == [0, 0, -7, -1]
    for (st, ids, gains, r), g, qq in zip(out[:2], gs[:2], qs[:2]):
        same((ids, gains, r), hs.hsaw_solve(g, qq))


def test_batch_reports_per_instance_errors(inst):
    graphs, queries = inst
    bad = hs.Query(sources=np.array([0, 0], np.int32), k=1, n_hsaw=10)  # duplicate source
    out = hs.hsaw_solve_batch(graphs[:3] + [graphs[3]], queries[:3] + [bad], concurrency=4)
    assert [o[0] for o in out[:3]] == [0, 0, 0] and out[3][0] == -1
    for (st, ids, gains, r), q, g in zip(out[:3], queries[:3], graphs[:3]):
        same((ids, gains, r), hs.hsaw_solve(g, q))


def test_server_mix_matches_alone(inst):
    graphs, queries = inst
    srv = hs.Server(graphs[:4], workers=6)
    plan = [(i % 4, queries[i % 4]) for i in range(16)]
    tickets = [srv.submit(gi, q) for gi, q in plan]  # they overlap on the GPU
    results = [srv.poll(t) for t in tickets]
    for (gi, q), (ids, gains, r, lat) in zip(plan, results):
        same((ids, gains, r), hs.hsaw_solve(graphs[gi], q))
        assert lat > 0
    srv.close()


def test_server_rejects_over_budget(inst):
    graphs, queries = inst
    srv = hs.Server(graphs[:1], mem_budget=1 << 20, workers=1)
    with pytest.raises(hs.HsawError) as e:
        srv.submit(0, queries[0])
    assert e.value.status == -8
    srv.close()


def slow_setup():
    """A 2^20-node graph without edges: a query hits only when its attempt starts on the
    source (probability 2^-20 per attempt), so N hits take ~N * 2^20 attempts."""
    n = 1 << 20
    g = hs.hsaw_graph_from_edges(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    return g, np.array([12345], np.int32)


def test_server_cancel_queued_and_running(inst):
    g, S = slow_setup()
    d = synth.workload_c1()
    g1 = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    srv = hs.Server([g, g1], workers=1)
    long_q = hs.Query(sources=S, mode=hs.HSAW_NODE, k=1, n_hsaw=1_000_000, seed=9)  # ~1e12 attempts
    t_run = srv.submit(0, long_q)
    t_wait = srv.submit(0, long_q)          # queued behind it (one worker)
    time.sleep(0.3)
    srv.cancel(t_wait)
    srv.cancel(t_run)
    for t in (t_run, t_wait):
        with pytest.raises(hs.HsawError) as e:
            srv.poll(t, timeout_ms=60_000)
        assert e.value.status == -9
    # the server keeps serving after cancellations
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_EDGE, k=10, n_hsaw=5000, seed=4)
    ids, gains, r, lat = srv.poll(srv.submit(1, q))
    same((ids, gains, r), hs.hsaw_solve(g1, q))
    srv.close()


def test_server_poll_timeout_keeps_ticket():
    g, S = slow_setup()
    srv = hs.Server([g], workers=1)
    q = hs.Query(sources=S, mode=hs.HSAW_NODE, k=1, n_hsaw=300, seed=9)  # ~3e8 attempts
    t = srv.submit(0, q)
    with pytest.raises(hs.HsawError) as e:
        srv.poll(t, timeout_ms=0)
    assert e.value.status == -10  # HSAW_E_PENDING: still running, ticket kept
    ids, gains, r, lat = srv.poll(t)
    assert r["hits"] == 300 and ids[0] == 12345
    # a query whose own attempt budget runs out reports HSAW_E_TIMEOUT, and its ticket is gone
    t2 = srv.submit(0, hs.Query(sources=S, mode=hs.HSAW_NODE, k=1, n_hsaw=300, seed=9, max_attempts=1 << 20))
    with pytest.raises(hs.HsawError) as e:
        srv.poll(t2)
    assert e.value.status == -7
    with pytest.raises(hs.HsawError) as e:
        srv.poll(t2, timeout_ms=0)
    assert e.value.status == -1  # unknown ticket
    srv.close()
