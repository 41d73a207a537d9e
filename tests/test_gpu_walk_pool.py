"""Walk-pool reuse gives exactly the oracle's results and the plain solver's (GPU).

A pool indexes attempt traces that do not depend on the query (per block of 2^22 attempts,
each node's list of attempts whose trace passes through it); queries with the pool's walk
seed take their hits inside the pool from their sources' lists and sample the rest.  Pooled
streams and solves are compared with the oracle's stream (Alg. 3) and solve (Alg. 4-9) on
the same seed, and with the same call on a graph without a pool.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hs = pytest.importorskip("paper_1702_05854_gb300")


def pair(d):
    plain = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    pooled = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    return plain, pooled


POOL = (1 << 22) + (1 << 21) + 777  # two index blocks, the second one partial


@pytest.fixture(scope="module")
def c1():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = synth.workload_c1()
    plain, pooled = pair(d)
    pooled.build_walk_pool(seed=4, attempts=POOL)
    return d, plain, pooled, oracle.Graph(d["n"], d["src"], d["dst"], d["w"])


def same_prefix(a, b, n):
    """The first n walks of two exported streams (they may hold different overshoots)."""
    (aa, oa, na, ea), (ab, ob, nb, eb) = a, b
    assert np.array_equal(aa[:n], ab[:n]) and np.array_equal(oa[:n + 1], ob[:n + 1])
    assert np.array_equal(na[:oa[n]], nb[:ob[n]]) and np.array_equal(ea[:oa[n] - n], eb[:ob[n] - n])


def same_solve(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for f in ("rounds_t", "hits", "attempts", "cov_R", "cov_Rprime", "hits_Rprime", "attempts_Rprime",
              "spread_base_est", "spread_reduction_est"):
        assert a[2][f] == b[2][f], f


def same_as_oracle(res, ores):
    """Integer outputs bit-exact, FP64 estimates within 1e-12 relative."""
    ids, gains, r = res
    oids, ogains, o = ores
    assert np.array_equal(ids, oids) and np.array_equal(gains, ogains)
    for f in ("rounds_t", "hits", "attempts", "cov_R", "cov_Rprime", "hits_Rprime", "attempts_Rprime"):
        assert r[f] == o[f], f
    for f in ("spread_base_est", "spread_reduction_est", "eps_t"):
        if math.isnan(o[f]):
            assert math.isnan(r[f]), f
        else:
            assert r[f] == pytest.approx(o[f], rel=1e-12, abs=0), f


@pytest.mark.parametrize("mode", [hs.HSAW_EDGE, hs.HSAW_NODE])
def test_pooled_solves_match_oracle_and_plain(c1, mode):
    d, plain, pooled, og = c1
    p = synth.probabilities(len(d["sources"]))
    S, S1 = d["sources"], d["sources"][:1]
    queries = [  # (hsaw query, oracle solve arguments)
        (hs.Query(sources=S, mode=mode, k=10, n_hsaw=20_000, seed=4), (S, None, 4, dict(k=10, n_hsaw=20_000))),
        (hs.Query(sources=S, mode=mode, k=10, sampling=hs.HSAW_STOP_RULE, eps=0.1, seed=4),
         (S, None, 4, dict(k=10, stop_rule=True, eps=0.1))),
        (hs.Query(sources=S, p_fixed=p, mode=mode, k=20, n_hsaw=8_000, seed=4), (S, p, 4, dict(k=20, n_hsaw=8_000))),
        # one source, hit rate ~0.17%: needs attempts beyond the pool (index, then sampler)
        (hs.Query(sources=S1, mode=mode, k=5, n_hsaw=15_000, seed=4), (S1, None, 4, dict(k=5, n_hsaw=15_000))),
        # other seed: no pool
        (hs.Query(sources=S, mode=mode, k=10, n_hsaw=5_000, seed=5), (S, None, 5, dict(k=10, n_hsaw=5_000))),
    ]
    omode = oracle.MODE_EDGE if mode == hs.HSAW_EDGE else oracle.MODE_NODE
    for q, (src, pf, seed, kw) in queries:
        got = hs.hsaw_solve(pooled, q)
        same_as_oracle(got, oracle.solve(oracle.Query(og, src, p_fixed=pf, seed=seed), omode, **kw))
        same_solve(got, hs.hsaw_solve(plain, q))
    assert hs.hsaw_solve(pooled, queries[3][0])[2]["attempts"] > POOL


def assert_stream_is_oracles(exported, ostream):
    """The first len(ostream) walks of an exported stream are the oracle's, bit for bit."""
    aid, off, nodes, edges = exported
    W = ostream.export()
    n = len(W)
    assert np.array_equal(aid[:n], W.aid) and np.array_equal(off[:n + 1], W.node_off)
    assert np.array_equal(nodes[:W.node_off[n]], W.nodes) and np.array_equal(edges[:W.node_off[n] - n], W.edges)


def test_pooled_streams_match_oracle_and_plain(c1):
    d, plain, pooled, og = c1
    q = hs.Query(sources=d["sources"], k=1, seed=4)
    p = synth.probabilities(len(d["sources"]))
    qp = hs.Query(sources=d["sources"], p_fixed=p, k=1, seed=4)
    # windows inside the first block, across the block boundary, across the pool's end
    for first in (0, 12345, (1 << 22) - 1000, POOL - 3000):
        got = hs.hsaw_sample(pooled, q, first, 3000).export()
        ost = oracle.Stream(oracle.Query(og, d["sources"], seed=4), first_aid=first).extend(3000)
        assert_stream_is_oracles(got, ost)
        if first == POOL - 3000:
            assert int(ost.export().aid[-1]) >= POOL  # the window runs past the pool's end
        same_prefix(got, hs.hsaw_sample(plain, q, first, 3000).export(), 3000)
    # probabilistic suspects across the block boundary (the coin filters pooled entries)
    first = (1 << 22) - 300_000
    got = hs.hsaw_sample(pooled, qp, first, 1500).export()
    ost = oracle.Stream(oracle.Query(og, d["sources"], p_fixed=p, seed=4), first_aid=first).extend(1500)
    assert int(ost.export().aid[-1]) >= 1 << 22
    assert_stream_is_oracles(got, ost)
    # residual graphs bypass the pool and still agree
    er = (np.arange(d["m"]) % 7 == 0).astype(np.uint8)
    same_prefix(hs.hsaw_sample(pooled, q, 0, 2000, edge_removed=er).export(),
                hs.hsaw_sample(plain, q, 0, 2000, edge_removed=er).export(), 2000)


def test_pooled_unequal_weights_and_served(c1):
    d = synth.workload_rmat(14, "random", 50, 20, "node")
    plain, pooled = pair(d)
    pooled.build_walk_pool(seed=7, attempts=1 << 21)
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_NODE, k=20, sampling=hs.HSAW_STOP_RULE, eps=0.2, seed=7)
    got = hs.hsaw_solve(pooled, q)
    og = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    same_as_oracle(got, oracle.solve(oracle.Query(og, d["sources"], seed=7), oracle.MODE_NODE, 20, stop_rule=True,
                                     eps=0.2))
    same_solve(got, hs.hsaw_solve(plain, q))
    srv = hs.Server([pooled], workers=4)
    ts = [srv.submit(0, q) for _ in range(6)]
    ref = hs.hsaw_solve(plain, q)
    for t in ts:
        ids, gains, r, lat = srv.poll(t)
        same_solve((ids, gains, r), ref)
    srv.close()
    pooled.drop_walk_pool()
    same_solve(hs.hsaw_solve(pooled, q), ref)


def test_pool_rebuild_drop_and_invalid(c1):
    d = synth.workload_c1()
    plain, pooled = pair(d)
    q4 = hs.Query(sources=d["sources"], mode=hs.HSAW_NODE, k=10, n_hsaw=4_000, seed=4)
    q9 = hs.Query(sources=d["sources"], mode=hs.HSAW_NODE, k=10, n_hsaw=4_000, seed=9)
    with pytest.raises(hs.HsawError) as e:
        pooled.build_walk_pool(seed=4, attempts=(1 << 32) + 1)
    assert e.value.status == -1
    pooled.build_walk_pool(seed=4, attempts=1 << 20)
    pooled.build_walk_pool(seed=9, attempts=(1 << 21) + 5)  # replaces the seed-4 pool
    for q in (q4, q9):                                      # seed 4: plain path; seed 9: pooled
        same_solve(hs.hsaw_solve(pooled, q), hs.hsaw_solve(plain, q))
    pooled.build_walk_pool(seed=9, attempts=0)              # zero attempts: no pool
    same_solve(hs.hsaw_solve(pooled, q9), hs.hsaw_solve(plain, q9))
