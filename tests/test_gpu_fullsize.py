"""Full-size parity: the billion-edge eSI workload in the launch configuration bench.py times,
and the nSI R-MAT 20 random-LT workload with N = 10 M HSAWs.

R-MAT scale 26 (67,108,864 nodes, 1,073,741,824 edges), weighted-cascade weights,
|S| = 1,000, k = 1,000, stopping rule eps = 0.1, delta = 1/n.  The oracle cannot solve
this size, so it checks sampled outputs one by one (walks re-derived from their attempt
ids, every attempt of random windows classified), and the counting and greedy are
checked through properties that hold at any size (recounts, the greedy's first pick,
non-increasing gains, gains adding up to the coverage, Check recomputed from the counts).
Needs a GB300 and about 60 GB of host memory; takes a few minutes.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hs = pytest.importorskip("paper_1702_05854_gb300")


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = synth.workload_c3(26)
    g = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_EDGE, k=d["k"], sampling=hs.HSAW_STOP_RULE, eps=d["eps"],
                 seed=synth.SEED_WALKS)
    ids, gains, res = hs.hsaw_solve(g, q)
    walks = hs.hsaw_sample(g, q, 0, res["hits"])
    aid, off, nodes, edges = walks.export()
    og = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    oq = oracle.Query(og, d["sources"], seed=synth.SEED_WALKS)
    return dict(d=d, g=g, q=q, ids=ids, gains=gains, res=res, aid=aid, off=off, nodes=nodes, edges=edges, og=og,
                oq=oq)


def test_fullsize_walks_rederived_by_oracle(full):
    aid, off, nodes, edges, oq = full["aid"], full["off"], full["nodes"], full["edges"], full["oq"]
    rng = np.random.default_rng(26)
    for j in rng.choice(full["res"]["hits"], size=300, replace=False):
        r, on, oe = oq.attempt(int(aid[j]))
        assert r == oracle.HIT
        assert np.array_equal(nodes[off[j]:off[j + 1]], on)
        assert np.array_equal(edges[off[j] - j:off[j + 1] - j - 1], oe)


def test_fullsize_attempt_windows_match_oracle(full):
    """Every attempt of random windows: same outcome on both sides, and the stream holds
    exactly the oracle's hits of the window (nothing skipped, nothing extra, in order)."""
    aid, oq, g, q = full["aid"], full["oq"], full["g"], full["q"]
    last = int(aid[-1])
    rng = np.random.default_rng(7)
    for first in list(rng.integers(0, last - 4000, size=3)) + [0, last - 2999]:
        first = int(first)
        out, _ = oq.classify(first, 3000)
        gout, _ = hs.hsaw_classify(g, q, first, 3000)
        assert np.array_equal(gout.cpu().numpy(), out)
        want = first + np.nonzero(out == oracle.HIT)[0].astype(np.uint64)
        sel = (aid >= first) & (aid < first + 3000)
        assert np.array_equal(aid[sel], want)


def test_fullsize_counts_and_greedy_properties(full):
    res, ids, gains, off, edges = full["res"], full["ids"], full["gains"], full["off"], full["edges"]
    half = res["hits"] // 2
    R = edges[:off[half] - half]
    walk_of = np.repeat(np.arange(half), np.diff(off[:half + 1]) - 1)
    uid, cnt = np.unique(R, return_counts=True)
    # first pick = largest count, smallest id on ties (Alg. 4 line 3)
    top = cnt.max()
    assert gains[0] == top and ids[0] == uid[np.nonzero(cnt == top)[0][0]]
    assert np.all(np.diff(gains.astype(np.int64)) <= 0)          # submodular coverage
    covered = np.zeros(half, bool)
    covered[walk_of[np.isin(R, ids)]] = True
    assert int(gains.sum()) == int(covered.sum()) == res["cov_R"]
    # out-of-sample coverage on R'_t
    Rp = edges[off[half] - half:off[2 * half] - 2 * half]
    wp = np.repeat(np.arange(half), np.diff(off[half:2 * half + 1]) - 1)
    cp = np.zeros(half, bool)
    cp[wp[np.isin(Rp, ids)]] = True
    assert int(cp.sum()) == res["cov_Rprime"]
    # the library's histogram of R_t is the recount
    huid, hcnt = hs.hsaw_histogram(hs.hsaw_sample(full["g"], full["q"], 0, half), hs.HSAW_EDGE, 0, half)
    assert np.array_equal(huid, uid.astype(np.int32)) and np.array_equal(hcnt, cnt.astype(np.uint32))


def test_fullsize_estimates_and_check(full):
    res, d = full["res"], full["d"]
    n = d["n"]
    assert res["attempts"] == int(full["aid"][res["hits"] - 1]) + 1
    assert res["spread_base_est"] == pytest.approx(n * res["hits"] / res["attempts"], rel=1e-12)
    assert res["spread_reduction_est"] == pytest.approx(n * (res["cov_R"] + res["cov_Rprime"]) / res["attempts"],
                                                        rel=1e-12)
    c = oracle.stop_constants(d["m"], d["k"], d["eps"], 1.0 / n)
    assert res["hits_Rprime"] * 2 == res["hits"] == math.ceil(c["Lambda"]) * 2 ** res["rounds_t"]
    ok, et = oracle.check(res["cov_R"], res["cov_Rprime"], res["hits_Rprime"], res["rounds_t"], d["eps"], c["Lambda1"])
    assert et == pytest.approx(res["eps_t"], rel=1e-12)
    assert ok or res["rounds_t"] == c["t_max"]


# ----------------------------------------------------------------------------- C2 at full size
@pytest.fixture(scope="module")
def c2():
    """nSI R-MAT 20 with random LT weights, |S| = 100, k = 100, N = 10 M HSAWs."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = synth.workload_c2()
    g = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_NODE, k=d["k"], n_hsaw=d["n_hsaw"], seed=synth.SEED_WALKS)
    ids, gains, res = hs.hsaw_solve(g, q)
    walks = hs.hsaw_sample(g, q, 0, d["n_hsaw"])
    aid, off, nodes, edges = walks.export()
    og = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    oq = oracle.Query(og, d["sources"], seed=synth.SEED_WALKS)
    return dict(d=d, g=g, q=q, ids=ids, gains=gains, res=res, aid=aid, off=off, nodes=nodes, edges=edges, oq=oq)


def test_c2_fullsize_sampled(c2):
    d, res, aid, off, nodes, edges, oq = (c2[k] for k in ("d", "res", "aid", "off", "nodes", "edges", "oq"))
    N = d["n_hsaw"]
    assert res["hits"] == N and res["attempts"] == int(aid[N - 1]) + 1
    rng = np.random.default_rng(20)
    for j in rng.choice(N, size=300, replace=False):   # walks re-derived from attempt ids
        r, on, oe = oq.attempt(int(aid[j]))
        assert r == oracle.HIT
        assert np.array_equal(nodes[off[j]:off[j + 1]], on) and np.array_equal(edges[off[j] - j:off[j + 1] - j - 1], oe)
    last = int(aid[N - 1])
    for first in [int(x) for x in rng.integers(0, last - 200_000, size=3)] + [0]:
        out, _ = oq.classify(first, 200_000)        # every attempt of the window
        want = first + np.nonzero(out == oracle.HIT)[0].astype(np.uint64)
        sel = (aid >= first) & (aid < first + 200_000)
        assert np.array_equal(aid[sel], want)


def test_c2_fullsize_counts_and_greedy(c2):
    d, res, ids, gains, off, nodes = (c2[k] for k in ("d", "res", "ids", "gains", "off", "nodes"))
    N = d["n_hsaw"]
    R = nodes[:off[N]]
    cnt = np.bincount(R, minlength=d["n"])
    top = cnt.max()
    assert gains[0] == top and ids[0] == int(np.nonzero(cnt == top)[0][0])
    assert np.all(np.diff(gains.astype(np.int64)) <= 0)
    walk_of = np.repeat(np.arange(N), np.diff(off[:N + 1]))
    covered = np.zeros(N, bool)
    covered[walk_of[np.isin(R, ids)]] = True
    assert int(gains.sum()) == int(covered.sum()) == res["cov_R"]
    assert res["spread_reduction_est"] == pytest.approx(d["n"] * res["cov_R"] / res["attempts"], rel=1e-12)
