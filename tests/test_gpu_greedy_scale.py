"""Greedy max-coverage (Alg. 4 / Alg. 7) against the oracle, pick by pick, at R-MAT 22 scale.

Two streams of N = 100,000 HSAWs on R-MAT scale 22 (4,194,304 nodes, 67,108,864 edges):
eSI with weighted-cascade weights and 4,000 sources (about 6.8 M walk edges, 6.4 M of
them distinct), and nSI with random LT weights and 20,000 sources.  k = 1,000 picks are
compared id by id and gain by gain with the oracle's greedy over the oracle's own stream,
on the cluster greedy with on-chip counts (the nSI stream; the eSI stream's 6.4 M
elements do not fit on chip), on the cluster greedy with counts in global memory (both;
each checked from its launch record to run on at least 8 CTAs with more than one element
group per CTA), and on the grid-wide fallback.  The cluster versions cover a pick either
by ownership (every CTA reads the pick's walks and takes down its own elements) or across
the cluster (each walk by one CTA, decrements sent to the owners); the variants force the
second form on every pick, and a threshold at the median pick's walk entries mixes both
in one run, each checked from the launch record's count of picks covered across.  The
oracle draws the stream on all host cores (consecutive attempt ranges joined in order)
and runs the greedy that keeps its gains, which the CPU tests hold equal to the
recounting greedy.
"""
import math
import os
import re

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hs = pytest.importorskip("paper_1702_05854_gb300")

N = 100_000
K = 1000
CASES = {
    "esi-wc-4000": dict(weights="wc", n_sources=4000, mode="edge"),
    "nsi-random-20000": dict(weights="random", n_sources=20000, mode="node"),
}
LOG = re.compile(r"k_greedy_(cluster|onchip) walks=(\d+) entries=(\d+) unique=(\d+) cluster=(\d+) (gshift|per)=(\d+) "
                 r"k=(\d+) picks=(\d+) spread=(\d+)")


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = CASES[request.param]
    d = synth.workload_rmat(22, c["weights"], c["n_sources"], K, c["mode"])
    omode = oracle.MODE_EDGE if c["mode"] == "edge" else oracle.MODE_NODE
    M = d["m"] if c["mode"] == "edge" else d["n"]
    og = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    st = oracle.Stream(oracle.Query(og, d["sources"], seed=synth.SEED_WALKS))
    st.extend_threads(N, threads=min(32, os.cpu_count() or 1))
    oids, ogains = st.greedy(omode, 0, N, M, K, kept_gains=True)
    W = st.export()
    el = W.elements(omode)[0]
    walks_of_pick = np.bincount(el, minlength=M)[oids]  # each pick's walk-list length
    mixed = int(np.median(walks_of_pick)) * math.ceil(el.shape[0] / N)
    g = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    q = hs.Query(sources=d["sources"], mode=hs.HSAW_EDGE if c["mode"] == "edge" else hs.HSAW_NODE, k=K, n_hsaw=N,
                 seed=synth.SEED_WALKS)
    return dict(g=g, q=q, oids=oids, ogains=ogains, attempts=int(W.aid[N - 1]) + 1,
                entries=int(el.shape[0]), esi=c["mode"] == "edge", mixed=mixed)


def _solve(case, capfd, monkeypatch, variant):
    monkeypatch.setenv("HSAW_LOG_LAUNCHES", "1")
    for v in ("HSAW_GREEDY_HEAVY", "HSAW_GREEDY", "HSAW_GREEDY_OWNED_MAX"):
        monkeypatch.delenv(v, raising=False)
    if variant == "all-elements":
        monkeypatch.setenv("HSAW_GREEDY_HEAVY", "0")
    if variant in ("cluster", "cluster-spread", "grid"):
        monkeypatch.setenv("HSAW_GREEDY", variant.split("-")[0])
    if variant.endswith("spread"):
        monkeypatch.setenv("HSAW_GREEDY_OWNED_MAX", "0")
    if variant == "mixed":
        monkeypatch.setenv("HSAW_GREEDY_OWNED_MAX", str(case["mixed"]))
    capfd.readouterr()
    ids, gains, r = hs.hsaw_solve(case["g"], case["q"])
    return ids, gains, r, capfd.readouterr().err


def _same_as_oracle(case, ids, gains, r):
    assert np.array_equal(gains, case["ogains"]), np.nonzero(gains != case["ogains"])[0][:5]
    assert np.array_equal(ids, case["oids"]), np.nonzero(ids != case["oids"])[0][:5]
    assert r["hits"] == N and r["attempts"] == case["attempts"]
    assert r["cov_R"] == int(case["ogains"].sum())
    assert case["ogains"][-1] > 0  # every pick is a real argmax, not a zero-gain fill


@pytest.mark.parametrize("variant", ["default", "cluster", "all-elements", "spread", "cluster-spread", "mixed"])
def test_cluster_greedy_matches_oracle_at_scale(case, capfd, monkeypatch, variant):
    """default: the elements that occur in two or more walks first, then (once every gain is
    below 2) all of them, each phase with on-chip counts when they fit the cluster;
    cluster: counts in global memory throughout;
    all-elements: no first phase (the eSI stream's 6.4 M elements then do not fit on chip);
    spread, cluster-spread: every pick covered across the cluster; mixed: both forms."""
    ids, gains, r, err = _solve(case, capfd, monkeypatch, variant)
    runs = LOG.findall(err)
    assert runs, err[-2000:]
    picks = spread = 0
    for kind, walks, entries, unique, csize, what, size, k, p, sp in runs:
        walks, entries, unique, csize, size = (int(x) for x in (walks, entries, unique, csize, size))
        assert walks == N and entries == case["entries"]
        if kind == "onchip":
            groups_per_cta = math.ceil(size / 32)
        else:
            groups_per_cta = math.ceil(math.ceil(unique / (1 << size)) / csize)
        assert csize >= 8 and groups_per_cta > 1  # the multi-CTA paths ran
        if variant.startswith("cluster"):
            assert kind == "cluster"
        # a run covers each pick but its last (and that one too when it stops early)
        assert int(sp) <= int(p)
        if variant.endswith("spread"):
            assert int(sp) >= int(p) - 1
        picks += int(p)
        spread += int(sp)
    assert picks == K
    if variant == "mixed":
        assert 0 < spread < picks - len(runs), (spread, picks)
    if variant == "all-elements":
        assert len(runs) == 1 and runs[0][0] == ("cluster" if case["esi"] else "onchip")
    _same_as_oracle(case, ids, gains, r)


def test_grid_greedy_matches_oracle_at_scale(case, capfd, monkeypatch):
    ids, gains, r, err = _solve(case, capfd, monkeypatch, "grid")
    assert "k_greedy_cluster" not in err and "k_greedy_onchip" not in err
    _same_as_oracle(case, ids, gains, r)
