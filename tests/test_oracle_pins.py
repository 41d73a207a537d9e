"""Pins of the CPU oracle against things other than itself (no GPU).

Each test names what fixes the expected value: a published known-answer vector, a closed
form of the LT live-edge model (Sec. 2.1), brute-force enumeration of live-edge worlds,
the walk-probability equation (Eq. "compute_path_inf"), the HSAW definition's invariants
(Def. "self_walk"), exact integer binomials, or brute-force optimal max-coverage.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tinygraphs import ONE, fx, random_tiny, world_count

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Random123 / SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def test_philox_lanes_uniform():
    """Chi-square uniformity of the 4 output lanes over 4096 counters (16 bins each)."""
    outs = np.array([oracle.philox4x32_10([i, 7, 3, 0], [4, 0]) for i in range(4096)], np.uint64)
    for lane in range(4):
        h = np.bincount((outs[:, lane] >> 28).astype(np.int64), minlength=16)
        chi2 = ((h - 256.0) ** 2 / 256.0).sum()
        assert chi2 < 50.0  # 15 dof: P(chi2 > 50) ~ 1e-5


# ----------------------------------------------------------------------------- graph build
def test_graph_build_stable_and_thresholds():
    n, src, dst, w = random_tiny(3, n=9, m=40)
    g = oracle.Graph(n, src, dst, w)
    rp, s, d, thr, ii = g.arrays()
    # stable sort by destination: input indices increase within each node
    assert np.all(np.diff(d) >= 0)
    for v in range(n):
        seg = ii[rp[v]:rp[v + 1]]
        assert np.all(np.diff(seg) > 0)
        # thresholds are running sums of the node's weights, exactly
        acc = np.cumsum(w[seg].astype(np.uint64))
        assert np.array_equal(thr[rp[v]:rp[v + 1]].astype(np.uint64), acc)
    assert np.array_equal(s, src[ii]) and np.array_equal(d, dst[ii])


def test_graph_build_rejects_overweight_and_range():
    src = np.array([0, 1], np.int32)
    dst = np.array([2, 2], np.int32)
    with pytest.raises(ValueError):
        oracle.Graph(3, src, dst, np.array([0x80000000, 0x80000000], np.uint32))  # sum = 2^32 > 2^32-1
    oracle.Graph(3, src, dst, np.array([0x80000000, 0x7FFFFFFF], np.uint32))     # sum = 2^32-1 is fine
    with pytest.raises(ValueError):
        oracle.Graph(2, src, dst, np.array([1, 1], np.uint32))


def test_select_in_edge_boundaries():
    """Inverse-CDF selection: in-edge j is live exactly for r in [thr[j-1], thr[j]), so the
    number of draws choosing it is w_fixed[j] (probability w / 2^32, Sec. 2.1)."""
    w = np.array([5, 0, 7, 0xFFFFFFF0 - 12], np.uint32)   # sum 0xFFFFFFF0 < 2^32 - 1
    g = oracle.Graph(2, np.array([1, 0, 1, 0], np.int32), np.array([0, 0, 0, 0], np.int32), w)
    assert [g.select_in_edge(0, r) for r in (0, 4)] == [0, 0]
    assert g.select_in_edge(0, 5) == 2            # the zero-weight edge 1 is never live
    assert g.select_in_edge(0, 11) == 2 and g.select_in_edge(0, 12) == 3
    assert g.select_in_edge(0, 0xFFFFFFEF) == 3
    assert g.select_in_edge(0, 0xFFFFFFF0) == -1 and g.select_in_edge(0, 0xFFFFFFFF) == -1
    assert g.select_in_edge(1, 0) == -1           # no in-edges


def test_source_coin_boundaries():
    """Source coin: probability p32 / 2^32 (x1 < p32), p32 = 0xFFFFFFFF certain."""
    assert not oracle.source_coin(0, 0) and not oracle.source_coin(0xFFFFFFFF, 0)
    assert oracle.source_coin(9, 10) and not oracle.source_coin(10, 10)
    assert oracle.source_coin(0xFFFFFFFF, 0xFFFFFFFF) and oracle.source_coin(0, 0xFFFFFFFF)
    assert not oracle.source_coin(0xFFFFFFFE, 0xFFFFFFFE)


def test_attempt_walks_are_self_avoiding_chains():
    """Every attempt, hit or miss, walks a self-avoiding chain of live in-edges (the
    backward chain of one live-edge world, Sec. 3.1 "Self-avoiding")."""
    for gseed in range(6):
        n, src, dst, w = random_tiny(500 + gseed, n=6, m=14)
        g = oracle.Graph(n, src, dst, w)
        rp, s, d, thr, ii = g.arrays()
        q = oracle.Query(g, np.array([gseed % n], np.int32), seed=gseed)
        outs = set()
        for a in range(3000):
            r, nodes, edges = q.attempt(a)
            outs.add(r)
            assert len(set(nodes.tolist())) == len(nodes)
            for i, e in enumerate(edges):
                assert d[e] == nodes[i] and s[e] == nodes[i + 1]
            if r == oracle.MISS_CYCLE:  # the last choice closed a cycle
                pass
        assert oracle.STEP_CAP not in outs


# ----------------------------------------------------------------------------- brute force closed forms
def test_bruteforce_closed_forms():
    """Live-edge model closed forms (Sec. 2.1): edge, chain, cycle, independent suspects, removal."""
    w1, w2, w3 = fx(0.3), fx(0.6), fx(0.45)
    p = lambda x: x / 4294967296.0
    # single edge s(0) -> v(1): I = 1 + w
    g = oracle.Graph(2, np.array([0], np.int32), np.array([1], np.int32), np.array([w1], np.uint32))
    assert oracle.bruteforce_spread(g, [0]) == pytest.approx(1 + p(w1), rel=1e-12)
    assert oracle.bruteforce_spread(g, [0], edge_removed=[1]) == pytest.approx(1.0, rel=1e-12)
    # chain 0 -> 1 -> 2: I = 1 + w1 + w1 w2
    g = oracle.Graph(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.array([w1, w2], np.uint32))
    assert oracle.bruteforce_spread(g, [0]) == pytest.approx(1 + p(w1) + p(w1) * p(w2), rel=1e-12)
    # removing node 1 leaves only the seed
    assert oracle.bruteforce_spread(g, [0], node_removed=[0, 1, 0]) == pytest.approx(1.0, rel=1e-12)
    # cycle 0 -> 1 -> 2 -> 0 with seed 0: the edge into the seed is irrelevant
    g = oracle.Graph(3, np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32),
                     np.array([w1, w2, w3], np.uint32))
    assert oracle.bruteforce_spread(g, [0]) == pytest.approx(1 + p(w1) + p(w1) * p(w2), rel=1e-12)
    # two isolated suspects with probabilities: I = p1 + p2 (Eq. "prob_src_set")
    g = oracle.Graph(3, np.array([0], np.int32), np.array([0], np.int32), np.array([0], np.uint32))
    pa, pb = fx(0.25), fx(0.7)
    assert oracle.bruteforce_spread(g, [1, 2], p_fixed=[pa, pb]) == pytest.approx(p(pa) + p(pb), rel=1e-12)
    # v with two in-edges from seeds a, b (weights wa + wb <= 1): P(v infected) = wa + wb
    g = oracle.Graph(3, np.array([0, 1], np.int32), np.array([2, 2], np.int32), np.array([w1, w2], np.uint32))
    assert oracle.bruteforce_spread(g, [0, 1]) == pytest.approx(2 + p(w1) + p(w2), rel=1e-12)


# ----------------------------------------------------------------------------- sampler vs brute force
def _se(q, A, n):
    return n * math.sqrt(max(q * (1 - q), 1e-12) / A)


def _estimate(g, sources, A, seed, **kw):
    q = oracle.Query(g, sources, seed=seed, **kw)
    out, _ = q.classify(0, A)
    assert not np.any(out == oracle.STEP_CAP)
    return g.n * float((out == oracle.HIT).sum()) / A


@pytest.mark.parametrize("gseed", list(range(12)))
def test_sampler_spread_matches_bruteforce(gseed):
    """n * hits / attempts estimates I_G(V_I) (Thm. "rr_edge" with T = E): within 4 SE."""
    n, src, dst, w = random_tiny(100 + gseed, n=7, m=13)
    if world_count(n, dst) > 200_000:
        pytest.skip("too many worlds")
    g = oracle.Graph(n, src, dst, w)
    rng = np.random.default_rng(gseed)
    S = np.sort(rng.choice(n, size=1 + gseed % 3, replace=False)).astype(np.int32)
    p = None
    if gseed % 2 == 1:
        p = np.array([fx(x) for x in rng.uniform(0.2, 1.0, S.size)], np.uint32)
    exact = oracle.bruteforce_spread(g, S, p_fixed=p)
    A = 200_000
    est = _estimate(g, S, A, seed=11 + gseed, p_fixed=p)
    assert abs(est - exact) <= 4 * _se(exact / n, A, n) + 1e-9, (est, exact)


@pytest.mark.parametrize("gseed", list(range(10)))
def test_reduction_estimate_matches_bruteforce(gseed):
    """D(T) = I_G(V_I) Pr[T interdicts h] (Thms. "rr_edge" / "rr_node"): n * Cov(T) / attempts
    estimates I_G - I_G' for a fixed edge set (even seeds) or node set (odd seeds)."""
    n, src, dst, w = random_tiny(200 + gseed, n=7, m=12)
    g = oracle.Graph(n, src, dst, w)
    rng = np.random.default_rng(50 + gseed)
    S = np.sort(rng.choice(n, size=2, replace=False)).astype(np.int32)
    node_mode = gseed % 2 == 1
    M = n if node_mode else g.m
    T = np.sort(rng.choice(M, size=2, replace=False))
    mask = np.zeros(M, np.uint8)
    mask[T] = 1
    if node_mode:
        exact = oracle.bruteforce_spread(g, S) - oracle.bruteforce_spread(g, S, node_removed=mask)
    else:
        exact = oracle.bruteforce_spread(g, S) - oracle.bruteforce_spread(g, S, edge_removed=mask)
    q = oracle.Query(g, S, seed=77 + gseed)
    st = oracle.Stream(q).extend(1 << 62, max_attempts=150_000)
    A = st.attempts
    cov = st.coverage(oracle.MODE_NODE if node_mode else oracle.MODE_EDGE, 0, len(st), M, T)
    est = n * cov / A
    assert abs(est - exact) <= 4 * _se(exact / n, A, n) + 1e-9, (est, exact)
    # the residual-graph estimate agrees as well (walks respect the removed set)
    kw = dict(node_removed=mask) if node_mode else dict(edge_removed=mask)
    resid = _estimate(g, S, 150_000, seed=91 + gseed, **kw)
    exact_resid = oracle.bruteforce_spread(g, S, **kw)
    assert abs(resid - exact_resid) <= 4 * _se(exact_resid / n, 150_000, n) + 1e-9


def test_walk_probability_equation():
    """Frequency of each distinct HSAW among attempts = Pr[h] / n, with Pr[h] from
    Eq. "compute_path_inf" (p(v_l) * prod (1 - p(u)) over earlier suspects * prod w)."""
    n, src, dst, w = random_tiny(7, n=6, m=11)
    g = oracle.Graph(n, src, dst, w)
    rp, s, d, thr, ii = g.arrays()
    wcsr = w[ii].astype(np.float64) / 4294967296.0
    S = np.array([1, 4], np.int32)
    p32 = np.array([fx(0.6), ONE], np.uint32)
    pmap = {1: p32[0] / 4294967296.0, 4: 1.0}
    q = oracle.Query(g, S, p_fixed=p32, seed=5)
    A = 300_000
    counts = {}
    st = oracle.Stream(q).extend(1 << 62, max_attempts=A)
    W = st.export()
    for j in range(len(W)):
        nodes, edges = W.walk(j)
        key = tuple(int(e) for e in edges) + (int(nodes[0]),)
        counts[key] = counts.get(key, 0) + 1
    # walk nodes/edges consistency + equation
    for key, c in counts.items():
        edges, start = key[:-1], key[-1]
        nodes = [start] + [int(s[e]) for e in edges]
        pr = 1.0
        for e in edges:
            pr *= wcsr[e]
        last = nodes[-1]
        pr *= pmap[last]
        for u in nodes[:-1]:
            if u in pmap:
                pr *= (1.0 - pmap[u])
        expect = pr / n
        freq = c / A
        se = math.sqrt(expect * (1 - expect) / A)
        assert abs(freq - expect) <= 4 * se + 1e-9, (key, freq, expect)
    assert len(counts) > 3


# ----------------------------------------------------------------------------- invariants on the C1 shape
@pytest.fixture(scope="module")
def c1_small():
    d = synth.workload_c1()
    g = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    q = oracle.Query(g, d["sources"], seed=synth.SEED_WALKS)
    st = oracle.Stream(q).extend(3000)
    return d, g, st


def test_hsaw_invariants(c1_small):
    """Def. "self_walk": consecutive nodes are joined by the walked edge (v_{i+1}, v_i),
    nodes are distinct, the last node is in S, no earlier node is in S (p = 1)."""
    d, g, st = c1_small
    rp, s, dd, thr, ii = g.arrays()
    W = st.export()
    Sset = set(int(x) for x in d["sources"])
    assert np.all(np.diff(W.aid.astype(np.int64)) > 0)
    for j in range(len(W)):
        nodes, edges = W.walk(j)
        assert len(set(nodes.tolist())) == len(nodes)
        assert int(nodes[-1]) in Sset
        assert not any(int(x) in Sset for x in nodes[:-1])
        for i, e in enumerate(edges):
            assert dd[e] == nodes[i] and s[e] == nodes[i + 1]


def test_histogram_recount(c1_small):
    d, g, st = c1_small
    W = st.export()
    for mode, M in ((oracle.MODE_EDGE, g.m), (oracle.MODE_NODE, g.n)):
        els, off = W.elements(mode)
        cnt = st.histogram(mode, 0, len(W), M)
        assert np.array_equal(cnt, np.bincount(els, minlength=M).astype(np.uint32))
        assert int(cnt.sum()) == int(off[-1] - off[0])
        part = st.histogram(mode, 100, 500, M)
        assert np.array_equal(part, np.bincount(els[off[100]:off[600]], minlength=M).astype(np.uint32))


# ----------------------------------------------------------------------------- greedy
def _coverage(sets, T):
    T = set(T)
    return sum(1 for s in sets if T & set(s))


@pytest.mark.parametrize("gseed", list(range(8)))
def test_greedy_against_bruteforce_max_coverage(gseed):
    """Greedy (Alg. 4 / Alg. 7) reaches >= (1 - 1/e) OPT of max-coverage (brute force over
    all k-subsets); k = 1 is the exact optimum with the smallest-id tie rule."""
    n, src, dst, w = random_tiny(300 + gseed, n=8, m=14)
    g = oracle.Graph(n, src, dst, w)
    q = oracle.Query(g, np.array([gseed % n], np.int32), seed=3 + gseed)
    st = oracle.Stream(q).extend(60)
    W = st.export()
    for mode, M in ((oracle.MODE_NODE, n), (oracle.MODE_EDGE, g.m)):
        els, off = W.elements(mode)
        sets = [els[off[j]:off[j + 1]].tolist() for j in range(len(W))]
        for k in (1, 2, 3):
            if k > M:
                continue
            ids, gains = st.greedy(mode, 0, len(W), M, k)
            assert len(set(ids.tolist())) == k
            assert np.all(np.diff(gains.astype(np.int64)) <= 0)           # submodular: gains fall
            assert int(gains.sum()) == _coverage(sets, ids.tolist())       # gains add up to Cov
            opt = max(_coverage(sets, c) for c in itertools.combinations(range(M), k))
            assert gains.sum() >= (1 - 1 / math.e) * opt - 1e-9
            if k == 1:
                cnt = np.bincount(els, minlength=M)
                assert ids[0] == int(np.argmax(cnt)) and gains[0] == cnt.max()


def test_greedy_zero_gain_and_candidates():
    """Zero-gain picks take the smallest unpicked candidate; candidate masks are honoured."""
    # chain 0 -> 1 -> 2 with certain edges; S = {0}: every attempt from 1 or 2 hits.
    g = oracle.Graph(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.array([ONE, ONE], np.uint32))
    q = oracle.Query(g, np.array([0], np.int32), seed=1)
    st = oracle.Stream(q).extend(50)
    W = st.export()
    els, off = W.elements(oracle.MODE_NODE)
    cnt = np.bincount(els, minlength=3)
    ids, gains = st.greedy(oracle.MODE_NODE, 0, len(W), 3, 3)
    assert ids[0] == 0 and gains[0] == len(W)           # the source is on every walk
    assert list(ids[1:]) == [1, 2] and list(gains[1:]) == [0, 0]
    mask = np.array([0, 1, 1], np.uint8)
    ids, gains = st.greedy(oracle.MODE_NODE, 0, len(W), 3, 2, cand_mask=mask)
    assert ids[0] == 1 and gains[0] == cnt[1]
    assert ids[1] == 2 and gains[1] == 0   # every walk through 2 also passes 1
    with pytest.raises(ValueError):
        st.greedy(oracle.MODE_NODE, 0, len(W), 3, 3, cand_mask=mask)  # k > |C|


# ----------------------------------------------------------------------------- stopping rule
def test_log_binomial_exact():
    for M, k in ((1000, 10), (131072, 10), (1 << 20, 100), (5000, 2500)):
        exact = math.log(math.comb(M, k))
        assert oracle.stop_constants(M, k, 0.1, 1e-3)["lnC"] == pytest.approx(exact, rel=1e-10)


def test_stop_constants_structure():
    """t_max doubles Upsilon past 2 N_max (Lemma "tmax"); Lambda_1 = 1 + (1 + eps) Lambda;
    values agree with an independent FP64 evaluation of the stopping-rule constants."""
    cases = [  # (M, k, eps, delta, N_max, Upsilon, t_max, Lambda, Lambda1), independent evaluation
        (1 << 30, 1000, 0.1, 1.0 / (1 << 26), 8.809e12, 3951.6, 33, 4674.17, 5142.59),
        (1 << 20, 100, 0.1, 1.0 / (1 << 20), 5.993e9, 3092.1, 22, 3730.87, 4104.96),
        (131072, 10, 0.1, 1.0 / 16384, 8.242e8, 2232.6, 20, 2851.67, 3137.84),
    ]
    for M, k, eps, delta, nmax, ups, tmax, lam, lam1 in cases:
        c = oracle.stop_constants(M, k, eps, delta)
        assert c["N_max"] == pytest.approx(nmax, rel=1e-3)
        assert c["Upsilon"] == pytest.approx(ups, rel=1e-4)
        assert c["t_max"] == tmax
        assert c["Lambda"] == pytest.approx(lam, rel=1e-5)
        assert c["Lambda1"] == pytest.approx(lam1, rel=1e-5)
        r = 2 * c["N_max"] / c["Upsilon"]
        assert 2 ** (c["t_max"] - 1) < r <= 2 ** c["t_max"]
        assert c["Lambda1"] == pytest.approx(1 + (1 + eps) * c["Lambda"], rel=1e-14)


def test_check_behaviour():
    """Check (Alg. 5): no bound below Lambda_1; the bound shrinks as the verification
    coverage grows at a fixed in-sample / out-of-sample ratio; an overfit in-sample
    coverage (c >> c') fails."""
    lam1 = 3137.84
    ok, et = oracle.check(3000, 3000, 10000, 1, 0.1, lam1)
    assert not ok and math.isnan(et)
    prev = math.inf
    for t in range(1, 12):
        size = 2851 * 2 ** (t - 1)
        cp = 0.6 * size
        ok, et = oracle.check(cp, cp, size, t, 0.1, lam1)
        if cp >= lam1:
            assert et < prev
            prev = et
    assert ok
    ok, et = oracle.check(2 * 0.6 * 2851 * 1024, 0.6 * 2851 * 1024, 2851 * 1024, 11, 0.1, lam1)
    assert not ok and et > 0.1
    # with unbiased in-sample coverage the bound vanishes as the samples double without
    # end (eps_2, eps_3 are Chernoff deviations of |R'_t| = Lambda 2^(t-1) samples)
    size = 2851 * 2 ** 39
    ok, et = oracle.check(0.6 * size, 0.6 * size, size, 40, 0.1, lam1)
    assert ok and et < 1e-3
    # the bound never drops below the in-sample bias term eps_1 (1 - 1/e - eps)
    ok, et = oracle.check(1.2 * 0.6 * size, 0.6 * size, size, 40, 0.1, lam1)
    assert et >= 0.2 * (1 - 1 / math.e - 0.1)


# Check (Alg. 5) evaluated by hand.  With |R'_t| = L 2^(t-1) (L = ceil(Lambda)) the
# quantity under eps_2's root is rho = |R'_t| (1 + eps) / (2^(t-1) c'), so
#   eps_2 = eps sqrt(rho),   eps_3 = eps sqrt(rho (1 - 1/e - eps) / (1 + eps/3)),
#   eps_t = ((c / c') (1 + eps_2) - 1)(1 - 1/e - eps) + (1 - 1/e) eps_3,
# using eps_1 + eps_2 + eps_1 eps_2 = (1 + eps_1)(1 + eps_2) - 1 and 1 + eps_1 = c / c'
# (the factorisation the paper's proof of Lemma "e2e" part (C) uses).  The numbers below
# were worked out digit by digit (25-digit arithmetic) and are literals here.
CHECK_CASES = [
    # eps, t, |R'_t|, c', c, expected eps_t
    # (a) t = 3, L = 1000: rho = 4000 * 1.5 / (4 * 1500) = 1, eps_2 = 0.5, eps_1 = 1800/1500 - 1 = 0.2,
    #     gap = 1 - 1/e - 0.5 = 0.1321205588285577, eps_3 = 0.5 sqrt(gap / (7/6))
    #     = 0.5 sqrt(0.1132461932816209) = 0.5 * 0.3365207174627156 = 0.1682603587313578,
    #     eps_t = 1.2 * 1.5 - 1 = 0.8 times gap = 0.1056964470628461
    #           + (1 - 1/e) eps_3 = 0.6321205588285577 * 0.1682603587313578 = 0.1063608319899595
    #           = 0.2120572790528056
    (0.5, 3, 4000, 1500, 1800, 0.2120572790528056),
    # (b) t = 1, L = 5000: rho = 5000 * 1.1 / 4400 = 1.25, eps_2 = 0.1 sqrt(1.25) = 0.1118033988749895,
    #     eps_1 = 4840/4400 - 1 = 0.1, gap = 0.5321205588285577,
    #     eps_3 = 0.1 sqrt(1.25 gap / (31/30)) = 0.1 sqrt(0.6436942243893843) = 0.08023055679660863,
    #     eps_t = (0.1 + 1.1 * 0.1118033988749895) gap = 0.1186542316799765
    #           + 0.6321205588285577 * 0.08023055679660863 = 0.05071538439739858
    #           = 0.1693696160773750
    (0.1, 1, 5000, 4400, 4840, 0.1693696160773750),
    # (c) t = 5, L = 4675 (C3's Lambda rounded up): |R'_5| = 4675 * 16 = 74800, c' = 41140,
    #     rho = 74800 * 1.1 / (16 * 41140) = 0.125, eps_2 = 0.1 sqrt(0.125) = 0.03535533905932738,
    #     eps_1 = 44880/41140 - 1 = 1/11, eps_3 = 0.1 sqrt(0.125 gap / (31/30))
    #     = 0.1 sqrt(0.06436942243893843) = 0.02537112974207858,
    #     eps_t = (1/11 + (12/11) 0.03535533905932738) gap = 0.06889819928749333
    #           + 0.6321205588285577 * 0.02537112974207858 = 0.01603761271067455
    #           = 0.08493581199816789
    (0.1, 5, 74800, 41140, 44880, 0.08493581199816789),
]


@pytest.mark.parametrize("eps,t,size,cp,c,want", CHECK_CASES)
def test_check_hand_evaluated(eps, t, size, cp, c, want):
    """eps_t of Alg. 5 equals hand-evaluated values; the call passes iff eps_t <= eps.
    A dropped eps_1 eps_2 term moves (a) by 0.013, (c) by 0.0017; 2^t in place of 2^(t-1)
    moves eps_2 by a factor sqrt(2); swapping (1 - 1/e) and (1 - 1/e - eps) moves (a) by
    0.06.  Each is far outside the 1e-12 tolerance."""
    ok, et = oracle.check(c, cp, size, t, eps, 1.0)
    assert et == pytest.approx(want, rel=1e-12, abs=0)
    assert ok == (want <= eps)


@pytest.mark.parametrize("eps,t,eps1", [(0.1, 2, 0.0), (0.1, 6, 0.05), (0.2, 3, 0.1), (0.3, 4, 0.2)])
def test_check_threshold_closed_form(eps, t, eps1):
    """Solving eps_t = eps for the verification coverage c' at a fixed ratio c / c' = 1 + eps_1
    (a closed form, not the oracle's expression): with s = sqrt(L (1 + eps) / c'),
        eps_t = eps_1 g + eps s [(1 + eps_1) g + (1 - 1/e) sqrt(g / (1 + eps/3))],  g = 1 - 1/e - eps,
    so Check passes exactly when c' >= c*' = L (1 + eps) / s*^2 with
        s* = (eps - eps_1 g) / (eps [(1 + eps_1) g + (1 - 1/e) sqrt(g / (1 + eps/3))])."""
    L = 4675
    size = L * 2 ** (t - 1)
    g = 1 - 1 / math.e - eps
    s_star = (eps - eps1 * g) / (eps * ((1 + eps1) * g + (1 - 1 / math.e) * math.sqrt(g / (1 + eps / 3))))
    cp_star = L * (1 + eps) / s_star ** 2
    assert cp_star < size  # a coverage the round can reach
    for f, expect in ((1 + 1e-9, True), (1 - 1e-9, False)):
        cp = cp_star * f
        ok, et = oracle.check((1 + eps1) * cp, cp, size, t, eps, 1.0)
        assert ok == expect, (f, et)
    ok, et = oracle.check((1 + eps1) * cp_star, cp_star, size, t, eps, 1.0)
    assert et == pytest.approx(eps, rel=1e-12)


# ----------------------------------------------------------------------------- end-to-end quality
@pytest.mark.parametrize("gseed", list(range(6)))
def test_solve_quality_against_bruteforce(gseed):
    """Thm. "app": D(T_hat) >= (1 - 1/e - eps) OPT_k (brute force over every k-set)."""
    n, src, dst, w = random_tiny(400 + gseed, n=7, m=12)
    g = oracle.Graph(n, src, dst, w)
    S = np.array([gseed % n], np.int32)
    node_mode = gseed % 2 == 1
    mode = oracle.MODE_NODE if node_mode else oracle.MODE_EDGE
    M = n if node_mode else g.m
    k = 2
    q = oracle.Query(g, S, seed=9 + gseed)
    ids, gains, res = oracle.solve(q, mode, k, stop_rule=True, eps=0.2, delta=0.1)
    base = oracle.bruteforce_spread(g, S)

    def D(T):
        mask = np.zeros(M, np.uint8)
        mask[list(T)] = 1
        kw = dict(node_removed=mask) if node_mode else dict(edge_removed=mask)
        return base - oracle.bruteforce_spread(g, S, **kw)

    opt = max(D(T) for T in itertools.combinations(range(M), k))
    assert D(ids.tolist()) >= (1 - 1 / math.e - 0.2) * opt - 1e-9
    assert res["hits"] == 2 * res["hits_Rprime"] and res["rounds_t"] >= 1
    assert res["spread_base_est"] == pytest.approx(n * res["hits"] / res["attempts"], rel=1e-15)


# ----------------------------------------------------------------------------- harness
@pytest.mark.parametrize("want,chunk", [(3000, 4096), (2500, 1000), (1, 700)])
def test_threaded_stream_equals_sequential(want, chunk):
    """The threaded stream harness (consecutive attempt ranges joined in order) yields
    exactly the sequential stream: same walks, same attempt count, same next attempt."""
    d = synth.workload_c1()
    g = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    q = oracle.Query(g, d["sources"], seed=4)
    a = oracle.Stream(q, first_aid=777).extend(want)
    b = oracle.Stream(q, first_aid=777).extend_threads(want, threads=3, chunk=chunk)
    A, B = a.export(), b.export()
    assert len(A) == len(B) == want
    for x, y in ((A.aid, B.aid), (A.node_off, B.node_off), (A.nodes, B.nodes), (A.edges, B.edges)):
        assert np.array_equal(x, y)
    assert a.attempts == b.attempts and a._next == b._next == int(A.aid[-1]) + 1
    # both continue identically
    a.extend(want + 500)
    b.extend_threads(want + 500, threads=2, chunk=chunk)
    assert np.array_equal(a.export().aid, b.export().aid) and a.attempts == b.attempts


def test_greedy_kept_gains_equals_recount():
    """The greedy that keeps and decrements gains returns exactly the picks and gains of the
    greedy that recounts them every round (Alg. 4 / 7, same tie and zero-gain rules), on
    the C1 stream and an R-MAT 14 stream, both modes, with candidate masks and with k
    large enough to reach zero-gain picks."""
    cases = []
    d = synth.workload_c1()
    g = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    cases.append((g, oracle.Stream(oracle.Query(g, d["sources"], seed=4)).extend(4000)))
    r = synth.workload_rmat(14, "random", 50, 20, "node")
    gr = oracle.Graph(r["n"], r["src"], r["dst"], r["w"])
    cases.append((gr, oracle.Stream(oracle.Query(gr, r["sources"], seed=4)).extend(3000)))
    for g, st in cases:
        W = st.export()
        for mode in (oracle.MODE_EDGE, oracle.MODE_NODE):
            M = g.m if mode == oracle.MODE_EDGE else g.n
            touched = np.unique(W.elements(mode)[0]).size
            for k, first, count in ((1, 0, len(W)), (50, 100, len(W) - 300), (min(M, touched + 20), 0, len(W))):
                a = st.greedy(mode, first, count, M, k)
                b = st.greedy(mode, first, count, M, k, kept_gains=True)
                assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
            cm = (np.arange(M) % 3 != 1).astype(np.uint8)
            a = st.greedy(mode, 0, len(W), M, 40, cand_mask=cm)
            b = st.greedy(mode, 0, len(W), M, 40, cand_mask=cm, kept_gains=True)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with pytest.raises(ValueError):
        cases[0][1].greedy(oracle.MODE_NODE, 0, 10, 3, 4, kept_gains=True)  # k > |C|
