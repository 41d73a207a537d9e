"""Benchmark: HSAWs/s of the eSI billion-edge solve on one GB300 (or N independent replicas).

Workload (default): R-MAT scale 26 (67,108,864 nodes, 1,073,741,824 edges, a,b,c =
0.57, 0.19, 0.19), weighted-cascade LT weights in uint32 fixed point, |S| = 1,000 random
sources, k = 1,000, the sample-doubling stopping rule with eps = 0.1, delta = 1/n.  A step
is one full solve (sampling, ordered compaction, counting, inverted index, greedy,
out-of-sample coverage, Check) on the resident graph; value = HSAWs used by the solves
(|R_t| + |R'_t|) / device time.  The graph (9.6 GB on the device) is larger than L2, so
no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hsaw|reference]

Under torchrun with N ranks each rank solves its own replica (its own walk seed);
value = HSAWs of all ranks / the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "HSAWs/s at 1B edges (eSI stop-rule solve, R-MAT scale 26)"
METRIC_OTHER = {"c2": "HSAWs/s (nSI R-MAT 20 random LT, N = 10 M)", "c1": "HSAWs/s (eSI Chung-Lu 16 K, N = 200 K)"}
UNIT = "HSAW/s"
BYTES_PER_STEP = 96  # three random 32-byte sectors per live-edge draw: node record, threshold, tail node
# DRAM bytes (read + write) per live-edge draw of the sampler kernel from an ncu capture,
# keyed by (hash of the kernel's source, workload).  A workload without a capture of the
# current kernel reports traffic = null.
NCU_TRAFFIC = {("783e77c95bea", "rmat22-wc-eSI"): 122.9,   # profiles/k_sample_rmat22_dram.md
               ("783e77c95bea", "rmat26-wc-eSI"): 122.9}   # the scale-22 figure, scaled by draws


def sampler_hash():
    """Hash of k_sample's own source text and the device helpers it calls (Philox, draws,
    edge pick, checkpoints in common.cuh)."""
    csrc = os.path.join(ROOT, "paper_1702_05854_gb300", "csrc")
    src = open(os.path.join(csrc, "sample.cu")).read()
    i = src.index("template <bool HAS_P, bool HAS_REM>\n__global__ void __launch_bounds__(256, 6) k_sample")
    j = src.index("\n}\n", i)
    common = open(os.path.join(csrc, "common.cuh")).read()
    a = common.index("// ------------------------------------------------------------------ Philox4x32-10")
    b = common.index("// ------------------------------------------------------------------ primitives")
    h = hashlib.sha1()
    h.update(src[i:j].encode())
    h.update(common[a:b].encode())
    return h.hexdigest()[:12]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def reduce_over_ranks(dist, torch, device, elapsed, hits):
    """Whole-job figures of N replicas: the slowest rank's time and the HSAWs of all ranks."""
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    h = torch.tensor([float(hits)], dtype=torch.float64, device=device)
    dist.all_reduce(h)
    return float(t.item()), float(h.item())


def make_workload(scale, which="c3"):
    """c3: the billion-edge eSI stop-rule solve (default); c2: the nSI R-MAT 20 random-LT
    solve with N = 10 M HSAWs; c1: the eSI Chung-Lu 16 K solve with N = 200 K."""
    t0 = time.time()
    if which == "c2":
        d = synth.workload_c2()
    elif which == "c1":
        d = synth.workload_c1()
    else:
        d = synth.workload_c3(scale)
    d["gen_s"] = time.time() - t0
    return d


def query_for(hs, d, seed):
    mode = hs.HSAW_EDGE if d["mode"] == "edge" else hs.HSAW_NODE
    if "n_hsaw" in d:
        return hs.Query(sources=d["sources"], mode=mode, k=d["k"], n_hsaw=d["n_hsaw"], seed=seed)
    return hs.Query(sources=d["sources"], mode=mode, k=d["k"], sampling=hs.HSAW_STOP_RULE, eps=d["eps"], seed=seed)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(d, seed, seconds):
    """The oracle as it stands on a bounded sample of the same workload: on every host core
    (consecutive attempt ranges, one per thread, joined in attempt order) and on one core
    (the paper's single-core convention)."""
    import oracle
    t0 = time.time()
    og = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    build_s = time.time() - t0
    q = oracle.Query(og, d["sources"], seed=seed)
    cal = oracle.Stream(q)
    t0 = time.time()
    cal.extend(1 << 62, max_attempts=20_000)
    rate = 20_000 / max(time.time() - t0, 1e-6)
    attempts = max(20_000, int(rate * seconds / 2))
    st = oracle.Stream(q)
    t0 = time.time()
    st.extend(1 << 62, max_attempts=attempts)
    dt1 = time.time() - t0
    one = {"value": len(st) / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"first {attempts} attempts of the query stream ({len(st)} HSAWs, {dt1:.1f} s)"}
    cores = host_cores()
    chunk = max(1024, attempts // 4)
    attempts_all = chunk * cores * 4
    st = oracle.Stream(q)
    t0 = time.time()
    st.extend_threads(1 << 62, threads=cores, max_attempts=attempts_all, chunk=chunk)
    dt = time.time() - t0
    return {"value": len(st) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {attempts_all} attempts of the same query stream on {cores} threads "
                      f"({len(st)} HSAWs, {dt:.1f} s; oracle graph build {build_s:.0f} s untimed)",
            "single_core": one}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, as it stands, timed on every host core over bounded
    samples of the same workload (each step: the next attempts of the query stream)."""
    if rank != 0:
        return
    import oracle
    d = make_workload(args.scale, args.workload)
    og = oracle.Graph(d["n"], d["src"], d["dst"], d["w"])
    q = oracle.Query(og, d["sources"], seed=synth.SEED_WALKS)
    cores = host_cores()
    chunk = max(1024, args.ref_attempts // 4)
    per_step = chunk * cores * 4
    st = oracle.Stream(q)
    for _ in range(args.warmup):
        st.extend_threads(1 << 62, threads=cores, max_attempts=chunk * cores, chunk=chunk)
    hits0 = len(st)
    t0 = time.time()
    for _ in range(args.steps):
        st.extend_threads(1 << 62, threads=cores, max_attempts=per_step, chunk=chunk)
    dt = time.time() - t0
    v = (len(st) - hits0) / dt
    line = {"impl": "reference", "metric": METRIC_OTHER.get(args.workload, METRIC), "value": v, "unit": UNIT,
            "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": d["name"], "n": d["n"], "m": d["m"], "sources": len(d["sources"]), "k": d["k"],
                       "eps": d.get("eps"), "n_hsaw": d.get("n_hsaw"), "delta": "1/n", "parallelism": f"replicas{world}"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} attempts per step of the query stream on {cores} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def same_result(a, b):
    """Equal result counters and estimates (NaN equal to NaN); `steps` counts the draws a
    solve executed (none for attempts served from a walk pool), not part of the result."""
    for key in a:
        if key == "steps":
            continue
        x, y = a[key], b[key]
        if isinstance(x, float) and x != x:
            if y == y:
                return False
        elif x != y:
            return False
    return True


def batch_workload(count, n_max, n_hsaw, seed=1):
    """256 Chung-Lu instances: n log-uniform [1e3, n_max], average degree uniform [8, 32],
    |S| log-uniform [1, 1000], k uniform [10, 500] (clipped to |C|), eSI/nSI alternating,
    N HSAWs each (the batched configuration)."""
    rng = np.random.default_rng(seed)
    inst = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(n_max))))
        deg = int(rng.integers(8, 33))
        src, dst = synth.chung_lu_graph(n, n * deg, 2.1, seed=1000 + i)
        w = synth.wc_weights(n, dst)
        ns = int(min(n, max(1, round(np.exp(rng.uniform(0, np.log(1000)))))))
        mode = "edge" if i % 2 == 0 else "node"
        M = n * deg if mode == "edge" else n
        k = int(min(M, rng.integers(10, 501)))
        inst.append(dict(n=n, m=n * deg, src=src, dst=dst, w=w, sources=synth.sources(n, ns, seed=2000 + i),
                         mode=mode, k=k, n_hsaw=n_hsaw, seed=synth.SEED_WALKS + i))
    return inst


def run_batch_mode(args, hs, torch, emit=True):
    t0 = time.time()
    inst = batch_workload(args.batch_count, args.batch_nmax, args.batch_nhsaw)
    gen_s = time.time() - t0
    graphs = [hs.hsaw_graph_from_edges(x["n"], x["src"], x["dst"], x["w"]) for x in inst]
    queries = [hs.Query(sources=x["sources"], mode=hs.HSAW_EDGE if x["mode"] == "edge" else hs.HSAW_NODE, k=x["k"],
                        n_hsaw=x["n_hsaw"], seed=x["seed"]) for x in inst]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # warm-up: a few instances each way
    for g, q in list(zip(graphs, queries))[:3]:
        hs.hsaw_solve(g, q)
    hs.hsaw_solve_batch(graphs[:8], queries[:8], concurrency=args.batch_workers)
    clocks = Clocks(0)
    clocks.start()
    e0.record(stream)
    serial = [hs.hsaw_solve(g, q) for g, q in zip(graphs, queries)]
    e1.record(stream)
    torch.cuda.synchronize()
    t_serial = e0.elapsed_time(e1) / 1e3
    hs.hsaw_profile_enable(False)  # resets the launch counter; no phase timers in either timed pass
    e0.record(stream)
    batched = hs.hsaw_solve_batch(graphs, queries, concurrency=args.batch_workers)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    prof = hs.hsaw_profile_read()
    hs.hsaw_profile_enable(False)
    ck = clocks.stop()
    identical = all(st == 0 and np.array_equal(ids, a[0]) and np.array_equal(gains, a[1]) and same_result(r, a[2])
                    for (st, ids, gains, r), a in zip(batched, serial))
    n = len(inst)
    breakdown = None
    if args.batch_profile:  # a third, profiled serial pass: per-instance time and sampler time
        per = []
        for x, g, q in zip(inst, graphs, queries):
            hs.hsaw_profile_enable(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hs.hsaw_solve(g, q)
            torch.cuda.synchronize()
            p = hs.hsaw_profile_read()
            per.append({"n": x["n"], "m": x["m"], "sources": len(x["sources"]), "k": x["k"], "mode": x["mode"],
                        "s": time.perf_counter() - t0, "sampler_s": p["sampler_ms"] / 1e3,
                        "draws": p["sampler_steps"]})
        hs.hsaw_profile_enable(False)
        tot, samp = sum(r["s"] for r in per), sum(r["sampler_s"] for r in per)
        per.sort(key=lambda r: -r["s"])
        breakdown = {"serial_s": tot, "sampler_s": samp, "sampler_share": samp / tot, "bound_batched_vs_serial":
                     tot / samp, "slowest": per[:15], "under_50ms": sum(1 for r in per if r["s"] < 0.05)}
    line = {"metric": f"batched SI solves/s ({n} Chung-Lu eSI/nSI instances, N={args.batch_nhsaw} HSAWs each)",
            "value": n / t_batch, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batched", "instances": n, "n_range": [1000, args.batch_nmax],
                       "avg_degree": [8, 32], "sources": [1, 1000], "k": [10, 500], "n_hsaw": args.batch_nhsaw,
                       "workers": args.batch_workers, "graph_gen_s": gen_s,
                       "edges_total": int(sum(x["m"] for x in inst))},
            "serial_solves_per_s": n / t_serial, "batched_vs_serial": t_serial / t_batch,
            "identical_to_serial": bool(identical), "gpu_launches": prof["kernel_launches"], "clocks": ck,
            "serial_profile": breakdown}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def serve_queries(count, graphs_meta, min_sources, seed=5):
    """Serving queries: graph uniform, |S| log-uniform [lo, 1000], k log-uniform [10, 1000],
    eSI or nSI uniform, eps in {0.1, 0.2}, stopping rule."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        gi = int(rng.integers(0, len(graphs_meta)))
        n, m = graphs_meta[gi]
        ns = int(round(np.exp(rng.uniform(np.log(min_sources), np.log(1000)))))
        mode = int(rng.integers(0, 2))
        k = int(round(np.exp(rng.uniform(np.log(10), np.log(1000)))))
        eps = float(rng.choice([0.1, 0.2]))
        out.append((gi, dict(sources=synth.sources(n, ns, seed=7000 + i), mode=mode, k=min(k, n if mode else m),
                             sampling=1, eps=eps, seed=synth.SEED_WALKS + i)))
    return out


def serve_pool_sizes(pool_attempts, ns):
    """Walk-pool attempts per graph: in proportion to the graph's nodes (hit rates fall as
    1/n for the same source-set sizes), whole index blocks of 2^22 attempts, the largest
    graph getting pool_attempts (0: no pools)."""
    if not pool_attempts:
        return [0 for _ in ns]
    n_max = max(ns)
    return [max(1 << 22, (pool_attempts * n // n_max) >> 22 << 22) for n in ns]


def run_serve_mode(args, hs, torch, emit=True):
    scales = [int(x) for x in args.serve_scales.split(",")]
    gm, graphs = [], []
    for sc in scales:
        src, dst = synth.rmat_graph(sc, 16, seed=synth.SEED_GRAPH)
        n = 1 << sc
        graphs.append(hs.hsaw_graph_from_edges(n, src, dst, synth.wc_weights(n, dst)))
        gm.append((n, int(src.shape[0])))
    qs = serve_queries(args.serve_queries, gm, args.serve_min_sources)
    pool_attempts = int(args.serve_pool_attempts)
    pool_sizes = serve_pool_sizes(pool_attempts, [n for n, _ in gm])
    if pool_attempts:  # every query on a graph shares its walk seed, so traces can be reused
        for _, kw in qs:
            kw["seed"] = synth.SEED_WALKS
    if args.serve_max_attempts:  # an attempt budget per query: beyond it, HSAW_E_TIMEOUT
        for _, kw in qs:
            kw["max_attempts"] = int(args.serve_max_attempts)
    queries = [(gi, hs.Query(**kw)) for gi, kw in qs]

    def solve(gi, q):
        try:
            return (0,) + tuple(hs.hsaw_solve(graphs[gi], q))
        except hs.HsawError as e:
            return (e.status, None, None, None)

    # serial: one query at a time on the same stream of queries
    solve(*queries[0])
    t0 = time.perf_counter()
    alone = [solve(gi, q) for gi, q in queries]
    t_serial = time.perf_counter() - t0
    serial_rate = len(queries) / t_serial
    pool_s, pool_gb = 0.0, 0.0
    serial_pooled, serial_pooled_phase = None, None
    if pool_attempts:
        free0 = torch.cuda.mem_get_info()[0]
        t0 = time.perf_counter()
        for g, pa in zip(graphs, pool_sizes):
            g.build_walk_pool(synth.SEED_WALKS, pa)
        torch.cuda.synchronize()
        pool_s = time.perf_counter() - t0
        pool_gb = (free0 - torch.cuda.mem_get_info()[0]) / 1e9
        solve(*queries[0])
        # serial again, now reading the pools: what reuse alone buys (timed without the
        # library's phase timers, whose events cost host time), then where time goes
        t0 = time.perf_counter()
        for gi, q in queries:
            solve(gi, q)
        serial_pooled = len(queries) / (time.perf_counter() - t0)
        hs.hsaw_profile_enable(True)
        for gi, q in queries:
            solve(gi, q)
        serial_pooled_phase = hs.hsaw_profile_read()["phase_ms"]
        hs.hsaw_profile_enable(False)
    rates = [float(x) for x in args.serve_rates.split(",")]
    per_rate = []
    identical = True
    clocks = Clocks(0)
    clocks.start()
    for rate in rates:
        srv = hs.Server(graphs, workers=args.serve_workers)
        rng = np.random.default_rng(int(rate))
        gaps = rng.exponential(1.0 / rate, size=len(queries))
        tickets = []
        t_start = time.perf_counter()
        t_next = t_start
        for (gi, q), gap in zip(queries, gaps):
            t_next += gap
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(gi, q))
        lats = []
        for t, a in zip(tickets, alone):
            try:
                ids, gains, r, lat = srv.poll(t)
                lats.append(lat)
                identical &= bool(a[0] == 0 and np.array_equal(ids, a[1]) and np.array_equal(gains, a[2]) and
                                  same_result(r, a[3]))
            except hs.HsawError as e:  # the same status as alone (an attempt budget that ran out)
                identical &= bool(e.status == a[0])
        t_end = time.perf_counter()
        srv.close()
        per_rate.append({"offered_qps": rate, "solves_per_s": len(queries) / (t_end - t_start),
                         "p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99))})
    ck = clocks.stop()
    best = max(per_rate, key=lambda x: x["solves_per_s"])
    line = {"metric": "served SI solves/s and p50/p99 latency (Poisson arrivals)", "value": best["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "steps": len(rates), "warmup": 1,
            "ms_per_step": 1e3 / best["solves_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "serving", "graphs": [f"rmat{sc}-wc" for sc in scales],
                       "queries_per_rate": len(queries), "sources": [args.serve_min_sources, 1000], "k": [10, 1000],
                       "eps": [0.1, 0.2], "workers": args.serve_workers, "walk_pool_attempts": pool_sizes,
                       "walk_pool_build_s": pool_s, "walk_pool_gb": round(pool_gb, 2),
                       "walk_seed": ("shared per graph: queries on a graph draw the same live-edge worlds, each "
                                     "result is its own estimator, errors across queries correlate")
                       if pool_attempts else "per query",
                       "max_attempts_per_query": int(args.serve_max_attempts) or None},
            "queries_over_budget": sum(1 for a in alone if a[0] != 0),
            "serial_solves_per_s": serial_rate, "served_vs_serial": best["solves_per_s"] / serial_rate,
            "serial_pooled_solves_per_s": serial_pooled, "serial_pooled_device_ms_by_phase": serial_pooled_phase,
            "per_rate": per_rate, "identical_to_alone": bool(identical), "clocks": ck}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_sweep_mode(args, hs, torch):
    """Scalability sweep in the shape of the paper's Fig. "scale": R-MAT graphs with n = 2^13
    .. 2^27 nodes and m/n in {5, 10, 15}; nSI stop-rule solves with the paper's experimental
    query: 1,000 random suspects with random probabilities p, k = 100, eps = 0.1,
    delta = 1/n (Sec. 6 "Parameter Settings")."""
    scales = [int(x) for x in args.sweep_scales.split(",")]
    dens = [int(x) for x in args.sweep_density.split(",")]
    rows = []
    for sc in scales:
        for dn in dens:
            n = 1 << sc
            t0 = time.time()
            src, dst = synth.rmat_graph(sc, dn, seed=synth.SEED_GRAPH)
            w = synth.wc_weights(n, dst)
            S = synth.sources(n, min(1000, n), seed=synth.SEED_SOURCES)
            p = synth.probabilities(S.shape[0], seed=synth.SEED_SOURCES)
            gen_s = time.time() - t0
            g = hs.hsaw_graph_from_edges(n, src, dst, w)
            del src, dst, w
            q = hs.Query(sources=S, p_fixed=p, mode=hs.HSAW_NODE, k=100, sampling=hs.HSAW_STOP_RULE, eps=0.1,
                         seed=synth.SEED_WALKS)
            hs.hsaw_solve(g, q)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ids, gains, r = hs.hsaw_solve(g, q)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            rows.append({"n": n, "m": dn * n, "solve_s": dt, "hsaws": r["hits"], "rounds_t": r["rounds_t"],
                         "hsaws_per_s": r["hits"] / dt, "gen_s": gen_s})
            g.close()
            print(json.dumps({"sweep_point": rows[-1]}), file=sys.stderr, flush=True)
    line = {"metric": "nSI solve time vs graph size (R-MAT, 1000 suspects with random p, k = 100)",
            "value": rows[-1]["solve_s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": rows[-1]["solve_s"] * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "sweep", "scales": scales, "density": dens}, "points": rows}
    print(json.dumps(line), flush=True)


def run_probe_mode(args, hs, torch):
    """Dependent random 32-byte reads per second (the walk's memory pattern without its
    arithmetic) over tables from L2-resident to the size of the billion-edge walk records,
    with 1, 2 and 4 independent chains per lane: the random-request ceiling the sampler's
    draws/s is compared with."""
    rows = []
    for gb in [float(x) for x in args.probe_gb.split(",")]:
        for chains, bps in [(1, b) for b in (1, 2, 3, 4, 5, 6)] + [(2, 6), (2, 3), (4, 6)]:
            steps = max(256, 8192 * bps // (6 * chains))
            rate, ms = hs.hsaw_probe_gather(int(gb * (1 << 30)), chains, steps, bps)
            rows.append({"table_gb": gb, "chains_per_lane": chains, "blocks_per_sm": bps, "reads_per_s": rate,
                         "ms": ms, "gb_per_s_32B": rate * 32 / 1e9})
            print(json.dumps({"probe_point": rows[-1]}), file=sys.stderr, flush=True)
    big = [r for r in rows if r["table_gb"] == max(x["table_gb"] for x in rows)]
    line = {"metric": "dependent random 32-byte reads/s (gather ceiling probe)",
            "value": max(r["reads_per_s"] for r in big), "unit": "reads/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": "gather-probe", "tables_gb": args.probe_gb}, "points": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hsaw", choices=["hsaw", "reference"])
    ap.add_argument("--scale", type=int, default=26)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and served workloads")
    ap.add_argument("--no-probe", action="store_true", help="skip the gather-ceiling probe after the timing")
    ap.add_argument("--ref-attempts", type=int, default=40_000)
    ap.add_argument("--mode", default="solve", choices=["solve", "batch", "serve", "sweep", "probe"])
    ap.add_argument("--sweep-scales", default="13,17,20,23,27")
    ap.add_argument("--probe-gb", default="0.0625,0.25,1,8,32")
    ap.add_argument("--sweep-density", default="5,10,15")
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "c1"])
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-nmax", type=float, default=1e6)
    ap.add_argument("--batch-nhsaw", type=int, default=100_000)
    ap.add_argument("--batch-workers", type=int, default=16)
    ap.add_argument("--batch-profile", action="store_true", help="add a profiled serial pass (per-instance times)")
    ap.add_argument("--serve-scales", default="18,20")
    ap.add_argument("--serve-queries", type=int, default=200)
    ap.add_argument("--serve-rates", default="10,30,100,300,1000,2000")
    ap.add_argument("--serve-workers", type=int, default=16)
    ap.add_argument("--serve-min-sources", type=int, default=16)
    ap.add_argument("--serve-pool-attempts", type=float, default=536870912)
    ap.add_argument("--serve-max-attempts", type=float, default=0)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_1702_05854_gb300 as hs

    torch.cuda.set_device(local)
    if args.mode == "batch":
        return run_batch_mode(args, hs, torch)
    if args.mode == "serve":
        return run_serve_mode(args, hs, torch)
    if args.mode == "sweep":
        return run_sweep_mode(args, hs, torch)
    if args.mode == "probe":
        return run_probe_mode(args, hs, torch)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    d = make_workload(args.scale, args.workload)
    seed = synth.SEED_WALKS + rank
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g = hs.hsaw_graph_from_edges(d["n"], d["src"], d["dst"], d["w"])
    e1.record(stream)
    torch.cuda.synchronize()
    ingest_s = e0.elapsed_time(e1) / 1e3
    q = query_for(hs, d, seed)

    for _ in range(args.warmup):
        hs.hsaw_solve(g, q)

    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    hs.hsaw_profile_enable(True)
    hits = 0
    rounds = []
    e0.record(stream)
    for _ in range(args.steps):
        ids, gains, r = hs.hsaw_solve(g, q)
        hits += r["hits"]
        rounds.append(r["rounds_t"])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    prof = hs.hsaw_profile_read()
    hs.hsaw_profile_enable(False)
    ck = clocks.stop()
    if dist:
        elapsed, hits_all = reduce_over_ranks(dist, torch, "cuda", elapsed, hits)
    else:
        hits_all = float(hits)
    value = hits_all / elapsed

    # roofline of the dominant kernel (the sampler): algorithmic bytes per launch / launch time
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    launches = max(prof["sampler_launches"], 1)
    avg_launch_s = prof["sampler_ms"] / 1e3 / launches
    bytes_per_launch = BYTES_PER_STEP * prof["sampler_steps"] / launches
    achieved = bytes_per_launch / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    traffic = None
    per_draw = NCU_TRAFFIC.get((sampler_hash(), d["name"]))
    if per_draw is not None:
        traffic = per_draw * prof["sampler_steps"] / launches
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "k_sample", "peak_source": "measured" if peaks else "fallback",
                "sampler_share_of_step": prof["sampler_ms"] / 1e3 / elapsed,
                "steps_per_s": prof["sampler_steps"] / (prof["sampler_ms"] / 1e3) if prof["sampler_ms"] else 0.0,
                "phase_ms_per_step": {k_: v_ / args.steps for k_, v_ in prof["phase_ms"].items()}}

    # end to end through the C ABI with host buffers: graph ingest from host arrays + solve
    e2e = None
    if args.e2e_steps > 0:
        h2d = int(d["src"].nbytes + d["dst"].nbytes + d["w"].nbytes + d["sources"].nbytes)
        d2h = d["k"] * 12
        # the step's inputs sit in pinned host memory (numpy views of pinned buffers)
        src_h, dst_h, w_h = (torch.from_numpy(d[k_]).pin_memory().numpy() for k_ in ("src", "dst", "w"))
        e_hits = 0
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.e2e_steps):
            g2 = hs.hsaw_graph_from_edges(d["n"], src_h, dst_h, w_h)
            ids, gains, r = hs.hsaw_solve(g2, q)
            e_hits += r["hits"]
            g2.close()
        e1.record(stream)
        torch.cuda.synchronize()
        et = e0.elapsed_time(e1) / 1e3
        e2e = {"value": e_hits * (world if dist else 1) / et, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "what": "hsaw_graph_from_edges(pinned host edge list) + hsaw_solve per step"}

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(d, seed, args.cpu_seconds)
    gbytes = 16.0 * d["n"] + 56.0 * d["m"]  # node records + edge, walk-record and index arrays
    config = {"workload": d["name"], "n": d["n"], "m": d["m"], "sources": len(d["sources"]), "k": d["k"],
              "eps": d.get("eps"), "n_hsaw": d.get("n_hsaw"), "delta": "1/n", "parallelism": f"replicas{world}",
              "l2": (f"inputs larger than L2 ({gbytes / 1e9:.2f} GB graph)" if gbytes > 129e6 else
                     f"inputs fit L2 ({gbytes / 1e6:.0f} MB graph, not flushed: diagnostic only)"),
              "hits_per_step": hits / args.steps,
              "rounds_t": rounds[-1], "graph_gen_s": d["gen_s"], "graph_ingest_s": ingest_s}
    line = {
        "metric": METRIC_OTHER.get(args.workload, METRIC), "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "config": config,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": prof["kernel_launches"],
        "clocks": ck,
    }
    if cpu:  # the paper's convention (one core) and all host cores, as context
        line["gpu_over_oracle"] = {"one_core": value / cpu["single_core"]["value"], "all_cores": value / cpu["value"],
                                   "cores": cpu["cores"]}
    roofline["attempts_per_s"] = prof["sampler_attempts"] / (prof["sampler_ms"] / 1e3) if prof["sampler_ms"] else 0.0
    if not args.no_probe:  # the random-access ceiling the draws run into, measured after the timed region
        try:
            best = max(hs.hsaw_probe_gather(32 << 30, 1, 2048, b)[0] for b in (1, 2, 6))
            roofline["gather_ceiling"] = {"reads_per_s": best, "what": "dependent random 32 B reads over a 32 GB "
                                          "table, best of 1, 2 and 6 blocks of 256 per SM (bench.py --mode probe)",
                                          "draws_over_ceiling": roofline["steps_per_s"] / best}
        except Exception as e:  # e.g. no room beside the graph
            roofline["gather_ceiling"] = {"unavailable": str(e)[:120]}
    if world == 1 and not args.no_extras:
        # the batched and served workloads, on the same GPU once the billion-edge graph is freed
        g.close()
        del g, d
        import gc
        gc.collect()
        torch.cuda.synchronize()
        line["batched"] = run_batch_mode(args, hs, torch, emit=False)
        line["served"] = run_serve_mode(args, hs, torch, emit=False)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
