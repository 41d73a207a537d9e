"""CPU oracle for HSAW spread interdiction (test infrastructure only).

This package is the plain, slow, obviously-correct statement of what the CUDA path
computes (``oracle.c``; each C function cites the paper passage it follows).  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it;
the product library never imports it and shares no code with it.

Pins: see the header of ``oracle.c`` and ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_EDGE, MODE_NODE = 0, 1
MISS_NO_EDGE, HIT, MISS_CYCLE, MISS_REMOVED, STEP_CAP = 0, 1, 2, 3, -6


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so with gcc (no GPU needed)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Result(ctypes.Structure):
    _fields_ = [("n_selected", ctypes.c_int32), ("rounds_t", ctypes.c_int32),
                ("hits", ctypes.c_uint64), ("attempts", ctypes.c_uint64), ("steps", ctypes.c_uint64),
                ("cov_R", ctypes.c_uint64), ("cov_Rprime", ctypes.c_uint64),
                ("hits_Rprime", ctypes.c_uint64), ("attempts_Rprime", ctypes.c_uint64),
                ("spread_base_est", ctypes.c_double), ("spread_reduction_est", ctypes.c_double),
                ("eps_t", ctypes.c_double), ("status", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_OUT)
            p, i64, u64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
            L.oracle_philox4x32_10.argtypes = [p, p, p]
            L.oracle_graph_build.argtypes = [i64, i64, p, p, p, ctypes.POINTER(p)]
            L.oracle_graph_free.argtypes = [p]
            L.oracle_graph_n.argtypes = [p]; L.oracle_graph_n.restype = i64
            L.oracle_graph_m.argtypes = [p]; L.oracle_graph_m.restype = i64
            L.oracle_graph_export.argtypes = [p, p, p, p, p, p]
            L.oracle_ctx_new.argtypes = [p, p, i64, p, p, p, u64]; L.oracle_ctx_new.restype = p
            L.oracle_ctx_free.argtypes = [p]
            L.oracle_attempt.argtypes = [p, u64, p, p, p]; L.oracle_attempt.restype = ctypes.c_int
            L.oracle_walks_new.argtypes = [u64]; L.oracle_walks_new.restype = p
            L.oracle_walks_free.argtypes = [p]
            L.oracle_stream_extend.argtypes = [p, p, i64, u64]; L.oracle_stream_extend.restype = ctypes.c_int
            L.oracle_classify.argtypes = [p, u64, i64, p, p]
            L.oracle_walks_count.argtypes = [p]; L.oracle_walks_count.restype = i64
            L.oracle_walks_nodes_total.argtypes = [p]; L.oracle_walks_nodes_total.restype = i64
            L.oracle_walks_attempts.argtypes = [p]; L.oracle_walks_attempts.restype = u64
            L.oracle_walks_steps.argtypes = [p]; L.oracle_walks_steps.restype = u64
            L.oracle_walks_export.argtypes = [p, p, p, p, p]
            L.oracle_walks_append.argtypes = [p, p, u64, i64]; L.oracle_walks_append.restype = ctypes.c_int
            L.oracle_histogram.argtypes = [p, ctypes.c_int, i64, i64, i64, p]
            L.oracle_coverage.argtypes = [p, ctypes.c_int, i64, i64, i64, p, i32]; L.oracle_coverage.restype = i64
            L.oracle_greedy.argtypes = [p, ctypes.c_int, i64, i64, i64, p, i32, p, p]; L.oracle_greedy.restype = ctypes.c_int
            L.oracle_greedy_lists.argtypes = [p, ctypes.c_int, i64, i64, i64, p, i32, p, p]
            L.oracle_greedy_lists.restype = ctypes.c_int
            L.oracle_stop_constants.argtypes = [i64, i32, dbl, dbl, p]
            L.oracle_check.argtypes = [dbl, dbl, dbl, ctypes.c_int, dbl, dbl, ctypes.POINTER(dbl)]
            L.oracle_check.restype = ctypes.c_int
            L.oracle_solve.argtypes = [p, ctypes.c_int, p, i32, ctypes.c_int, i64, dbl, dbl, u64, p, p,
                                       ctypes.POINTER(_Result)]
            L.oracle_solve.restype = ctypes.c_int
            L.oracle_source_coin.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.oracle_source_coin.restype = ctypes.c_int
            L.oracle_select_in_edge.argtypes = [p, ctypes.c_int32, ctypes.c_uint32]
            L.oracle_select_in_edge.restype = i64
            L.oracle_bruteforce_spread.argtypes = [p, p, i32, p, p, p]
            L.oracle_bruteforce_spread.restype = dbl
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(counter, key):
    """Philox4x32-10 block for a 4-word counter and 2-word key (uint32 words)."""
    c = np.ascontiguousarray(counter, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.empty(4, np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


class Graph:
    """In-adjacency graph with cumulative uint32 thresholds (oracle's own build)."""

    def __init__(self, n, src, dst, w):
        L = _load()
        self._keep = [np.ascontiguousarray(src, np.int32), np.ascontiguousarray(dst, np.int32),
                      np.ascontiguousarray(w, np.uint32)]
        self.n, self.m = int(n), int(self._keep[0].shape[0])
        h = ctypes.c_void_p()
        rc = L.oracle_graph_build(self.n, self.m, _ptr(self._keep[0]), _ptr(self._keep[1]),
                                  _ptr(self._keep[2]), ctypes.byref(h))
        self.status = rc
        if rc != 0:
            raise ValueError(f"oracle graph build failed ({rc})")
        self._h = h
        self._keep = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_graph_free(h)
            self._h = None

    def select_in_edge(self, v: int, r: int) -> int:
        """CSR id of v's live in-edge for the draw r, or -1."""
        return int(_load().oracle_select_in_edge(self._h, v, r))

    def arrays(self):
        """(row_ptr int64[n+1], src int32[m], dst int32[m], thr uint32[m], input_index int64[m])"""
        rp = np.empty(self.n + 1, np.int64)
        s = np.empty(self.m, np.int32)
        d = np.empty(self.m, np.int32)
        t = np.empty(self.m, np.uint32)
        ii = np.empty(self.m, np.int64)
        _load().oracle_graph_export(self._h, _ptr(rp), _ptr(s), _ptr(d), _ptr(t), _ptr(ii))
        return rp, s, d, t, ii


def source_coin(x1: int, p32: int) -> bool:
    """Source coin rule: x1 < p32, with p32 = 0xFFFFFFFF certain."""
    return bool(_load().oracle_source_coin(x1, p32))


class Query:
    """Suspects (with optional p), optional removed edges/nodes, and the walk seed."""

    def __init__(self, graph: Graph, sources, p_fixed=None, edge_removed=None, node_removed=None, seed=4):
        self.graph = graph
        self._src = np.ascontiguousarray(sources, np.int32)
        self._p = None if p_fixed is None else np.ascontiguousarray(p_fixed, np.uint32)
        self._er = None if edge_removed is None else np.ascontiguousarray(edge_removed, np.uint8)
        self._nr = None if node_removed is None else np.ascontiguousarray(node_removed, np.uint8)
        self._h = _load().oracle_ctx_new(graph._h, _ptr(self._src), self._src.shape[0], _ptr(self._p),
                                         _ptr(self._er), _ptr(self._nr), seed)
        if not self._h:
            raise MemoryError("oracle_ctx_new")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_ctx_free(h)
            self._h = None

    def attempt(self, a: int):
        """(outcome, nodes, edges) of attempt a."""
        n = self.graph.n
        nodes = np.empty(n + 1, np.int32)
        edges = np.empty(n + 1, np.int32)
        ln = ctypes.c_int64()
        r = _load().oracle_attempt(self._h, a, _ptr(nodes), _ptr(edges), ctypes.byref(ln))
        l = ln.value
        return r, nodes[:l].copy(), edges[:max(l - 1, 0)].copy()

    def classify(self, first: int, count: int):
        """Outcome code and walk length of every attempt in [first, first+count)."""
        out = np.empty(count, np.int8)
        ln = np.empty(count, np.int32)
        _load().oracle_classify(self._h, first, count, _ptr(out), _ptr(ln))
        return out, ln


@dataclass
class Walks:
    aid: np.ndarray
    node_off: np.ndarray
    nodes: np.ndarray
    edges: np.ndarray
    attempts: int
    steps: int

    def __len__(self):
        return self.aid.shape[0]

    def walk(self, j):
        b, e = int(self.node_off[j]), int(self.node_off[j + 1])
        return self.nodes[b:e], self.edges[b - j:e - j - 1]

    def elements(self, mode):
        """Concatenated element ids and per-walk offsets for the mode."""
        if mode == MODE_NODE:
            return self.nodes, self.node_off
        return self.edges, self.node_off - np.arange(self.node_off.shape[0], dtype=np.int64)


class Stream:
    """The ordered HSAW stream of a query (Alg. 3), extended on demand."""

    def __init__(self, query: Query, first_aid: int = 0):
        self.query = query
        self._h = _load().oracle_walks_new(first_aid)
        self._next = first_aid

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_walks_free(h)
            self._h = None

    def extend(self, want_hits: int, max_attempts: int = 1 << 62):
        a0 = self.attempts
        rc = _load().oracle_stream_extend(self.query._h, self._h, want_hits, max_attempts)
        if rc != 0:
            raise RuntimeError(f"oracle stream failed ({rc})")
        self._next += self.attempts - a0
        return self

    def extend_threads(self, want_hits: int, threads: int, max_attempts: int = 1 << 62, chunk: int = 1 << 16):
        """extend() with the attempts examined by `threads` host threads in consecutive
        ranges of `chunk` attempts, joined in attempt order: the same walks as extend()
        (attempts are independent, Alg. 3).  Harness only; the oracle's arithmetic is the
        per-attempt code that extend() runs.  `steps` covers whole ranges only."""
        import concurrent.futures as cf
        L = _load()
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            while len(self) < want_hits and max_attempts > 0:
                firsts, parts = [], []
                for _ in range(threads):
                    if max_attempts <= 0:
                        break
                    c = min(chunk, max_attempts)
                    firsts.append((self._next + sum(x[1] for x in firsts), c))
                    max_attempts -= c
                parts = [Stream(self.query, f) for f, _ in firsts]
                list(ex.map(lambda pc: pc[0].extend(1 << 62, pc[1]), zip(parts, [c for _, c in firsts])))
                for part, (f, c) in zip(parts, firsts):
                    need = want_hits - len(self)
                    cut = need <= len(part)
                    rc = L.oracle_walks_append(self._h, part._h, f, need if cut else -1)
                    if rc != 0:
                        raise RuntimeError(f"oracle stream join failed ({rc})")
                    self._next = int(part.export().aid[need - 1]) + 1 if cut else f + c
                    if len(self) >= want_hits:
                        break
        return self

    def __len__(self):
        return int(_load().oracle_walks_count(self._h))

    @property
    def attempts(self):
        return int(_load().oracle_walks_attempts(self._h))

    @property
    def steps(self):
        return int(_load().oracle_walks_steps(self._h))

    def export(self) -> Walks:
        L = _load()
        cnt = int(L.oracle_walks_count(self._h))
        tot = int(L.oracle_walks_nodes_total(self._h))
        aid = np.empty(cnt, np.uint64)
        off = np.empty(cnt + 1, np.int64)
        nodes = np.empty(tot, np.int32)
        edges = np.empty(tot - cnt, np.int32)
        L.oracle_walks_export(self._h, _ptr(aid), _ptr(off), _ptr(nodes), _ptr(edges))
        return Walks(aid, off, nodes, edges, self.attempts, self.steps)

    def histogram(self, mode, first, count, M):
        cnt = np.empty(M, np.uint32)
        _load().oracle_histogram(self._h, mode, first, count, M, _ptr(cnt))
        return cnt

    def coverage(self, mode, first, count, M, T):
        T = np.ascontiguousarray(T, np.int64)
        return int(_load().oracle_coverage(self._h, mode, first, count, M, _ptr(T), T.shape[0]))

    def greedy(self, mode, first, count, M, k, cand_mask=None, kept_gains=False):
        """Greedy (Alg. 4 / 7): gains recounted every round, or (kept_gains) kept and
        decremented as walks are covered; both return the same picks."""
        ids = np.empty(k, np.int64)
        gains = np.empty(k, np.uint32)
        cm = None if cand_mask is None else np.ascontiguousarray(cand_mask, np.uint8)
        f = _load().oracle_greedy_lists if kept_gains else _load().oracle_greedy
        rc = f(self._h, mode, first, count, M, _ptr(cm), k, _ptr(ids), _ptr(gains))
        if rc != 0:
            raise ValueError(f"oracle greedy failed ({rc})")
        return ids, gains


def stop_constants(M: int, k: int, eps: float, delta: float):
    """dict(lnC, N_max, Upsilon, t_max, Lambda, Lambda1) of the stopping rule."""
    out = np.empty(6, np.float64)
    _load().oracle_stop_constants(M, k, eps, delta, _ptr(out))
    return dict(lnC=out[0], N_max=out[1], Upsilon=out[2], t_max=int(out[3]), Lambda=out[4], Lambda1=out[5])


def check(c, cp, size_rp, t, eps, lambda1):
    """(passes, eps_t) of the Check step."""
    et = ctypes.c_double()
    ok = _load().oracle_check(float(c), float(cp), float(size_rp), int(t), float(eps), float(lambda1),
                              ctypes.byref(et))
    return bool(ok), et.value


def solve(query: Query, mode: int, k: int, n_hsaw: int = 0, stop_rule: bool = False, eps: float = 0.1,
          delta: float = -1.0, cand_mask=None, max_attempts: int = 1 << 62):
    """Full oracle solve; returns (ids, gains, result dict)."""
    ids = np.empty(k, np.int64)
    gains = np.empty(k, np.uint32)
    res = _Result()
    cm = None if cand_mask is None else np.ascontiguousarray(cand_mask, np.uint8)
    rc = _load().oracle_solve(query._h, mode, _ptr(cm), k, int(stop_rule), n_hsaw, eps, delta, max_attempts,
                              _ptr(ids), _ptr(gains), ctypes.byref(res))
    if rc != 0:
        raise RuntimeError(f"oracle solve failed ({rc})")
    d = {f: getattr(res, f) for f, _ in _Result._fields_}
    return ids, gains, d


def bruteforce_spread(graph: Graph, sources, p_fixed=None, edge_removed=None, node_removed=None) -> float:
    """Exact I_G(V_I) (or I_G'(V_I) with removals) by live-edge world enumeration."""
    s = np.ascontiguousarray(sources, np.int32)
    p = None if p_fixed is None else np.ascontiguousarray(p_fixed, np.uint32)
    er = None if edge_removed is None else np.ascontiguousarray(edge_removed, np.uint8)
    nr = None if node_removed is None else np.ascontiguousarray(node_removed, np.uint8)
    return float(_load().oracle_bruteforce_spread(graph._h, _ptr(s), s.shape[0], _ptr(p), _ptr(er), _ptr(nr)))
