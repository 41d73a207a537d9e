"""Python binding of libhsaw.so, the GB300 HSAW spread-interdiction library.

Argument marshalling only: every step of the method runs in the CUDA library behind the
C ABI declared in ``include/hsaw.h``; the functions here carry the same names.  PyTorch
supplies device buffers and streams where a call takes device memory.  There is no CPU
fallback: importing this package without the built library (or calling it without a CUDA
device) raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

HSAW_OK = 0
STATUS = {0: "HSAW_OK", -1: "HSAW_E_INVALID", -2: "HSAW_E_WEIGHT_SUM", -3: "HSAW_E_RANGE", -4: "HSAW_E_NOMEM",
          -5: "HSAW_E_DEVICE", -6: "HSAW_E_STEP_CAP", -7: "HSAW_E_TIMEOUT", -8: "HSAW_E_REJECTED",
          -9: "HSAW_E_CANCELLED", -10: "HSAW_E_PENDING"}
HSAW_EDGE, HSAW_NODE = 0, 1
HSAW_FIXED_N, HSAW_STOP_RULE = 0, 1
HSAW_INPUT_DEVICE = 1

_lock = threading.Lock()
_lib = None

_p, _i64, _u64, _i32, _u32, _dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                     ctypes.c_uint32, ctypes.c_double)


class hsaw_query(ctypes.Structure):
    _fields_ = [("sources", _p), ("n_sources", _i32), ("p_fixed", _p), ("mode", ctypes.c_int), ("k", _i32),
                ("candidate_mask", _p), ("sampling", ctypes.c_int), ("n_hsaw", _i64), ("eps", _dbl),
                ("delta", _dbl), ("seed", _u64), ("max_attempts", _u64)]


class hsaw_result(ctypes.Structure):
    _fields_ = [("ids", _p), ("gains", _p), ("n_selected", _i32), ("rounds_t", _i32), ("hits", _u64),
                ("attempts", _u64), ("steps", _u64), ("cov_R", _u64), ("cov_Rprime", _u64), ("hits_Rprime", _u64),
                ("attempts_Rprime", _u64), ("spread_base_est", _dbl), ("spread_reduction_est", _dbl),
                ("eps_t", _dbl)]


class hsaw_profile(ctypes.Structure):
    _fields_ = [("kernel_launches", _u64), ("sampler_launches", _u64), ("sampler_ms", _dbl),
                ("sampler_steps", _u64), ("sampler_attempts", _u64), ("phase_ms", _dbl * 8)]


# name -> (restype, argtypes); mirrors include/hsaw.h
SIGNATURES = {
    "hsaw_graph_from_edges": (ctypes.c_int, [_i64, _i64, _p, _p, _p, _u32, _p, ctypes.POINTER(_p)]),
    "hsaw_graph_from_csr": (ctypes.c_int, [_i64, _i64, _p, _p, _p, _u32, _p, ctypes.POINTER(_p)]),
    "hsaw_graph_destroy": (ctypes.c_int, [_p]),
    "hsaw_graph_info": (ctypes.c_int, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "hsaw_graph_export": (ctypes.c_int, [_p, _p, _p, _p, _p, _p, _p]),
    "hsaw_solve": (ctypes.c_int, [_p, ctypes.POINTER(hsaw_query), ctypes.POINTER(hsaw_result), _p]),
    "hsaw_sample": (ctypes.c_int, [_p, ctypes.POINTER(hsaw_query), _u64, _i64, _p, _p, _u32, ctypes.POINTER(_p), _p]),
    "hsaw_walks_info": (ctypes.c_int, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_u64),
                                       ctypes.POINTER(_u64)]),
    "hsaw_walks_export": (ctypes.c_int, [_p, _p, _p, _p, _p, _p]),
    "hsaw_walks_export_device": (ctypes.c_int, [_p, _p, _p, _p, _p, _p]),
    "hsaw_walks_destroy": (ctypes.c_int, [_p]),
    "hsaw_classify": (ctypes.c_int, [_p, ctypes.POINTER(hsaw_query), _u64, _i64, _p, _p, _p]),
    "hsaw_histogram": (ctypes.c_int, [_p, ctypes.c_int, _i64, _i64, _p, _p, _i64, ctypes.POINTER(_i64), _p]),
    "hsaw_greedy": (ctypes.c_int, [_p, _p, ctypes.c_int, _i64, _i64, _p, _i32, _p, _p, _p]),
    "hsaw_coverage": (ctypes.c_int, [_p, ctypes.c_int, _i64, _i64, _p, _i32, ctypes.POINTER(_u64), _p]),
    "hsaw_stop_constants": (ctypes.c_int, [_i64, _i32, _dbl, _dbl, _p]),
    "hsaw_check": (ctypes.c_int, [_dbl, _dbl, _dbl, _i32, _dbl, _dbl, ctypes.POINTER(_dbl)]),
    "hsaw_sample_hits_static": (ctypes.c_int, [_p, _p, _u64, _u64, _i64, _p, _p, _i64, ctypes.POINTER(_i64), _p]),
    "hsaw_solve_batch": (ctypes.c_int, [_p, _p, _p, _p, _i32, _i32, _p]),
    "hsaw_graph_edge": (ctypes.c_int, [_p, _i64, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "hsaw_estimate_spread": (ctypes.c_int, [_p, ctypes.POINTER(hsaw_query), _p, _i32, ctypes.POINTER(_dbl),
                                            ctypes.POINTER(_dbl), _p]),
    "hsaw_debug_fail_alloc_after": (ctypes.c_int, [_i64]),
    "hsaw_set_allocator": (ctypes.c_int, [_p, _p, _p]),
    "hsaw_graph_build_walk_pool": (ctypes.c_int, [_p, _u64, _u64, _p]),
    "hsaw_graph_drop_walk_pool": (ctypes.c_int, [_p]),
    "hsaw_server_create": (ctypes.c_int, [_p, _i32, ctypes.c_size_t, _i32, ctypes.POINTER(_p)]),
    "hsaw_server_submit": (ctypes.c_int, [_p, _i32, ctypes.POINTER(hsaw_query), ctypes.POINTER(_u64)]),
    "hsaw_server_poll": (ctypes.c_int, [_p, _u64, ctypes.POINTER(hsaw_result), _i32, ctypes.POINTER(_dbl)]),
    "hsaw_server_cancel": (ctypes.c_int, [_p, _u64]),
    "hsaw_server_destroy": (ctypes.c_int, [_p]),
    "hsaw_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "hsaw_profile_read": (ctypes.c_int, [ctypes.POINTER(hsaw_profile)]),
    "hsaw_probe_gather": (ctypes.c_int, [_u64, _i32, ctypes.c_uint32, _i32, ctypes.POINTER(_dbl),
                                         ctypes.POINTER(_dbl), _p]),
    "hsaw_last_error": (ctypes.c_char_p, []),
    "hsaw_version": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load():
    """Load (building first if the sources are newer) libhsaw.so; raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class HsawError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(rc):
    if rc != HSAW_OK:
        raise HsawError(rc, load().hsaw_last_error().decode(errors="replace"))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(a.data_ptr()))  # torch tensor


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream))


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_1702_05854_gb300 needs a CUDA device (GB300, sm_103a); no CPU fallback exists")


# ------------------------------------------------------------------ C-ABI names
def hsaw_version() -> str:
    return load().hsaw_version().decode()


def hsaw_stop_constants(M, k, eps, delta):
    out = np.empty(6, np.float64)
    _check(load().hsaw_stop_constants(M, k, eps, delta, _ptr(out)))
    return dict(lnC=out[0], N_max=out[1], Upsilon=out[2], t_max=int(out[3]), Lambda=out[4], Lambda1=out[5])


def hsaw_check(c, cp, size_rprime, t, eps, lambda1):
    et = ctypes.c_double()
    ok = load().hsaw_check(float(c), float(cp), float(size_rprime), int(t), float(eps), float(lambda1),
                           ctypes.byref(et))
    return bool(ok), et.value


class Graph:
    """A device graph (hsaw_graph handle).  Build with hsaw_graph_from_edges / _from_csr."""

    def __init__(self, handle, n, m):
        self._h = handle
        self.n, self.m = int(n), int(m)

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hsaw_graph_destroy(h)
        self._h = None

    @property
    def handle(self):
        return self._h

    def build_walk_pool(self, seed: int, attempts: int, stream=None):
        """Index the query-independent traces of attempts [0, attempts) for walk seed `seed`
        (per node, the attempts whose trace passes through it); queries with that seed then
        take their hits below `attempts` from their sources' lists."""
        _check(load().hsaw_graph_build_walk_pool(self._h, seed, attempts, _stream(stream)))

    def drop_walk_pool(self):
        _check(load().hsaw_graph_drop_walk_pool(self._h))

    def export(self, stream=None):
        """Host copy of the device CSR: (row_ptr, src, dst, thr, input_index)."""
        rp = np.empty(self.n + 1, np.int64)
        s = np.empty(self.m, np.int32)
        d = np.empty(self.m, np.int32)
        t = np.empty(self.m, np.uint32)
        ii = np.empty(self.m, np.int64)
        _check(load().hsaw_graph_export(self._h, _ptr(rp), _ptr(s), _ptr(d), _ptr(t), _ptr(ii), _stream(stream)))
        return rp, s, d, t, ii


def hsaw_graph_edge(graph, edge_id: int):
    """(src, dst, input_index) of a CSR edge id."""
    a, b, c = _i32(), _i32(), _i64()
    _check(load().hsaw_graph_edge(graph.handle, edge_id, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def hsaw_estimate_spread(graph, query, removed=None, stream=None):
    """(spread, std_err) of V_I on the graph with `removed` edges (eSI) or nodes (nSI)."""
    rem = np.ascontiguousarray(removed if removed is not None else np.zeros(0), np.int64)
    q = query.c()
    sp, se = _dbl(), _dbl()
    _check(load().hsaw_estimate_spread(graph.handle, ctypes.byref(q), _ptr(rem) if rem.size else None, rem.size,
                                       ctypes.byref(sp), ctypes.byref(se), _stream(stream)))
    return sp.value, se.value


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None  # the installed callbacks, kept alive while the library holds them


def hsaw_set_allocator(alloc=None, release=None):
    """Scratch device memory from alloc(nbytes, stream) -> device pointer (an int; 0 when
    out of memory) and release(ptr, stream), stream being the raw cudaStream_t as an int;
    with no arguments, from CUDA's stream-ordered pool again.  Refused (HsawError) while
    the library still holds scratch of the current allocator."""
    global _allocator_refs
    if alloc is None and release is None:
        _check(load().hsaw_set_allocator(None, None, None))
        _allocator_refs = None
        return
    if alloc is None or release is None:
        raise ValueError("give both alloc and release, or neither")

    def a(nbytes, stream, ctx):
        try:
            return alloc(int(nbytes), stream or 0) or None
        except Exception:  # the library reports HSAW_E_NOMEM
            return None

    def r(ptr, stream, ctx):
        release(ptr, stream or 0)

    fa, fr = _ALLOC_FN(a), _FREE_FN(r)
    _check(load().hsaw_set_allocator(ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(fr, ctypes.c_void_p), None))
    _allocator_refs = (fa, fr)


def use_torch_allocator(on: bool = True):
    """Take the library's scratch from torch's caching allocator (on the stream the library
    runs on), or (on=False) from CUDA's pool again."""
    if not on:
        hsaw_set_allocator()
        return
    import torch
    hsaw_set_allocator(lambda nbytes, stream: torch.cuda.caching_allocator_alloc(nbytes, stream=stream),
                       lambda ptr, stream: torch.cuda.caching_allocator_delete(ptr))


def hsaw_debug_fail_alloc_after(n: int):
    """Test hook: make the n-th device allocation from now on fail (n <= 0 disables)."""
    _check(load().hsaw_debug_fail_alloc_after(n))


def hsaw_graph_from_edges(n, src, dst, w_fixed, stream=None) -> Graph:
    """Device graph from an edge list (numpy host arrays or torch CUDA tensors)."""
    _require_cuda()
    on_dev = not isinstance(src, np.ndarray)
    if not on_dev:
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        w_fixed = np.ascontiguousarray(w_fixed, np.uint32)
    m = int(src.shape[0])
    h = ctypes.c_void_p()
    _check(load().hsaw_graph_from_edges(n, m, _ptr(src), _ptr(dst), _ptr(w_fixed),
                                        HSAW_INPUT_DEVICE if on_dev else 0, _stream(stream), ctypes.byref(h)))
    return Graph(h, n, m)


def hsaw_graph_from_csr(n, row_ptr, src, w_fixed, stream=None) -> Graph:
    """Device graph from an in-adjacency CSR (edge ids = the given positions)."""
    _require_cuda()
    on_dev = not isinstance(src, np.ndarray)
    if not on_dev:
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        src = np.ascontiguousarray(src, np.int32)
        w_fixed = np.ascontiguousarray(w_fixed, np.uint32)
    m = int(src.shape[0])
    h = ctypes.c_void_p()
    _check(load().hsaw_graph_from_csr(n, m, _ptr(row_ptr), _ptr(src), _ptr(w_fixed),
                                      HSAW_INPUT_DEVICE if on_dev else 0, _stream(stream), ctypes.byref(h)))
    return Graph(h, n, m)


@dataclass
class Query:
    sources: np.ndarray
    mode: int = HSAW_EDGE
    k: int = 10
    sampling: int = HSAW_FIXED_N
    n_hsaw: int = 0
    eps: float = 0.1
    delta: float = -1.0
    seed: int = 4
    p_fixed: np.ndarray | None = None
    candidate_mask: np.ndarray | None = None
    max_attempts: int = 0

    def c(self):
        """ctypes hsaw_query; keeps the numpy arrays alive on the object."""
        self._src = np.ascontiguousarray(self.sources, np.int32)
        self._p = None if self.p_fixed is None else np.ascontiguousarray(self.p_fixed, np.uint32)
        self._cm = None if self.candidate_mask is None else np.ascontiguousarray(self.candidate_mask, np.uint8)
        return hsaw_query(_ptr(self._src), self._src.shape[0], _ptr(self._p), self.mode, self.k, _ptr(self._cm),
                          self.sampling, self.n_hsaw, self.eps, self.delta, self.seed, self.max_attempts)


def hsaw_solve(graph: Graph, query: Query, stream=None):
    """Solve one instance; returns (ids int64[k], gains uint32[k], result dict)."""
    ids = np.empty(query.k, np.int64)
    gains = np.empty(query.k, np.uint32)
    r = hsaw_result()
    r.ids = _ptr(ids)
    r.gains = _ptr(gains)
    q = query.c()
    _check(load().hsaw_solve(graph.handle, ctypes.byref(q), ctypes.byref(r), _stream(stream)))
    return ids, gains, _result_dict(r)


def _result_dict(r):
    return {f: getattr(r, f) for f, _ in hsaw_result._fields_ if f not in ("ids", "gains")}


def hsaw_solve_batch(graphs, queries, concurrency: int = 0, stream=None):
    """Solve instances (graphs[i], queries[i]) concurrently; returns a list of
    (status, ids, gains, result dict) in instance order."""
    n = len(queries)
    qa = (hsaw_query * n)(*[q.c() for q in queries])
    ra = (hsaw_result * n)()
    outs = []
    for i, q in enumerate(queries):
        ids = np.empty(q.k, np.int64)
        gains = np.empty(q.k, np.uint32)
        ra[i].ids = _ptr(ids)
        ra[i].gains = _ptr(gains)
        outs.append((ids, gains))
    ga = (ctypes.c_void_p * n)(*[g.handle for g in graphs])
    st = (ctypes.c_int * n)()
    load().hsaw_solve_batch(ga, qa, ra, st, n, concurrency, _stream(stream))
    return [(int(st[i]), outs[i][0], outs[i][1], _result_dict(ra[i])) for i in range(n)]


class Server:
    """Continuous-batching server over resident graphs (hsaw_server handle)."""

    def __init__(self, graphs, mem_budget: int = 0, workers: int = 0):
        self._graphs = list(graphs)
        ga = (ctypes.c_void_p * len(graphs))(*[g.handle for g in graphs])
        h = ctypes.c_void_p()
        _check(load().hsaw_server_create(ga, len(graphs), mem_budget, workers, ctypes.byref(h)))
        self._h = h
        self._k = {}

    def submit(self, graph_idx: int, query: Query) -> int:
        q = query.c()
        t = _u64()
        _check(load().hsaw_server_submit(self._h, graph_idx, ctypes.byref(q), ctypes.byref(t)))
        self._k[t.value] = query.k
        return int(t.value)

    def poll(self, ticket: int, timeout_ms: int = -1):
        """(ids, gains, result dict, latency_ms); raises HsawError (HSAW_E_PENDING while running,
        else the query's own failing status)."""
        k = self._k.get(ticket, 1)  # an unknown ticket: the library reports HSAW_E_INVALID
        ids = np.empty(k, np.int64)
        gains = np.empty(k, np.uint32)
        r = hsaw_result()
        r.ids = _ptr(ids)
        r.gains = _ptr(gains)
        lat = _dbl()
        rc = load().hsaw_server_poll(self._h, ticket, ctypes.byref(r), timeout_ms, ctypes.byref(lat))
        if rc != -10:
            self._k.pop(ticket, None)
        _check(rc)
        return ids, gains, _result_dict(r), lat.value

    def cancel(self, ticket: int):
        _check(load().hsaw_server_cancel(self._h, ticket))

    def close(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hsaw_server_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


class Walks:
    """An ordered HSAW stream on the device (hsaw_walks handle)."""

    def __init__(self, handle):
        self._h = handle

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hsaw_walks_destroy(h)
        self._h = None

    @property
    def handle(self):
        return self._h

    def info(self):
        c, t, a, s = _i64(), _i64(), _u64(), _u64()
        _check(load().hsaw_walks_info(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(a), ctypes.byref(s)))
        return dict(count=c.value, total_nodes=t.value, attempts=a.value, steps=s.value)

    def export(self, stream=None):
        inf = self.info()
        cnt, tot = inf["count"], inf["total_nodes"]
        aid = np.empty(cnt, np.uint64)
        off = np.empty(cnt + 1, np.int64)
        nodes = np.empty(tot, np.int32)
        edges = np.empty(max(tot - cnt, 0), np.int32)
        _check(load().hsaw_walks_export(self._h, _ptr(aid), _ptr(off), _ptr(nodes), _ptr(edges), _stream(stream)))
        return aid, off, nodes, edges

    def export_device(self, stream=None):
        """The same arrays as export(), as torch CUDA tensors (aid as int64 bits of uint64),
        copied on the device into caller-owned buffers."""
        import torch
        inf = self.info()
        cnt, tot = inf["count"], inf["total_nodes"]
        aid = torch.empty(cnt, dtype=torch.int64, device="cuda")
        off = torch.empty(cnt + 1, dtype=torch.int64, device="cuda")
        nodes = torch.empty(tot, dtype=torch.int32, device="cuda")
        edges = torch.empty(max(tot - cnt, 0), dtype=torch.int32, device="cuda")
        _check(load().hsaw_walks_export_device(self._h, _ptr(aid), _ptr(off), _ptr(nodes), _ptr(edges),
                                               _stream(stream)))
        return aid, off, nodes, edges


def hsaw_sample(graph: Graph, query: Query, first_attempt: int, n_hits: int, edge_removed=None, node_removed=None,
                stream=None) -> Walks:
    q = query.c()
    er = None if edge_removed is None else np.ascontiguousarray(edge_removed, np.uint8)
    nr = None if node_removed is None else np.ascontiguousarray(node_removed, np.uint8)
    h = ctypes.c_void_p()
    _check(load().hsaw_sample(graph.handle, ctypes.byref(q), first_attempt, n_hits, _ptr(er), _ptr(nr), 0,
                              ctypes.byref(h), _stream(stream)))
    return Walks(h)


HSAW_STATIC_MAX_ATTEMPTS = 1 << 18


def hsaw_sample_hits_static(graph: Graph, suspect_bits, seed: int, first_attempt: int, n_attempts: int, aid_out,
                            len_out, stream=None) -> int:
    """Allocation-free hit search over an attempt range (see include/hsaw.h).

    suspect_bits (int32 view of uint32, at least ceil(n / 32) words), aid_out (int64 view
    of uint64) and len_out (int32 view of uint32) are caller-owned contiguous torch CUDA
    tensors; returns the number of hits written.  The output capacity is the shorter of
    the two output tensors."""
    import torch
    for name, t, dt in (("suspect_bits", suspect_bits, torch.int32), ("aid_out", aid_out, torch.int64),
                        ("len_out", len_out, torch.int32)):
        if not (t.is_cuda and t.is_contiguous() and t.dtype == dt):
            raise ValueError(f"{name} must be a contiguous CUDA tensor of {dt}")
    if suspect_bits.numel() < (graph.n + 31) // 32:
        raise ValueError("suspect_bits must hold ceil(n / 32) words")
    n = _i64()
    cap = min(int(aid_out.numel()), int(len_out.numel()))
    _check(load().hsaw_sample_hits_static(graph.handle, _ptr(suspect_bits), seed, first_attempt, n_attempts,
                                          _ptr(aid_out), _ptr(len_out), cap, ctypes.byref(n), _stream(stream)))
    return int(n.value)


def hsaw_classify(graph: Graph, query: Query, first: int, count: int, stream=None):
    """(outcome int8, length int32) torch CUDA tensors for attempts [first, first+count)."""
    import torch
    out = torch.empty(count, dtype=torch.int8, device="cuda")
    ln = torch.empty(count, dtype=torch.int32, device="cuda")
    q = query.c()
    _check(load().hsaw_classify(graph.handle, ctypes.byref(q), first, count, _ptr(out), _ptr(ln), _stream(stream)))
    return out, ln


def hsaw_histogram(walks: Walks, mode: int, first: int, count: int, stream=None):
    L = load()
    nu = _i64()
    cap = max(1, walks.info()["total_nodes"])
    uid = np.empty(cap, np.int32)
    cnt = np.empty(cap, np.uint32)
    _check(L.hsaw_histogram(walks.handle, mode, first, count, _ptr(uid), _ptr(cnt), cap, ctypes.byref(nu),
                            _stream(stream)))
    return uid[:nu.value].copy(), cnt[:nu.value].copy()


def hsaw_greedy(walks: Walks, graph: Graph, mode: int, first: int, count: int, k: int, candidate_mask=None,
                stream=None):
    ids = np.empty(k, np.int64)
    gains = np.empty(k, np.uint32)
    cm = None if candidate_mask is None else np.ascontiguousarray(candidate_mask, np.uint8)
    _check(load().hsaw_greedy(walks.handle, graph.handle, mode, first, count, _ptr(cm), k, _ptr(ids), _ptr(gains),
                              _stream(stream)))
    return ids, gains


def hsaw_coverage(walks: Walks, mode: int, first: int, count: int, T, stream=None) -> int:
    T = np.ascontiguousarray(T, np.int64)
    cov = _u64()
    _check(load().hsaw_coverage(walks.handle, mode, first, count, _ptr(T), T.shape[0], ctypes.byref(cov),
                                _stream(stream)))
    return int(cov.value)


def hsaw_profile_enable(on: bool = True):
    _check(load().hsaw_profile_enable(1 if on else 0))


def hsaw_profile_read():
    p = hsaw_profile()
    _check(load().hsaw_profile_read(ctypes.byref(p)))
    d = {f: getattr(p, f) for f, _ in hsaw_profile._fields_ if f != "phase_ms"}
    d["phase_ms"] = {"sampling": p.phase_ms[0], "counting": p.phase_ms[1], "greedy": p.phase_ms[2],
                     "coverage": p.phase_ms[3]}
    return d


def hsaw_probe_gather(table_bytes: int, chains: int = 1, steps: int = 256, blocks_per_sm: int = 0, stream=None):
    """(dependent random 32-byte reads per second, timed ms) over a table of table_bytes."""
    r, ms = _dbl(), _dbl()
    _check(load().hsaw_probe_gather(table_bytes, chains, steps, blocks_per_sm, ctypes.byref(r), ctypes.byref(ms),
                                    _stream(stream)))
    return r.value, ms.value


def hsaw_last_error() -> str:
    return load().hsaw_last_error().decode(errors="replace")
