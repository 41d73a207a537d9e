"""Seeded synthetic inputs (graphs, LT weights, sources, suspect probabilities).

A module of its own: it makes inputs only and holds none of the interdiction method's
arithmetic.  The CUDA library's tests, the benchmark and the CPU oracle all take their
inputs from here.  The C source is ``synth.c``; ``build()`` compiles it with gcc.

Workload recipes (the paper's datasets, Sec. 6 Table "Datasets' Statistics", are social
graphs of 0.6M-42M nodes and 2M-1.5G edges; these synthetic graphs stand in for them):

* ``chung_lu_graph``: directed Chung-Lu, power-law exponent gamma on in- and out-degree.
* ``rmat_graph``: R-MAT with (a, b, c) = (0.57, 0.19, 0.19), edge factor 16.
* ``wc_weights``: weighted cascade w(u,v) = 1/d_in(v) (Sec. 6 "Parameter Settings").
* ``random_lt_weights``: uniform per in-edge, normalised to a node in-sum U(0.5, 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

SEED_GRAPH, SEED_WEIGHTS, SEED_SOURCES, SEED_WALKS = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile synth.c into _build/libsynth.so (gcc, no GPU needed)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_OUT)
            i64, u64, i32, dbl, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.synth_chung_lu.argtypes = [i64, i64, dbl, u64, i32, p, p]
            lib.synth_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, i32, p, p]
            lib.synth_wc_weights.argtypes = [i64, i64, p, p]
            lib.synth_random_lt_weights.argtypes = [i64, i64, p, u64, p]
            lib.synth_sources.argtypes = [i64, i64, u64, p]
            lib.synth_probabilities.argtypes = [i64, u64, p]
            lib.synth_draw.argtypes = [u64, u64, u64]
            lib.synth_draw.restype = u64
            _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"synth: {what} failed with code {rc}")


def chung_lu_graph(n: int, m: int, gamma: float = 2.1, seed: int = SEED_GRAPH):
    """Directed Chung-Lu edge list (src, dst) as int32 arrays of length m."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    _check(_load().synth_chung_lu(n, m, gamma, seed, _threads(), _ptr(src), _ptr(dst)), "chung_lu")
    return src, dst


def rmat_graph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = SEED_GRAPH):
    """R-MAT edge list with n = 2^scale nodes and m = edge_factor * n edges."""
    m = edge_factor << scale
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    _check(_load().synth_rmat(scale, m, a, b, c, seed, _threads(), _ptr(src), _ptr(dst)), "rmat")
    return src, dst


def wc_weights(n: int, dst: np.ndarray) -> np.ndarray:
    """Weighted-cascade weights floor((2^32-1)/d_in(v)) per edge (uint32)."""
    dst = np.ascontiguousarray(dst, np.int32)
    w = np.empty(dst.shape[0], np.uint32)
    _check(_load().synth_wc_weights(n, dst.shape[0], _ptr(dst), _ptr(w)), "wc_weights")
    return w


def random_lt_weights(n: int, dst: np.ndarray, seed: int = SEED_WEIGHTS) -> np.ndarray:
    """Random LT weights with per-node in-sum U(0.5,1) (uint32 fixed point)."""
    dst = np.ascontiguousarray(dst, np.int32)
    w = np.empty(dst.shape[0], np.uint32)
    _check(_load().synth_random_lt_weights(n, dst.shape[0], _ptr(dst), seed, _ptr(w)), "random_lt_weights")
    return w


def sources(n: int, count: int, seed: int = SEED_SOURCES) -> np.ndarray:
    """`count` distinct uniform nodes in ascending order (int32)."""
    out = np.empty(count, np.int32)
    _check(_load().synth_sources(n, count, seed, _ptr(out)), "sources")
    return out


def probabilities(count: int, seed: int = SEED_SOURCES) -> np.ndarray:
    """Uniform suspect probabilities p(v) as uint32 fixed point (p = value / 2^32)."""
    out = np.empty(count, np.uint32)
    _check(_load().synth_probabilities(count, seed, _ptr(out)), "probabilities")
    return out


def draw(seed: int, stream: int, i: int) -> int:
    """One raw 64-bit draw of the counter-based SplitMix64 stream (seed, stream)."""
    return int(_load().synth_draw(seed, stream, i))


# ------------------------------------------------------------------ named workloads
def workload_c1():
    """eSI plain: Chung-Lu n=16,384, m=131,072, gamma=2.1, WC weights, |S|=16, k=10."""
    n, m = 16384, 131072
    src, dst = chung_lu_graph(n, m, 2.1, SEED_GRAPH)
    return dict(name="chung-lu-16k-eSI", n=n, m=m, src=src, dst=dst, w=wc_weights(n, dst),
                sources=sources(n, 16, SEED_SOURCES), k=10, mode="edge", n_hsaw=200_000)


def workload_rmat(scale: int, weights: str, n_sources: int, k: int, mode: str, **extra):
    n = 1 << scale
    src, dst = rmat_graph(scale, 16, seed=SEED_GRAPH)
    w = wc_weights(n, dst) if weights == "wc" else random_lt_weights(n, dst, SEED_WEIGHTS)
    d = dict(name=f"rmat{scale}-{weights}-{'eSI' if mode == 'edge' else 'nSI'}", n=n, m=int(src.shape[0]),
             src=src, dst=dst, w=w, sources=sources(n, n_sources, SEED_SOURCES), k=k, mode=mode)
    d.update(extra)
    return d


def workload_c2(n_hsaw: int = 10_000_000):
    """nSI: R-MAT scale 20, random LT weights, |S|=100, k=100, N HSAWs."""
    return workload_rmat(20, "random", 100, 100, "node", n_hsaw=n_hsaw)


def workload_c3(scale: int = 26):
    """eSI billion-edge: R-MAT scale 26, WC weights, |S|=1000, k=1000, stopping rule eps=0.1."""
    return workload_rmat(scale, "wc", 1000, 1000, "edge", eps=0.1)
