"""Hand-built and seeded random tiny graphs for the brute-force pins (test-only helpers).

Weights are uint32 fixed point (w = w_fixed / 2^32) with every node's in-sum at most
2^32 - 1, as the LT model requires (in-weight sum <= 1, Sec. 2.1).
"""
import numpy as np

ONE = 0xFFFFFFFF  # largest representable in-sum (probability 1 - 2^-32)


def fx(p: float) -> int:
    """Fixed-point weight for probability p (truncated)."""
    return min(int(p * 4294967296.0), ONE)


def random_tiny(seed: int, n: int = 7, m: int = 12, allow_self_loops: bool = True):
    """Random directed graph with random in-weights whose per-node sum is in [0.3, 1]."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if not allow_self_loops:
        same = src == dst
        dst[same] = (dst[same] + 1) % n
    w = np.zeros(m, np.uint32)
    for v in range(n):
        idx = np.nonzero(dst == v)[0]
        if idx.size == 0:
            continue
        x = rng.random(idx.size) + 0.05
        total = rng.uniform(0.3, 1.0)
        ws = np.floor(x / x.sum() * total * 4294967295.0).astype(np.uint64)
        w[idx] = ws.astype(np.uint32)
    return n, src, dst, w


def world_count(n, dst):
    deg = np.bincount(dst, minlength=n)
    return int(np.prod(deg.astype(np.float64) + 1.0))
