"""Host-side helpers of bench.py (no GPU)."""
import math

import bench


def test_serve_pool_sizes():
    assert bench.serve_pool_sizes(0, [1 << 18, 1 << 20]) == [0, 0]
    assert bench.serve_pool_sizes(1 << 29, [1 << 18, 1 << 20]) == [1 << 27, 1 << 29]
    # whole blocks of 2^22, at least one block
    assert bench.serve_pool_sizes(1 << 29, [1000, 1 << 20]) == [1 << 22, 1 << 29]
    assert all(x % (1 << 22) == 0 for x in bench.serve_pool_sizes(3 * 10 ** 8, [123457, 999999, 1 << 20]))


def test_same_result_ignores_steps_and_matches_nan():
    a = {"hits": 10, "attempts": 99, "steps": 5, "eps_t": math.nan}
    assert bench.same_result(a, dict(a, steps=7))
    assert not bench.same_result(a, dict(a, attempts=98))
    assert not bench.same_result(a, dict(a, eps_t=0.1))
    assert bench.same_result(dict(a, eps_t=0.25), dict(a, eps_t=0.25))
