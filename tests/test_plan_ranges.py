"""The persistent solver's tile-range planner (host logic, no GPU; the device
re-plans a batch with the same function): every tile in exactly one
contiguous range, at most max_blocks ranges, at most 8 systems a range,
the smallest chunk that fits, and each system's record slots (the ranges
its tiles fall in) consistent with the ranges."""
import ctypes

import numpy as np
import pytest

from paper_2604_01800_gb300 import _lib

SMAX = 8


def plan(ntiles, max_blocks, max_ranges=4096):
    lib = _lib.load(build_if_missing=False)
    n = len(ntiles)
    nt = np.ascontiguousarray(ntiles, dtype=np.int32)
    tile0, blk0, nparts, part0 = (np.zeros(n, np.int32) for _ in range(4))
    ranges = np.zeros((max_ranges, 4), np.int32)
    nr, ns = ctypes.c_int(), ctypes.c_int()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = lib.ppe_debug_plan_ranges(n, p(nt), max_blocks, max_ranges, p(tile0), p(blk0), p(nparts), p(part0),
                                   p(ranges), ctypes.byref(nr), ctypes.byref(ns))
    assert st == 0
    return nr.value, ns.value, tile0, blk0, nparts, part0, ranges[:max(nr.value, 0)]


def system_of(tile0, ntiles, t):
    """The system that holds tile t (systems without tiles hold none)."""
    for s in range(len(ntiles)):
        if tile0[s] <= t < tile0[s] + ntiles[s]:
            return s
    raise AssertionError(t)


def min_ranges(ntiles):
    """Ranges the system limit alone forces (the planner's largest chunk)."""
    tile0 = np.concatenate([[0], np.cumsum(ntiles)[:-1]])
    total, t, n = sum(ntiles), 0, 0
    while t < total:
        s = system_of(tile0, ntiles, t)
        t = tile0[s + SMAX] if s + SMAX < len(ntiles) else total
        n += 1
    return n


def check(ntiles, max_blocks, max_ranges=4096):
    ntiles = list(ntiles)
    total = sum(ntiles)
    nr, ns, tile0, blk0, nparts, part0, R = plan(ntiles, max_blocks, max_ranges)
    assert list(tile0) == list(np.concatenate([[0], np.cumsum(ntiles)[:-1]]))
    if total == 0:
        assert nr == 0 and ns == 0 and all(nparts == 0)
        return
    if nr == -1:
        # only when the system limit alone needs more ranges than allowed
        assert min_ranges(ntiles) > min(max_blocks, max_ranges)
        return
    assert 1 <= nr <= min(max_blocks, max_ranges)
    # contiguous cover of [0, total)
    assert R[0, 0] == 0 and R[-1, 1] == total
    assert all(R[1:, 0] == R[:-1, 1]) and all(R[:, 1] > R[:, 0])
    # each range names the systems of its first and last tile, at most SMAX of them
    for t0, t1, s0, s1 in R:
        assert s0 == system_of(tile0, ntiles, t0) and s1 == system_of(tile0, ntiles, t1 - 1)
        assert s1 - s0 + 1 <= SMAX
    # the smallest chunk: one tile fewer per range would need more ranges than blocks
    chunk = int((R[:, 1] - R[:, 0]).max())
    assert chunk >= -(-total // max_blocks)
    # record slots: the ranges whose system span includes s, contiguous from blk0
    slots = 0
    for s in range(len(ntiles)):
        inside = [b for b, (_, _, s0, s1) in enumerate(R) if s0 <= s <= s1]
        if not inside:
            assert nparts[s] == 0 and ntiles[s] == 0
        else:
            assert blk0[s] == inside[0] and nparts[s] == len(inside) == inside[-1] - inside[0] + 1
        assert part0[s] == slots
        slots += nparts[s]
    assert ns == slots


@pytest.mark.parametrize("ntiles,max_blocks", [
    ([32], 152), ([32], 5), ([1], 1), ([5, 7, 9], 152), ([128], 152),
    ([0, 4, 0, 9], 3), ([3] * 40, 10), ([1] * 64, 152),
])
def test_plans(ntiles, max_blocks):
    check(ntiles, max_blocks)


def test_random_batches():
    g = np.random.default_rng(5)
    for _ in range(200):
        n = int(g.integers(1, 70))
        nt = g.integers(0, 60, n)
        nt[g.random(n) < 0.1] = 0
        check(nt, int(g.integers(1, 200)))


def test_all_empty_and_capacity():
    check([0, 0, 0], 4)
    # 20 systems fit in 3 ranges of at most 8 systems: the chunk grows to fit
    check([10] * 20, 152, max_ranges=3)
    assert plan([10] * 20, 152, max_ranges=3)[0] == 3
    # 40 systems need at least 5 ranges
    assert plan([1] * 40, 152, max_ranges=3)[0] == -1
    assert plan([1] * 40, 4)[0] == -1
