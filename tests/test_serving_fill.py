"""The serving scheduler's launch fill rule (zmc_serving_fill), on the CPU.

The rule decides how many chunks each live job (oldest first) contributes to
one persistent launch.  The library's scheduler calls the same function; here it
is checked against hand-worked cases and against a plain restatement of the
rule on random inputs.  No GPU is needed.
"""
import numpy as np
import pytest

from paper_2104_10073_gb300 import zmc

CS = 4160  # samples per serving chunk (26 quints)


def fill(left, budget, share=0, cut=0):
    return [int(x) for x in zmc.zmc_serving_fill(left, budget, share, cut, CS)]


def restated(left, budget, share, cut_backlog, chunk_samples):
    """The rule as zmc.h states it, written out plainly."""
    take = [0] * len(left)
    if share == 0:
        backlog = sum(x * chunk_samples for x in left)  # Python integers: no overflow
        cut = backlog < cut_backlog
        for i, x in enumerate(left):
            if budget == 0:
                break
            take[i] = min(x, budget)
            budget -= take[i]
            if cut and 0 < take[i] == x:
                break
        return take
    active = [i for i, x in enumerate(left) if x > 0]
    while budget > 0 and active:
        per = max(share, budget // len(active))
        still = []
        for i in active:
            t = min(per, budget, left[i] - take[i])
            take[i] += t
            budget -= t
            if take[i] < left[i]:
                still.append(i)
            if budget == 0:
                break
        active = still
    return take


def test_oldest_first_fills_the_budget_in_arrival_order():
    assert fill([5, 3, 10], 6) == [5, 1, 0]
    assert fill([5, 3, 10], 100) == [5, 3, 10]
    assert fill([5, 3, 10], 0) == [0, 0, 0]
    assert fill([], 10) == []


def test_short_backlog_ends_the_launch_at_the_first_completed_job():
    backlog = 18 * CS
    # below the threshold: the oldest job completes, the launch ends there
    assert fill([5, 3, 10], 100, cut=backlog + 1) == [5, 0, 0]
    # a job that does not complete in this launch takes the whole budget
    assert fill([50, 3, 10], 20, cut=10**18) == [20, 0, 0]
    # at or above the threshold every launch is filled
    assert fill([5, 3, 10], 100, cut=backlog) == [5, 3, 10]
    assert fill([5, 3, 10], 7, cut=backlog) == [5, 2, 0]
    # 0 never cuts
    assert fill([5, 3, 10], 100, cut=0) == [5, 3, 10]


def test_equal_shares():
    # one pass: max(2, 9 // 3) = 3 each
    assert fill([5, 3, 10], 9, share=2) == [3, 3, 3]
    # pass 1 gives max(1, 12 // 3) = 4 each (the second job has 3); pass 2 hands
    # the one chunk left to the oldest job with work left
    assert fill([5, 3, 10], 12, share=1) == [5, 3, 4]
    # the floor wins over an equal split: the oldest jobs get it first
    assert fill([100, 100, 100], 100, share=64) == [64, 36, 0]
    # the threshold plays no part with shares
    assert fill([5, 3, 10], 100, share=1, cut=10**18) == [5, 3, 10]


def test_backlog_saturates_instead_of_wrapping():
    # 2^63 chunks of 4160 samples overflow 64 bits (wrapped, 2^63 * 4160 is 0
    # mod 2^64): the backlog must read as huge (no cut: the second job also
    # gets chunks), not wrap around to something small
    assert fill([1, 2**63], 10, cut=2**63) == [1, 9]


@pytest.mark.parametrize("seed", range(20))
def test_matches_the_stated_rule_on_random_inputs(seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        n = int(rng.integers(0, 12))
        left = [int(x) for x in rng.integers(0, 2000, size=n)]
        budget = int(rng.integers(0, 8000))
        share = int(rng.choice([0, 0, 1, 7, 64, 500]))
        cut = int(rng.choice([0, 1, 10**5, 10**6, 10**7, 10**18]))
        got = fill(left, budget, share, cut)
        assert got == restated(left, budget, share, cut, CS), (left, budget, share, cut)
        assert sum(got) <= budget and all(0 <= g <= x for g, x in zip(got, left))


def test_rejects_bad_arguments():
    lib = zmc.lib()
    take = np.zeros(1, dtype=np.uint64)
    left = np.ones(1, dtype=np.uint64)
    assert lib.zmc_serving_fill(None, 1, 10, 0, 0, CS, take.ctypes.data) == zmc.ZMC_EINVAL
    assert lib.zmc_serving_fill(left.ctypes.data, 1, 10, 0, 0, 0, take.ctypes.data) == zmc.ZMC_EINVAL
    assert lib.zmc_serving_fill(None, 0, 10, 0, 0, CS, None) == zmc.ZMC_OK
