"""bench.py's model of the serving launch loop (launch_model), on the CPU.

The model explains the measured serving latencies: launches of a fixed cost plus
their samples at the kernels' rate, filled oldest job first and ended at the
first completed job under a short backlog, two launches in flight.  These tests
check it on streams small enough to work out by hand, and against the ideal
oldest-first server (fifo_bound), which it can never beat.
"""
import numpy as np
import pytest

import bench

CS = 4160


def job(at, chunks):
    return (at, chunks * CS, chunks)


def test_one_job_on_an_idle_server():
    cap = 100.0  # G samples/s delivered by full launches
    budget = 2**31 // CS
    rate = budget * CS / (budget * CS / (cap * 1e9) - 52e-6)
    m = bench.launch_model([job(0.0, 1000)], cap)
    want = 30e-6 + 52e-6 + 1000 * CS / rate
    assert m["p50_ms"] == pytest.approx(1e3 * want) and m["p99_ms"] == pytest.approx(1e3 * want)


def test_short_backlog_gives_each_job_its_own_launch():
    cap = 100.0
    budget = 2**31 // CS
    rate = budget * CS / (budget * CS / (cap * 1e9) - 52e-6)
    two = [job(0.0, 1000), job(0.0, 500)]
    # both built at once (two slots), the second launch right behind the first
    t1 = 30e-6 + 52e-6 + 1000 * CS / rate
    t2 = t1 + 52e-6 + 500 * CS / rate
    m = bench.launch_model(two, cap)
    assert m["p99_ms"] == pytest.approx(1e3 * t2)
    assert m["p50_ms"] == pytest.approx(1e3 * t2)  # upper median of two
    # with every launch filled (cut_backlog 0) both jobs share one launch and
    # finish together, one fixed cost sooner for the second
    f = bench.launch_model(two, cap, cut_backlog=0)
    t = 30e-6 + 52e-6 + 1500 * CS / rate
    assert f["p99_ms"] == pytest.approx(1e3 * t)


def test_launch_budget_splits_a_long_job():
    cap = 100.0
    budget = 100000  # 4.2 ms launches at 100 G samples/s
    m = bench.launch_model([job(0.0, 250000)], cap, budget_samples=budget * CS)
    full = budget * CS / (cap * 1e9)
    rate = budget * CS / (full - 52e-6)
    # three launches (100000, 100000, 50000 chunks) back to back
    want = 30e-6 + 3 * 52e-6 + 250000 * CS / rate
    assert m["p99_ms"] == pytest.approx(1e3 * want)


@pytest.mark.parametrize("seed", range(5))
def test_never_better_than_the_ideal_oldest_first_server(seed):
    rng = np.random.default_rng(seed)
    at = np.cumsum(rng.exponential(1 / 300.0, size=400))
    chunks = rng.integers(1, 200000, size=400)
    jobs = [(float(a), int(c) * CS, int(c)) for a, c in zip(at, chunks)]
    cap = 360.0
    ideal = bench.fifo_bound([(a, s) for a, s, _ in jobs], cap)
    for cut in (0, 2**34):
        m = bench.launch_model(jobs, cap, cut_backlog=cut)
        assert m["p50_ms"] >= ideal["p50_ms"] and m["p99_ms"] >= ideal["p99_ms"]
