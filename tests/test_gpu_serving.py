"""Continuous batching through zmc_submit / zmc_poll (GPU)."""
import time

import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sctx():
    from paper_2104_10073_gb300 import build

    build.build()
    # small iterations so that jobs interleave across many launches, every launch
    # filled to its budget (no launch ends early at a job's last chunks)
    c = zmc.Context(arena_bytes=1 << 30, serving=True, max_chunks_per_iter=4096,
                    serving_cut_backlog=1)
    yield c
    c.close()


def _jobs(n_jobs, seed, max_fns=40, hi_exp=5.5):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n_jobs):
        t = W.random_table(int(rng.integers(1, max_fns + 1)), rng, n_lo=1,
                           n_hi=int(10**hi_exp), seed=j)
        jobs.append(t)
    return jobs


def test_results_same_alone_and_mixed(sctx, sq_ctx):
    jobs = _jobs(12, seed=3)
    # alone: one job at a time through the serving loop
    alone = []
    for t in jobs:
        jid = zmc.zmc_submit(sctx.handle, t)
        st, res = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=-1)
        assert st == zmc.ZMC_OK
        alone.append(res)
    # one job at a time never shares a launch
    assert zmc.zmc_serving_stats_get(sctx.handle)["max_jobs_per_iter"] == 1
    before = zmc.zmc_serving_stats_get(sctx.handle)
    # mixed: all submitted at once, interleaved over shared persistent launches
    ids = [zmc.zmc_submit(sctx.handle, t) for t in jobs]
    for t, jid, a in zip(jobs, ids, alone):
        st, res = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=-1)
        assert st == zmc.ZMC_OK
        assert np.array_equal(res["estimate"], a["estimate"])
        assert np.array_equal(res["stderr"], a["stderr"], equal_nan=True)
        assert np.array_equal(res["n"], a["n"]) and np.array_equal(res["status"], a["status"])
    after = zmc.zmc_serving_stats_get(sctx.handle)
    # the mixed phase really shared launches: work items of several jobs ran in
    # the same persistent launch (a scheduler that ran the jobs one after the
    # other would leave both counters where the alone phase left them)
    assert after["shared_iterations"] - before["shared_iterations"] >= 1
    assert after["max_jobs_per_iter"] >= 2
    # and the same as the blocking batched call with the same chunk length, and
    # the oracle
    for t, a in zip(jobs[:4], alone[:4]):
        one = zmc.zmc_integrate(sq_ctx.handle, t)
        assert np.array_equal(one["estimate"], a["estimate"])
        want, _ = oracle.integrate(t)
        G.compare(t, a, want)


def test_results_same_under_both_share_policies(sctx):
    """Oldest-first launches (the default) and equal shares give the same
    results bit for bit: a chunk's record does not depend on what shares its
    launch."""
    jobs = _jobs(8, seed=17)
    ids = [zmc.zmc_submit(sctx.handle, t) for t in jobs]
    first = [zmc.zmc_poll(sctx.handle, j, len(t), wait_ms=-1)[1] for j, t in zip(ids, jobs)]
    with zmc.Context(arena_bytes=1 << 30, serving=True, max_chunks_per_iter=4096,
                     serving_share=64) as eq:
        ids = [zmc.zmc_submit(eq.handle, t) for t in jobs]
        for j, t, a in zip(ids, jobs, first):
            st, res = zmc.zmc_poll(eq.handle, j, len(t), wait_ms=-1)
            assert st == zmc.ZMC_OK
            assert np.array_equal(res["estimate"], a["estimate"])
            assert np.array_equal(res["stderr"], a["stderr"], equal_nan=True)
        assert zmc.zmc_serving_stats_get(eq.handle)["shared_iterations"] >= 1


def test_short_backlog_ends_launches_at_job_ends(sctx):
    """Oldest first, launches end with the first job they complete while the
    backlog is short, and are filled (several jobs sharing one) while it is long;
    results are the same bit for bit under either rule."""
    # a long first job (2^32 samples, ~250 launches here) holds the GPU while the
    # others queue behind it, so the backlog is known when their launches are built
    blocker = W.empty(1)
    W.harmonic(blocker[0], 1.0, 0.5, [3.0], [0.0], [1.0], 2**32, seed=99)
    jobs = [blocker] + _jobs(10, seed=31, max_fns=40, hi_exp=6.0)
    ids = [zmc.zmc_submit(sctx.handle, t) for t in jobs]
    filled = [zmc.zmc_poll(sctx.handle, j, len(t), wait_ms=-1)[1] for j, t in zip(ids, jobs)]
    rest = sum(W.total_samples(t) for t in jobs[1:])
    # the library default (2^34 samples) is above this stream's whole backlog:
    # every launch ends at a job's end, so no launch holds chunks of two jobs
    with zmc.Context(arena_bytes=1 << 30, serving=True, max_chunks_per_iter=4096) as c:
        ids = [zmc.zmc_submit(c.handle, t) for t in jobs]
        for j, t, a in zip(ids, jobs, filled):
            st, res = zmc.zmc_poll(c.handle, j, len(t), wait_ms=-1)
            assert st == zmc.ZMC_OK
            assert np.array_equal(res["estimate"], a["estimate"])
            assert np.array_equal(res["stderr"], a["stderr"], equal_nan=True)
        stats = zmc.zmc_serving_stats_get(c.handle)
        assert stats["max_jobs_per_iter"] == 1 and stats["shared_iterations"] == 0
    # a threshold below the backlog behind the first job: the launches that
    # finish the first job and start the queued ones are filled and shared; the
    # last ones (short backlog) end at job ends
    with zmc.Context(arena_bytes=1 << 30, serving=True, max_chunks_per_iter=4096,
                     serving_cut_backlog=rest // 3) as c:
        ids = [zmc.zmc_submit(c.handle, t) for t in jobs]
        for j, t, a in zip(ids, jobs, filled):
            st, res = zmc.zmc_poll(c.handle, j, len(t), wait_ms=-1)
            assert st == zmc.ZMC_OK
            assert np.array_equal(res["estimate"], a["estimate"])
        stats = zmc.zmc_serving_stats_get(c.handle)
        assert stats["shared_iterations"] >= 1
        assert stats["iterations"] > stats["shared_iterations"]


def test_poll_semantics(sctx):
    t = W.mixed(50, gen_seed=9, lo_exp=5.5, hi_exp=6.5)
    jid = zmc.zmc_submit(sctx.handle, t)
    st, _ = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=0)
    assert st in (zmc.ZMC_EAGAIN, zmc.ZMC_OK)
    if st == zmc.ZMC_OK:
        pytest.skip("job finished before the first poll")
    st, res = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=-1)
    assert st == zmc.ZMC_OK and res is not None
    st, _ = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=0)
    assert st == zmc.ZMC_ENOTFOUND
    st, _ = zmc.zmc_poll(sctx.handle, 987654321, 1, wait_ms=0)
    assert st == zmc.ZMC_ENOTFOUND


def test_timeout_then_complete(sctx):
    t = W.mixed(200, gen_seed=10, lo_exp=6.5, hi_exp=7.0)
    jid = zmc.zmc_submit(sctx.handle, t)
    st, _ = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=1)
    assert st in (zmc.ZMC_ETIMEOUT, zmc.ZMC_OK)
    if st != zmc.ZMC_OK:
        st, _ = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=60000)
    assert st == zmc.ZMC_OK


def test_cancel(sctx):
    big = W.mixed(300, gen_seed=11, lo_exp=6.5, hi_exp=7.0)
    jid = zmc.zmc_submit(sctx.handle, big)
    zmc.zmc_cancel(sctx.handle, jid)
    st, _ = zmc.zmc_poll(sctx.handle, jid, len(big), wait_ms=-1)
    assert st in (zmc.ZMC_ECLOSED, zmc.ZMC_OK)
    # the loop keeps serving after a cancellation
    small = W.harmonic_fig1(1000)[:5]
    jid = zmc.zmc_submit(sctx.handle, small)
    st, res = zmc.zmc_poll(sctx.handle, jid, len(small), wait_ms=-1)
    assert st == zmc.ZMC_OK
    want, _ = oracle.integrate(small)
    G.compare(small, res, want)


def test_job_larger_than_budget_is_refused():
    with zmc.Context(arena_bytes=64 << 20, serving=True) as c:
        t = W.empty(1)
        W.harmonic(t[0], 1.0, 1.0, [1.0], [0.0], [1.0], 2**36)  # 2^24 chunks, 128 MiB of records
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_submit(c.handle, t)
        assert e.value.status == zmc.ZMC_ENOMEM


def test_admission_waits_for_memory():
    """Jobs that do not all fit at once are admitted as earlier ones finish."""
    with zmc.Context(arena_bytes=12 << 20, serving=True, max_chunks_per_iter=4096) as c:
        chunk = 160 * zmc.SERVING_QUINTS_PER_LANE
        n = 2**31 // chunk * chunk  # 2^31 samples: 4 MiB of chunk records per job
        jobs = []
        for j in range(12):
            t = W.empty(1)
            W.harmonic(t[0], 1.0, 0.5, [3.0, 1.0], [0.0, 0.0], [1.0, 1.0], n, seed=j)
            jobs.append(t)
        ids = [zmc.zmc_submit(c.handle, t) for t in jobs]
        stats = zmc.zmc_serving_stats_get(c.handle)
        assert stats["queued"] >= 1  # 12 x 4 MiB cannot all be admitted into 12 MiB
        res = [zmc.zmc_poll(c.handle, i, 1, wait_ms=120000) for i in ids]
        assert all(st == zmc.ZMC_OK for st, _ in res)
        stats = zmc.zmc_serving_stats_get(c.handle)
        assert stats["completed"] >= 12


def test_poisson_stream_latency_recorded(sctx):
    jobs = _jobs(30, seed=5, max_fns=20)
    t0 = time.perf_counter()
    ids = []
    for t in jobs:
        ids.append((zmc.zmc_submit(sctx.handle, t), len(t), time.perf_counter()))
        time.sleep(0.002)
    lat = []
    for jid, n, ts in ids:
        st, _ = zmc.zmc_poll(sctx.handle, jid, n, wait_ms=-1)
        assert st == zmc.ZMC_OK
        lat.append(time.perf_counter() - ts)
    assert max(lat) < 60.0 and time.perf_counter() - t0 < 120.0


def test_injected_iteration_failure_poisons_context(monkeypatch):
    """A failure injected on the host at the first iteration fails the pending
    jobs with ZMC_ECUDA, poisons the context, and leaves the GPU usable."""
    monkeypatch.setenv("ZMC_SERVING_FAULT_AT", "1")
    c = zmc.Context(arena_bytes=128 << 20, serving=True)
    monkeypatch.delenv("ZMC_SERVING_FAULT_AT")
    try:
        t = W.harmonic_fig1(2000)[:10]
        jid = zmc.zmc_submit(c.handle, t)
        st, res = zmc.zmc_poll(c.handle, jid, len(t), wait_ms=30000)
        assert st == zmc.ZMC_ECUDA and res is None
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_integrate(c.handle, t)
        assert e.value.status == zmc.ZMC_ECUDA
    finally:
        c.close()
    with zmc.Context(arena_bytes=64 << 20) as ok:
        got = zmc.zmc_integrate(ok.handle, t)
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)


def test_poll_any_reports_each_finished_job_once(sctx):
    jobs = _jobs(8, seed=21, max_fns=10, hi_exp=4.5)
    ids = {zmc.zmc_submit(sctx.handle, t): len(t) for t in jobs}
    seen = []
    while len(seen) < len(ids):
        st, got = zmc.zmc_poll_any(sctx.handle, 3, 30000)
        assert st in (zmc.ZMC_OK, zmc.ZMC_EAGAIN) and len(got) <= 3
        seen += got
    assert sorted(seen) == sorted(ids)
    for jid, n in ids.items():
        st, res = zmc.zmc_poll(sctx.handle, jid, n, wait_ms=0)
        assert st == zmc.ZMC_OK and res is not None
    st, got = zmc.zmc_poll_any(sctx.handle, 4, 0)
    assert st == zmc.ZMC_EAGAIN and got == []
