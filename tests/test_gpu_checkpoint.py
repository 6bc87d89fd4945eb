"""Checkpoint and resume of serving jobs through zmc_checkpoint / zmc_submit_resume (GPU).

Every sample is addressed by its Philox counter, so the moments of the first n
samples of a stream plus a job that samples [n, N) of it reproduce the
uninterrupted run: the chunk records are the same, only the final FP64
combination differs (pairwise update instead of one k-way merge).
"""
import time

import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

CHUNK = 160 * zmc.SERVING_QUINTS_PER_LANE  # samples per chunk of a serving context


@pytest.fixture(scope="module")
def sctx():
    from paper_2104_10073_gb300 import build

    build.build()
    # small iterations so that a job spans many launches
    c = zmc.Context(arena_bytes=1 << 30, serving=True, max_chunks_per_iter=1024)
    yield c
    c.close()


def _close(got, want, table, rel=1e-12):
    """Estimates and standard errors equal up to FP64 rounding of the merge."""
    for g, w in zip(got, want):
        # |estimate| + V sigma_f: the size of the sums the merge rounds
        scale = abs(w["estimate"]) + w["stderr"] * np.sqrt(float(w["n"])) + 1e-300
        assert abs(g["estimate"] - w["estimate"]) <= rel * scale, (g, w)
        assert abs(g["stderr"] - w["stderr"]) <= 1e-9 * abs(w["stderr"]), (g, w)
        assert g["n"] == w["n"]


def _big_job(n_fn=6, n_samples=1 << 27, seed=0):
    rng = np.random.default_rng(seed)
    t = W.random_table(n_fn, rng, n_lo=1, n_hi=10, seed=seed)
    t["n_samples"] = n_samples
    return t


def _checkpoint_mid_run(sctx, t, delay_s):
    jid = zmc.zmc_submit(sctx.handle, t)
    time.sleep(delay_s)
    st, ck = zmc.zmc_checkpoint(sctx.handle, jid, len(t), wait_ms=30000)
    return jid, st, ck


def test_checkpoint_moments_equal_prefix_moments(sctx, sq_ctx):
    """A checkpoint's moments are those of the first n samples of each stream,
    bit for bit the same as zmc_integrate_moments over [0, n)."""
    t = _big_job(seed=1)
    jid, st, ck = _checkpoint_mid_run(sctx, t, 0.004)
    if st == zmc.ZMC_EAGAIN:
        pytest.skip("job issued all of its samples before the checkpoint")
    assert st == zmc.ZMC_OK
    n = ck["n"].astype(np.int64)
    assert np.all((n % CHUNK == 0) | (n == t["n_samples"]))
    assert np.all(n <= t["n_samples"])
    assert np.any((n > 0) & (n < t["n_samples"])), n
    # the id is released
    st2, _ = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=0)
    assert st2 == zmc.ZMC_ENOTFOUND
    rows = n > 0
    ref = zmc.zmc_integrate_moments(sq_ctx.handle, t[rows], np.zeros(rows.sum()), n[rows])
    assert np.array_equal(ck["mean"][rows], ref["mean"])
    assert np.array_equal(ck["m2"][rows], ref["m2"])
    assert np.all(ck["mean"][~rows] == 0) and np.all(ck["m2"][~rows] == 0)


@pytest.mark.parametrize("delay_s", [0.0, 0.002, 0.01])
def test_resume_equals_uninterrupted(sctx, sq_ctx, delay_s):
    t = _big_job(seed=2)
    want = zmc.zmc_integrate(sq_ctx.handle, t)
    jid, st, ck = _checkpoint_mid_run(sctx, t, delay_s)
    if st == zmc.ZMC_EAGAIN:
        st, got = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=120000)
        assert st == zmc.ZMC_OK
        assert np.array_equal(got["estimate"], want["estimate"])
        return
    assert st == zmc.ZMC_OK
    rid = zmc.zmc_submit_resume(sctx.handle, t, ck)
    st, got = zmc.zmc_poll(sctx.handle, rid, len(t), wait_ms=120000)
    assert st == zmc.ZMC_OK
    _close(got, want, t)


def test_chain_of_checkpoints_and_migration(sctx, sq_ctx):
    """Checkpoint, resume on another context, checkpoint again, resume back."""
    t = _big_job(n_fn=4, n_samples=1 << 28, seed=3)
    want = zmc.zmc_integrate(sq_ctx.handle, t)
    with zmc.Context(arena_bytes=1 << 30, serving=True, max_chunks_per_iter=1024) as other:
        jid, st, ck1 = _checkpoint_mid_run(sctx, t, 0.003)
        if st == zmc.ZMC_EAGAIN:  # finished before the checkpoint: nothing to chain
            st, got = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=120000)
            assert st == zmc.ZMC_OK
            assert np.array_equal(got["estimate"], want["estimate"])
            return
        assert st == zmc.ZMC_OK
        rid = zmc.zmc_submit_resume(other.handle, t, ck1)
        time.sleep(0.003)
        st, ck2 = zmc.zmc_checkpoint(other.handle, rid, len(t), wait_ms=30000)
        if st == zmc.ZMC_EAGAIN:
            st, got = zmc.zmc_poll(other.handle, rid, len(t), wait_ms=120000)
            assert st == zmc.ZMC_OK
            _close(got, want, t)
            return
        assert st == zmc.ZMC_OK
        assert np.all(ck2["n"] >= ck1["n"])
    rid = zmc.zmc_submit_resume(sctx.handle, t, ck2)
    st, got = zmc.zmc_poll(sctx.handle, rid, len(t), wait_ms=120000)
    assert st == zmc.ZMC_OK
    _close(got, want, t)


def test_checkpoint_of_queued_job():
    """A job still waiting for memory is released with its starting moments."""
    with zmc.Context(arena_bytes=128 << 20, serving=True) as c:
        big = W.empty(1)
        W.harmonic(big[0], 1.0, 0.5, [3.0, 1.0], [0.0, 0.0], [1.0, 1.0], 1 << 34, seed=9)
        a = zmc.zmc_submit(c.handle, big)
        # 64 MiB of chunk records each, next to ~13 MiB of iteration tables: b
        # waits for a's memory
        b = zmc.zmc_submit(c.handle, big)
        st, ck = zmc.zmc_checkpoint(c.handle, b, 1, wait_ms=30000)
        assert st in (zmc.ZMC_OK, zmc.ZMC_EAGAIN)
        if st == zmc.ZMC_OK:
            assert ck["n"][0] % CHUNK == 0
        zmc.zmc_cancel(c.handle, a)
        st, _ = zmc.zmc_poll(c.handle, a, 1, wait_ms=120000)
        assert st in (zmc.ZMC_ECLOSED, zmc.ZMC_OK)


def test_resume_from_moments_matches_oracle(sctx, sq_ctx):
    """Resume from zmc_integrate_moments over [0, n) for ragged n (multiples of 4,
    not of the chunk), every family; the result matches the FP64 oracle."""
    rng = np.random.default_rng(11)
    t = W.random_table(40, rng, n_lo=4, n_hi=300000, seed=4)
    n_all = t["n_samples"].astype(np.int64)
    n0 = rng.integers(0, n_all + 1) // 5 * 5
    n0[::7] = n_all[::7]  # some rows are complete already (any n_samples)
    n0[1::9] = 0          # some start afresh
    from_m = np.zeros(len(t), dtype=zmc.MOMENTS_DTYPE)
    rows = n0 > 0
    from_m[rows] = zmc.zmc_integrate_moments(sq_ctx.handle, t[rows], np.zeros(rows.sum()),
                                             n0[rows])
    rid = zmc.zmc_submit_resume(sctx.handle, t, from_m)
    st, got = zmc.zmc_poll(sctx.handle, rid, len(t), wait_ms=120000)
    assert st == zmc.ZMC_OK
    assert np.array_equal(got["n"], t["n_samples"])
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)


def test_resume_with_nothing_left(sctx, sq_ctx):
    t = W.harmonic_fig1(50000)[:8]
    full = zmc.zmc_integrate_moments(sq_ctx.handle, t, np.zeros(len(t)), t["n_samples"])
    rid = zmc.zmc_submit_resume(sctx.handle, t, full)
    st, got = zmc.zmc_poll(sctx.handle, rid, len(t), wait_ms=120000)
    assert st == zmc.ZMC_OK
    want = zmc.zmc_integrate(sq_ctx.handle, t)
    _close(got, want, t)


def test_resume_rejects_bad_moments(sctx):
    t = W.harmonic_fig1(1000)[:2]
    m = np.zeros(2, dtype=zmc.MOMENTS_DTYPE)
    m["n"] = [1004, 0]  # beyond n_samples
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_submit_resume(sctx.handle, t, m)
    assert e.value.status == zmc.ZMC_EINVAL
    m["n"] = [6, 0]  # not a multiple of 5
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_submit_resume(sctx.handle, t, m)
    assert e.value.status == zmc.ZMC_EINVAL
    m["n"] = [10, 0]
    m["m2"] = [-1.0, 0.0]
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_submit_resume(sctx.handle, t, m)
    assert e.value.status == zmc.ZMC_EINVAL


def test_checkpoint_after_completion_is_refused(sctx):
    t = W.harmonic_fig1(4000)[:3]
    jid = zmc.zmc_submit(sctx.handle, t)
    while True:
        st, ids = zmc.zmc_poll_any(sctx.handle, 64, 30000)
        assert st in (zmc.ZMC_OK, zmc.ZMC_EAGAIN)
        if jid in ids:
            break
    st, _ = zmc.zmc_checkpoint(sctx.handle, jid, len(t), wait_ms=0)
    assert st == zmc.ZMC_EAGAIN
    st, res = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=0)
    assert st == zmc.ZMC_OK and np.all(res["status"] == 0)
    st, _ = zmc.zmc_checkpoint(sctx.handle, 987654321, 1, wait_ms=0)
    assert st == zmc.ZMC_ENOTFOUND


def test_resume_combines_the_given_moments(sctx, sq_ctx):
    """The resumed result is Chan's combination of the moments passed in with the
    moments of samples [n, N): planted prior moments (not those of the stream)
    show up in the result exactly as the pairwise update predicts."""
    rng = np.random.default_rng(5)
    t = W.random_table(12, rng, n_lo=20000, n_hi=200000, seed=8)
    n_all = t["n_samples"].astype(np.int64)
    na = n_all // 3 // 5 * 5
    prior = np.zeros(len(t), dtype=zmc.MOMENTS_DTYPE)
    prior["n"] = na
    prior["mean"] = rng.uniform(-3.0, 3.0, len(t))
    prior["m2"] = rng.uniform(0.0, 50.0, len(t))
    rid = zmc.zmc_submit_resume(sctx.handle, t, prior)
    st, got = zmc.zmc_poll(sctx.handle, rid, len(t), wait_ms=120000)
    assert st == zmc.ZMC_OK
    rest = zmc.zmc_integrate_moments(sq_ctx.handle, t, na, n_all)
    vol = np.array([np.prod(r["hi"][:r["dim"]] - r["lo"][:r["dim"]]) for r in t])
    nb = n_all - na
    d = rest["mean"] - prior["mean"]
    mean = prior["mean"] + d * (nb / n_all)
    m2 = prior["m2"] + rest["m2"] + d * d * (na * nb / n_all)
    est = vol * mean
    se = vol * np.sqrt(m2 / (n_all * (n_all - 1.0)))
    assert np.array_equal(got["n"], n_all.astype(np.uint64))
    assert np.allclose(got["estimate"], est, rtol=1e-13, atol=1e-15 * np.abs(vol).max())
    assert np.allclose(got["stderr"], se, rtol=1e-12)


def test_concurrent_submitters_with_checkpoints(sctx, sq_ctx):
    """Four host threads submit, checkpoint, resume and collect jobs on one
    serving context at the same time; every final result equals the blocking
    call's within FP64 rounding of the merge."""
    import threading

    tables = [_big_job(n_fn=3, n_samples=(1 << 25) + 4096 * k, seed=50 + k) for k in range(8)]
    want = [zmc.zmc_integrate(sq_ctx.handle, t) for t in tables]
    errors = []

    def worker(w):
        try:
            for k in range(w, len(tables), 4):
                t = tables[k]
                jid = zmc.zmc_submit(sctx.handle, t)
                time.sleep(0.001 * (k % 3))
                st, ck = zmc.zmc_checkpoint(sctx.handle, jid, len(t), wait_ms=60000)
                if st == zmc.ZMC_OK:
                    jid = zmc.zmc_submit_resume(sctx.handle, t, ck)
                else:
                    assert st == zmc.ZMC_EAGAIN, st
                st, got = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=120000)
                assert st == zmc.ZMC_OK, st
                _close(got, want[k], t)
        except BaseException as e:  # reported on the main thread
            errors.append((w, repr(e)))

    threads = [threading.Thread(target=worker, args=(w,)) for w in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(300)
    assert not any(th.is_alive() for th in threads)
    assert not errors, errors


def test_cancel_during_checkpoint_and_shutdown():
    """A job cancelled while its checkpoint is pending reports ZMC_ECLOSED, and a
    context destroyed with jobs and checkpoints outstanding shuts down cleanly."""
    with zmc.Context(arena_bytes=1 << 30, serving=True, max_chunks_per_iter=256) as c:
        t = _big_job(n_fn=4, n_samples=1 << 28, seed=77)
        jid = zmc.zmc_submit(c.handle, t)
        time.sleep(0.002)
        st, _ = zmc.zmc_checkpoint(c.handle, jid, len(t), wait_ms=0)
        assert st in (zmc.ZMC_EAGAIN, zmc.ZMC_OK)
        if st == zmc.ZMC_EAGAIN:
            zmc.zmc_cancel(c.handle, jid)
            st, _ = zmc.zmc_checkpoint(c.handle, jid, len(t), wait_ms=60000)
            # cancelled while pending (the usual case), or finished / taken first
            assert st in (zmc.ZMC_ECLOSED, zmc.ZMC_OK, zmc.ZMC_ENOTFOUND, zmc.ZMC_EAGAIN)
        # leave work behind: the context must still close
        for k in range(3):
            zmc.zmc_submit(c.handle, _big_job(n_fn=2, n_samples=1 << 27, seed=80 + k))
