"""Thread safety of the C ABI (calls are thread-safe per context): blocking
calls of every kind made from several host threads at once on one context, and
one user-function module used by two contexts at once, return exactly the
results of the same calls made one after another.  Each call is deterministic
(fixed Philox keys, fixed chunk order in the merge), so the comparison is bit
for bit."""
import threading

import numpy as np
import pytest

from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests.test_gpu_udf import HARMONIC_F32

pytestmark = pytest.mark.gpu

FIELDS = ("estimate", "stderr", "n", "status")


def _run_threads(fns):
    """Run each callable in a thread of its own, all started together."""
    results = [None] * len(fns)
    errors = []
    start = threading.Barrier(len(fns))

    def wrap(i):
        try:
            start.wait(timeout=60)
            results[i] = fns[i]()
        except BaseException as e:  # re-raised in the test's thread
            errors.append(e)

    threads = [threading.Thread(target=wrap, args=(i,)) for i in range(len(fns))]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=600)
    assert not any(th.is_alive() for th in threads), "a call did not return"
    if errors:
        raise errors[0]
    return results


def _same(a, b):
    for f in FIELDS:
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)


def _calls(ctx, rng):
    """Six independent calls of five kinds, each a closure returning a result table."""
    tabs = [W.random_table(200, rng, n_hi=400_000, seed=s) for s in (1, 2, 3)]
    mom = W.random_table(50, rng, n_hi=100_000, seed=4)
    s_end = (mom["n_samples"] // 8) * 4 + 4
    base = W.harmonic_fig1(10**5)[7]
    kappa = rng.uniform(-20.0, 20.0, size=(300, 4))
    udf_tab = W.harmonic_fig1(2 * 10**5, seeds=(5,))
    udf = zmc.Udf(HARMONIC_F32, 4, zmc.ZMC_UDF_F32, amplitude=2.0)
    udf_tab["family"] = W.USER
    return udf, [
        lambda: zmc.zmc_integrate(ctx, tabs[0]),
        lambda: zmc.zmc_integrate(ctx, tabs[1]),
        lambda: zmc.zmc_integrate_plain(ctx, tabs[2]),
        lambda: zmc.zmc_integrate_moments(ctx, mom, np.zeros(len(mom), np.uint64), s_end),
        lambda: zmc.zmc_integrate_functional(ctx, base, [zmc.slot_p(2 + i) for i in range(4)],
                                             kappa),
        lambda: udf.integrate(ctx, udf_tab),
    ]


def test_blocking_calls_from_many_threads_one_context(zctx):
    rng = np.random.default_rng(2024)
    udf, calls = _calls(zctx.handle, rng)
    serial = [c() for c in calls]
    for _ in range(3):
        got = _run_threads(calls)
        for a, b in zip(got, serial):
            if a.dtype.names and "estimate" in a.dtype.names:
                _same(a, b)
            else:  # moments records
                np.testing.assert_array_equal(a, b)
    udf.close()


def test_one_udf_module_two_contexts_at_once():
    """A module's cubin is loaded once (under the module's own lock) and then
    launched from two contexts on two streams concurrently."""
    udf = zmc.Udf(HARMONIC_F32, 4, zmc.ZMC_UDF_F32, amplitude=2.0)
    tabs = []
    for s in (11, 12):
        t = W.harmonic_fig1(3 * 10**5, seeds=(s,))
        t["family"] = W.USER
        tabs.append(t)
    with zmc.Context(arena_bytes=1 << 28) as c0, zmc.Context(arena_bytes=1 << 28) as c1:
        got = _run_threads([lambda: udf.integrate(c0.handle, tabs[0]),
                            lambda: udf.integrate(c1.handle, tabs[1])])
        serial = [udf.integrate(c1.handle, tabs[0]), udf.integrate(c0.handle, tabs[1])]
    for a, b in zip(got, serial):
        _same(a, b)
    udf.close()


@pytest.fixture(scope="module")
def sctx(zctx):
    c = zmc.Context(arena_bytes=1 << 30, serving=True, max_chunks_per_iter=4096)
    yield c
    c.close()


def test_serving_and_blocking_calls_interleaved(sctx, sq_ctx):
    """Threads submitting and polling serving jobs while others make blocking
    calls on a second context: every job equals the blocking call of its table
    on a context with the serving chunk length."""
    rng = np.random.default_rng(99)
    tabs = [W.random_table(120, rng, n_hi=300_000, seed=20 + k) for k in range(4)]
    want = [zmc.zmc_integrate(sq_ctx.handle, t) for t in tabs]

    def served(t):
        jid = zmc.zmc_submit(sctx.handle, t)
        st, out = zmc.zmc_poll(sctx.handle, jid, len(t), wait_ms=120_000)
        assert st == zmc.ZMC_OK, st
        return out

    def blocking(t):
        return zmc.zmc_integrate(sq_ctx.handle, t)

    calls = [lambda t=t: served(t) for t in tabs] + [lambda t=t: blocking(t) for t in tabs]
    got = _run_threads(calls)
    for k in range(4):
        _same(got[k], want[k])
        _same(got[4 + k], want[k])
