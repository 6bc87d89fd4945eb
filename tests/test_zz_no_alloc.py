"""zmc_integrate_noalloc: the entry point for callers that cannot allocate.

Some callers may not allocate device memory at the moment they need a result
(a framework whose pool owns the device memory, a latency-bound loop, code
without a library context).  The no-allocation entry point keeps all of its
working memory in a fixed array inside the library; the caller passes only the
descriptor table and a device array for the results.  The test calls it through
the C ABI twice in a row on one stream, without waiting in between (the second
call rewrites the shared array behind the first call's queued kernels, which
only stream order keeps apart), each call writing its own output.  Both results
must equal the regular zmc_integrate entry point's bit for bit (same chunk
length, same records, same fixed-order merge), and separately match the FP64
oracle's own estimates within the parity tolerances (tests/gpu_common.py).
The file sorts last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import build
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


def _tables():
    a = W.random_table(40, np.random.default_rng(0), n_lo=1, n_hi=60000)
    b = np.concatenate([W.harmonic_fig1(10**5)[:50],
                        W.mixed(60, gen_seed=9, lo_exp=3.0, hi_exp=5.5)])
    return [a, b]


def test_noalloc_matches_integrate_two_calls_in_a_row():
    import torch

    build.build()
    tables = _tables()
    with zmc.Context(arena_bytes=256 << 20) as ctx:
        refs = [zmc.zmc_integrate(ctx.handle, t) for t in tables]
    stream = torch.cuda.Stream()
    # the caller owns the outputs; fill them with garbage to see them overwritten
    outs = [torch.full((len(t) * zmc.RESULT_DTYPE.itemsize,), 0xFF, dtype=torch.uint8,
                       device="cuda") for t in tables]
    torch.cuda.synchronize()
    for t, out in zip(tables, outs):
        st = zmc.zmc_integrate_noalloc(t, out.data_ptr(), stream.cuda_stream)
        assert st == zmc.ZMC_OK, zmc.zmc_last_error()
    stream.synchronize()
    for t, out, ref in zip(tables, outs, refs):
        got = out.cpu().numpy().view(zmc.RESULT_DTYPE)
        # the same computation as zmc_integrate: equal bit for bit
        assert np.array_equal(got["estimate"], ref["estimate"])
        assert np.array_equal(got["stderr"], ref["stderr"], equal_nan=True)
        assert np.array_equal(got["n"], ref["n"])
        assert np.array_equal(got["status"], ref["status"])
        # and, independently, the FP64 oracle on the same Philox samples
        want, _ = oracle.integrate(t)
        G.compare(t, got, want)


def test_noalloc_rejects_requests_beyond_its_fixed_size():
    import torch

    build.build()
    out = torch.zeros(32 * 4100, dtype=torch.uint8, device="cuda")
    too_many = np.repeat(W.harmonic_fig1(10)[:1], 4097)
    st = zmc.zmc_integrate_noalloc(too_many, out.data_ptr(), None)
    assert st == zmc.ZMC_EINVAL and "at most" in zmc.zmc_last_error()
    too_big = W.empty(1)
    W.harmonic(too_big[0], 1.0, 1.0, [1.0], [0.0], [1.0], 2**40)
    st = zmc.zmc_integrate_noalloc(too_big, out.data_ptr(), None)
    assert st == zmc.ZMC_ENOMEM and "fixed array" in zmc.zmc_last_error()
