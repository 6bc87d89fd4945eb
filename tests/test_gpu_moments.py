"""zmc_integrate_moments: moments over sample ranges of each stream (GPU).

Pieces of one stream merge (Chan) to the unsplit result: to FP64 rounding when
the pieces start on chunk boundaries, within the stated tolerance otherwise.
This is what splitting one integrand over GPUs, checkpointing between pieces
and extending a run to more samples rest on.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import shard
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu
CHUNK = 160 * zmc.DEFAULT_QUINTS_PER_LANE  # samples per chunk at the default


def _volumes(t):
    return [G.volume(r) for r in t]


def _merge(t, pieces):
    return shard.merge_moments(len(t), pieces, _volumes(t))


def test_chunk_aligned_pieces_merge_to_integrate(zctx):
    t = W.random_table(40, np.random.default_rng(31), n_lo=3 * CHUNK, n_hi=60000)
    full = zmc.zmc_integrate(zctx.handle, t)
    rows, b, e = [], [], []
    for i, r in enumerate(t):
        n = int(r["n_samples"])
        c1 = (n // 3) // CHUNK * CHUNK
        c2 = (2 * n // 3) // CHUNK * CHUNK
        for lo, hi in ((0, c1), (c1, c2), (c2, n)):
            if hi > lo:
                rows.append(i), b.append(lo), e.append(hi)
    m = zmc.zmc_integrate_moments(zctx.handle, t[rows], b, e)
    assert np.all(m["status"] == 0) and np.array_equal(m["n"], np.array(e) - np.array(b))
    got = _merge(t, [(r, k["n"], k["mean"], k["m2"]) for r, k in zip(rows, m)])
    want, _ = oracle.integrate(t)
    for i in range(len(t)):
        scale = G.volume(t[i]) * want["mean_abs"][i]
        assert abs(got["estimate"][i] - full["estimate"][i]) <= 1e-12 * scale + 1e-300
        assert abs(got["stderr"][i] - full["stderr"][i]) <= 1e-9 * full["stderr"][i]
    G.compare(t, np.array([(g["estimate"], g["stderr"], g["n"], 0, 0) for g in got],
                          dtype=zmc.RESULT_DTYPE), want)


def test_unaligned_pieces_match_oracle_moments(zctx):
    t = W.random_table(24, np.random.default_rng(32), n_lo=100, n_hi=30000)
    rng = np.random.default_rng(33)
    rows, b, e = [], [], []
    for i, r in enumerate(t):
        n = int(r["n_samples"])
        a = int(rng.integers(0, n // 5)) * 5
        z = int(rng.integers(a + 1, n + 1))
        rows.append(i), b.append(a), e.append(z)
    m = zmc.zmc_integrate_moments(zctx.handle, t[rows], b, e)
    for k, (i, a, z) in enumerate(zip(rows, b, e)):
        n, mean, m2, sum_abs = oracle.moments(t[i], a, z)
        assert m["n"][k] == n
        scale = sum_abs / n
        assert abs(m["mean"][k] - mean) <= 1e-6 * scale + 2.0**-100 * G.sample_scale(t[i])
        if n > 1:
            assert abs(m["m2"][k] - m2) <= 1e-4 * m2 + 2e-6 * scale * scale * math.sqrt(n)


def test_ranges_across_the_block_index_carry(zctx):
    """Sample ranges on both sides of Philox block 2^32 (counter word 2, block
    hi, becomes 1): chunks wholly past it run the per-chunk prefix with block
    hi = 1, the chunk that straddles it the general counter; against the
    oracle's moments of the same ranges, for every family."""
    rng = np.random.default_rng(36)
    rows, b, e = [], [], []
    for fam in (W.HARMONIC, W.ABSLIN, W.GAUSS, W.POLY):
        for d in (1, 3, 4, 7):
            t = W.random_table(1, rng, n_lo=2**36, n_hi=2**36, families=[fam], dims=[d],
                               seed=fam * 10 + d)
            s_carry = -(-(2**32) // d) * 5  # first sample whose blocks start past 2^32
            a = (s_carry - 3 * CHUNK - 5 * d) // 5 * 5
            rows.append(t[0]), b.append(a), e.append(a + 7 * CHUNK + 13)
    tab = W.empty(len(rows))
    for i, r in enumerate(rows):
        tab[i] = r
        tab[i]["stream_id"] = i
    m = zmc.zmc_integrate_moments(zctx.handle, tab, b, e)
    for k in range(len(tab)):
        n, mean, m2, sum_abs = oracle.moments(tab[k], b[k], e[k])
        assert m["n"][k] == n
        scale = sum_abs / n
        assert abs(m["mean"][k] - mean) <= 1e-6 * scale + 2.0**-100 * G.sample_scale(tab[k])
        assert abs(m["m2"][k] - m2) <= 1e-4 * m2 + 2e-6 * scale * scale * math.sqrt(n)


def test_progressive_refinement_extends_the_stream(zctx):
    """[0, N) and [N, 2N) merged equal a run with 2N samples."""
    base = W.random_table(12, np.random.default_rng(34), n_lo=CHUNK, n_hi=20 * CHUNK)
    base["n_samples"] = base["n_samples"] // CHUNK * CHUNK
    n = base["n_samples"].astype(np.int64)
    first = zmc.zmc_integrate_moments(zctx.handle, base, np.zeros(len(base)), n)
    second = zmc.zmc_integrate_moments(zctx.handle, base, n, 2 * n)
    pieces = [(i, k["n"], k["mean"], k["m2"]) for i, k in enumerate(first)]
    pieces += [(i, k["n"], k["mean"], k["m2"]) for i, k in enumerate(second)]
    got = _merge(base, pieces)
    doubled = base.copy()
    doubled["n_samples"] = 2 * base["n_samples"]
    full = zmc.zmc_integrate(zctx.handle, doubled)
    want, _ = oracle.integrate(doubled)
    for i in range(len(base)):
        scale = G.volume(base[i]) * want["mean_abs"][i]
        assert abs(got["estimate"][i] - full["estimate"][i]) <= 1e-12 * scale


def test_sample_partition_over_ranks_on_device(zctx):
    """shard.partition_samples on the device: three ranks' pieces (run here one
    after another) merge to the single-call results."""
    t = W.mixed(40, gen_seed=35, lo_exp=3.5, hi_exp=5.5)
    t["n_samples"] = (t["n_samples"] + CHUNK - 1) // CHUNK * CHUNK
    full = zmc.zmc_integrate(zctx.handle, t)
    pieces = []
    for rank_pieces in shard.partition_samples(t, 3, align=CHUNK):
        pieces += shard.rank_moments(zctx.handle, t, rank_pieces)
    got = _merge(t, pieces)
    want, _ = oracle.integrate(t)
    for i in range(len(t)):
        scale = G.volume(t[i]) * want["mean_abs"][i]
        assert abs(got["estimate"][i] - full["estimate"][i]) <= 1e-12 * scale + 1e-300


def test_bad_ranges_are_rejected(zctx):
    t = W.harmonic_fig1(1000)[:2]
    for b, e in (([2, 0], [10, 10]), ([8, 0], [10, 10]), ([0, 10], [10, 10]),
                 ([0, 15], [10, 5])):
        with pytest.raises(zmc.ZmcError) as err:
            zmc.zmc_integrate_moments(zctx.handle, t, b, e)
        assert err.value.status == zmc.ZMC_EINVAL
