"""CUDA path (through the C ABI) against the FP64 oracle on identical samples.

Tolerances are stated in tests/gpu_common.py.  Sizes span many chunks and
ragged tails (chunk = 160 * quints_per_lane = 16640 samples by default); the
full-size mixed table runs in the benchmark's launch configuration and is
checked on sampled rows the oracle computes one by one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import closed_forms as CF
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

# around lane quints (5 samples), warp rounds (160), accumulation blocks (65 per
# lane, 2080 per warp) and chunks (16640 by default, 4160 in serving contexts)
EDGE_SIZES = [1, 2, 3, 4, 5, 6, 7, 9, 10, 11, 159, 160, 161, 2079, 2080, 2081, 4159, 4160,
              4161, 8192, 10003, 16639, 16640, 16641, 33281, 65537]


# ------------------------------------------------------------------ generator
def test_philox_bitexact_vs_oracle(zctx):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(5000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(5000, 2), dtype=np.uint64).astype(np.uint32)
    edge = np.array([[0, 0, 0, 0], [2**32 - 1] * 4, [2**32 - 1, 0, 0, 0], [0, 2**32 - 1, 5, 0]],
                    dtype=np.uint32)
    ctr = np.concatenate([ctr, edge])
    key = np.concatenate([key, np.array([[0, 0], [2**32 - 1] * 2, [1, 0], [0, 1]],
                                        dtype=np.uint32)])
    got = zmc.zmc_philox4x32_10(zctx.handle, ctr, key)
    want = oracle.philox4x32_10(ctr, key)
    assert np.array_equal(got, want)


def test_philox_three_way_with_curand(zctx, curand_philox):
    """Library, oracle and cuRAND's device Philox4x32-10 agree bit for bit."""
    rng = np.random.default_rng(2)
    ctr = rng.integers(0, 2**32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(2000, 2), dtype=np.uint64).astype(np.uint32)
    cur = curand_philox(ctr, key)
    assert np.array_equal(cur, oracle.philox4x32_10(ctr, key))
    assert np.array_equal(cur, zmc.zmc_philox4x32_10(zctx.handle, ctr, key))


# ------------------------------------------------------------------ per sample
def _per_sample_rows():
    rng = np.random.default_rng(7)
    rows = []
    for fam in range(4):
        for d in range(1, 8):
            t = W.random_table(1, rng, n_lo=10**6, n_hi=10**6, families=[fam], dims=[d],
                               seed=int(rng.integers(0, 2**63)))
            t[0]["stream_id"] = int(rng.integers(0, 2**32))
            rows.append(t[0])
    # large phases: |k.x| up to ~420 rad
    t = W.empty(1)
    W.harmonic(t[0], 1.1, -0.8, [30.0] * 7, [-1.0] * 7, [1.0] * 7, 10**6, seed=3)
    rows.append(t[0])
    return rows


def test_eval_samples_match_oracle_per_sample(zctx):
    for row in _per_sample_rows():
        for s0 in (0, 1, 999_000):
            count = 997
            got = zmc.zmc_eval_samples(zctx.handle, row, s0, count).astype(np.float64)
            _, _, want = oracle.samples(row, s0, count)
            tol = 4e-6 * G.sample_scale(row)
            err = np.max(np.abs(got - want))
            assert err <= tol, (int(row["family"]), int(row["dim"]), s0, err, tol)


def test_poly_relative_accuracy_near_roots(zctx):
    """Product polynomials whose factors have roots inside the box: every
    sample's value keeps its relative accuracy, even where a factor nearly
    vanishes (the root form; Horner on the coefficients loses up to the ratio of
    the summed terms to the value there).  Factors are built from given roots so
    that several lie inside [lo, hi]."""
    rng = np.random.default_rng(77)
    for d, deg in ((1, 2), (2, 4), (3, 3), (5, 4), (7, 2), (7, 4)):
        t = W.empty(1)
        lo = rng.uniform(-1.0, 0.0, d)
        hi = lo + rng.uniform(0.5, 2.0, d)
        coef = np.zeros((d, deg + 1))
        for i in range(d):
            roots = list(rng.uniform(lo[i], hi[i], deg))
            if deg >= 2 and rng.random() < 0.5:  # a complex pair near the box
                a, b = rng.uniform(lo[i], hi[i]), rng.uniform(0.01, 0.3)
                roots[:2] = [a + 1j * b, a - 1j * b]
            c = np.array([rng.uniform(0.5, 2.0)], dtype=complex)
            for r in roots:
                c = np.convolve(c, [-r, 1.0])
            coef[i] = np.real(c)
        W.poly(t[0], coef, lo, hi, 10**6, seed=d, stream_id=deg)
        got = zmc.zmc_eval_samples(zctx.handle, t[0], 1000, 4000).astype(np.float64)
        _, _, want = oracle.samples(t[0], 1000, 4000)
        rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-30)
        # FP32: a few ulp per factor and per product; values within 1e-5 of a
        # root in relative terms are left to the absolute check
        ok = rel <= 2e-6
        assert np.mean(ok) >= 0.999, (d, deg, np.sort(rel)[-5:])
        assert np.max(np.abs(got - want)) <= 2e-6 * G.sample_scale(t[0]), (d, deg)


def test_eval_samples_across_block_index_carry(zctx):
    """Samples whose Philox block index crosses 2^32 (counter word 2, block hi, carries)."""
    for d in (1, 3, 7):
        t = W.empty(1)
        W.abslin(t[0], 1.0, [1.0] * d, [0.0] * d, [1.0] * d, 2**36, seed=9, stream_id=4)
        s0 = (5 * 2**32) // d - 40
        got = zmc.zmc_eval_samples(zctx.handle, t[0], s0, 80).astype(np.float64)
        _, _, want = oracle.samples(t[0], s0, 80)
        assert np.max(np.abs(got - want)) <= 4e-6 * G.sample_scale(t[0])


# ------------------------------------------------------------------ estimates
@pytest.mark.parametrize("fam", [W.HARMONIC, W.ABSLIN, W.GAUSS, W.POLY])
def test_integrate_edge_sizes_every_dim(zctx, fam):
    rng = np.random.default_rng(100 + fam)
    rows = []
    for d in range(1, 8):
        for n in EDGE_SIZES:
            t = W.random_table(1, rng, n_lo=n, n_hi=n, families=[fam], dims=[d], seed=d * 7 + n)
            t[0]["stream_id"] = len(rows)
            rows.append(t[0])
    tab = W.empty(len(rows))
    for i, r in enumerate(rows):
        tab[i] = r
    got = zmc.zmc_integrate(zctx.handle, tab)
    want, _ = oracle.integrate(tab)
    G.compare(tab, got, want)


@pytest.mark.parametrize("fam", [W.HARMONIC, W.ABSLIN, W.GAUSS, W.POLY])
def test_single_sample_rows_keep_relative_accuracy(zctx, fam):
    """1500 rows of one sample each: the tolerance is then per sample and
    relative, so every family must keep its relative accuracy wherever samples
    fall, next to zeros of cos, of c.x and of the polynomial factors included
    (an FP32 sum of c.x, for one, failed 91 of these 1500 abs-linear rows)."""
    rng = np.random.default_rng(300 + fam)
    t = W.random_table(1500, rng, n_lo=1, n_hi=1, families=[fam], seed=fam + 11)
    t["stream_id"] = np.arange(len(t))
    got = zmc.zmc_integrate(zctx.handle, t)
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)


def _equal_rate_harmonics(n_rows, rng, n_lo, n_hi):
    """Harmonic rows whose dimensions all advance the phase at the same rate
    (k_i (hi_i - lo_i) equal: a scalar wave number on a cube of any offset), the
    form the library evaluates through the phase of the coordinate sum: wave
    numbers of either sign up to the validation limit's neighbourhood,
    dimensions 2..7."""
    t = W.empty(n_rows)
    for i in range(n_rows):
        d = int(rng.integers(2, 8))
        width = float(rng.uniform(0.25, 2.0))
        lo = float(rng.uniform(-3.0, 1.0))
        kappa = float(rng.choice([-1.0, 1.0]) * 10 ** rng.uniform(-1.0, 3.0))
        n = int(rng.integers(n_lo, n_hi + 1))
        W.harmonic(t[i], float(rng.uniform(-2, 2)), float(rng.uniform(-2, 2)), [kappa] * d,
                   [lo] * d, [lo + width] * d, n, seed=int(rng.integers(0, 2**40)), stream_id=i)
    return t


def test_equal_rate_harmonics_per_sample(zctx):
    """Per-sample values of the equal-rate form against the oracle's FP64 cos."""
    t = _equal_rate_harmonics(40, np.random.default_rng(911), 10**6, 10**6)
    assert np.all(zmc.zmc_variant_of(t)["form"] == 1)  # the equal-rate form
    for row in t:
        for s0 in (0, 3, 500_000):
            got = zmc.zmc_eval_samples(zctx.handle, row, s0, 501).astype(np.float64)
            _, _, want = oracle.samples(row, s0, 501)
            err = np.max(np.abs(got - want))
            assert err <= 4e-6 * G.sample_scale(row), (int(row["dim"]), s0, err)


def test_equal_rate_harmonics_single_samples_and_edges(zctx):
    """Single-sample rows (relative accuracy next to zeros of cos) and sizes
    around the quint and chunk boundaries, against the oracle."""
    rng = np.random.default_rng(912)
    ones = _equal_rate_harmonics(1500, rng, 1, 1)
    assert np.all(zmc.zmc_variant_of(ones)["form"] == 1)
    got = zmc.zmc_integrate(zctx.handle, ones)
    want, _ = oracle.integrate(ones)
    G.compare(ones, got, want)
    edges = _equal_rate_harmonics(len(EDGE_SIZES), rng, 1, 1)
    edges["n_samples"] = EDGE_SIZES
    got = zmc.zmc_integrate(zctx.handle, edges)
    want, _ = oracle.integrate(edges)
    G.compare(edges, got, want)


def _abslin_scale_rows():
    """Abs-linear rows whose fixed-point scale 2^-F lands far from the usual:
    tiny, huge and mixed coefficient magnitudes, zero coefficients, boxes far
    from the origin and hyperplanes through the box."""
    rows = []
    rng = np.random.default_rng(77)
    cases = [([1e-20, -2e-20], [-1.0, 0.0], [1.0, 2.0]),
             ([3e15, -1e15, 2e15], [-1.0, -1.0, 0.0], [0.5, 1.0, 2.0]),
             ([1e8, 1e-8], [0.0, 0.0], [1.0, 1.0]),
             ([0.0, 1.0, 0.0], [-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]),
             ([0.0, 0.0], [0.0, 0.0], [1.0, 1.0]),
             ([1.0, -1.0], [1e3, 1e3], [1e3 + 1.0, 1e3 + 1.0]),
             ([1.0] * 7, [-0.5] * 7, [0.5] * 7),
             ([1.0, 1.0, -1.0], [-3e-9, -1e-9, -2e-9], [1e-9, 2e-9, 3e-9])]
    for c, lo, hi in cases:
        for n in (1, 7, 1000):
            t = W.empty(1)
            W.abslin(t[0], float(rng.uniform(0.5, 2.0)), c, lo, hi, n, seed=n,
                     stream_id=len(rows))
            rows.append(t[0])
    tab = W.empty(len(rows))
    for i, r in enumerate(rows):
        tab[i] = r
    return tab


def test_abslin_32bit_sum_rows(zctx):
    """Rows of >= 256 samples take the 32-bit sum of c.x: sizes around that
    threshold, every dimension, against the oracle.  Boxes: centred on the
    hyperplane (mean|f| smallest against max|f|), far from the origin with
    alternating coefficient signs (terms of 1e3 cancelling to c.x of order 1),
    tiny and huge coefficients, random coefficient signs."""
    rng = np.random.default_rng(4321)
    rows = []
    for d in range(1, 8):
        alt = [1.0 if i % 2 == 0 else -1.0 for i in range(d)]
        for n in (255, 256, 257, 1000, 4161):
            rnd = list(rng.choice([-1.0, 1.0], size=d))
            for c, lo, hi in ((rnd, [-0.5] * d, [0.5] * d),
                              (alt, [1e3] * d, [1e3 + 1.0] * d),
                              ([1e-12 * x for x in rnd], [-2.0] * d, [1.5] * d),
                              ([1e9 * x for x in alt], [-1.0] * d, [1.0] * d)):
                t = W.empty(1)
                W.abslin(t[0], float(rng.uniform(0.5, 2.0)), c, lo, hi, n, seed=n + d,
                         stream_id=len(rows))
                rows.append(t[0])
    tab = W.empty(len(rows))
    for i, r in enumerate(rows):
        tab[i] = r
    # both sums are reached: the 32-bit one from 256 samples on
    forms = zmc.zmc_variant_of(tab)["form"]
    assert np.array_equal(forms, (tab["n_samples"] >= 256).astype(forms.dtype))
    got = zmc.zmc_integrate(zctx.handle, tab)
    want, _ = oracle.integrate(tab)
    G.compare(tab, got, want)


def test_abslin_fixed_point_scale_edge_cases(zctx):
    t = _abslin_scale_rows()
    got = zmc.zmc_integrate(zctx.handle, t)
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)


def test_integrate_every_poly_degree(zctx):
    rng = np.random.default_rng(5)
    tab = W.empty(7 * 5 * 3)
    k = 0
    for d in range(1, 8):
        for deg in range(5):
            for n in (3, 2049, 30001):
                lo = rng.uniform(-1, 0, size=d)
                W.poly(tab[k], rng.standard_normal((d, deg + 1)), lo,
                       lo + rng.uniform(0.5, 2, size=d), n, seed=deg, stream_id=k)
                k += 1
    got = zmc.zmc_integrate(zctx.handle, tab)
    want, _ = oracle.integrate(tab)
    G.compare(tab, got, want)


def test_fig1_batched_matches_oracle_and_closed_form(zctx):
    import json
    import os

    tab = W.harmonic_fig1(10**5)
    got = zmc.zmc_integrate(zctx.handle, tab)
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "fig1_oracle_n1e5.json")))
    want = np.zeros(100, dtype=[("estimate", "f8"), ("stderr", "f8"), ("mean_abs", "f8")])
    for key in want.dtype.names:
        want[key] = [float.fromhex(v) for v in g[key]]
    G.compare(tab, got, want)
    for n in range(1, 101):
        exact = CF.fig1_closed_form(n)
        assert abs(got["estimate"][n - 1] - exact) <= 5 * got["stderr"][n - 1]


def test_fig1_plain_fp64_matches_oracle(zctx):
    tab = W.harmonic_fig1(10**5)
    got = zmc.zmc_integrate_plain(zctx.handle, tab)
    want, _ = oracle.integrate(tab)
    # FP64 on both sides: only the summation order differs
    G.compare(tab, got, want, est_rel=1e-11, se_rel=1e-9)


def test_plain_fp64_all_families(zctx):
    tab = W.random_table(60, np.random.default_rng(12), n_lo=1, n_hi=20000)
    got = zmc.zmc_integrate_plain(zctx.handle, tab)
    want, _ = oracle.integrate(tab)
    G.compare(tab, got, want, est_rel=1e-10, se_rel=1e-8)


def test_eq2_abslin_batched(zctx):
    tab = W.abslin_eq2(10**6)
    got = zmc.zmc_integrate(zctx.handle, tab)
    want, _ = oracle.integrate(tab)
    G.compare(tab, got, want)
    for i, row in enumerate(tab):
        assert abs(got["estimate"][i] - CF.exact(row)) <= 5 * got["stderr"][i]


def test_fig1_ten_repeats_one_launch(zctx):
    """The paper's 10 independent evaluations (keys 0..9) in one persistent launch:
    per-n mean over repeats against the closed form, and sampled rows against
    the oracle."""
    tab = W.harmonic_fig1(10**6, seeds=range(10))
    got = zmc.zmc_integrate(zctx.handle, tab)
    est = got["estimate"].reshape(10, 100)
    mean = est.mean(axis=0)
    std = est.std(axis=0, ddof=1)
    exact = np.array([CF.fig1_closed_form(n) for n in range(1, 101)])
    assert np.all(np.abs(mean - exact) <= 5 * std / math.sqrt(10) + 1e-12)
    # the repeat spread against the per-run standard error (chi^2_9 band)
    ratio = std / got["stderr"].reshape(10, 100).mean(axis=0)
    assert np.mean((ratio > math.sqrt(1.15 / 9)) & (ratio < math.sqrt(27.9 / 9))) >= 0.98
    pick = np.arange(0, 1000, 37)
    want, _ = oracle.integrate(tab[pick])
    G.compare(tab[pick], got[pick], want)


# ------------------------------------------------------------------ invariants
def test_results_independent_of_batch_composition(zctx):
    tab = W.random_table(40, np.random.default_rng(21), n_lo=1, n_hi=50000)
    full = zmc.zmc_integrate(zctx.handle, tab)
    for sl in (slice(0, 1), slice(5, 17), slice(39, 40), slice(0, 40, 3)):
        part = zmc.zmc_integrate(zctx.handle, tab[sl])
        assert np.array_equal(part["estimate"], full["estimate"][sl])
        assert np.array_equal(part["stderr"], full["stderr"][sl], equal_nan=True)


def test_row_partition_through_the_library(zctx):
    """Whole integrands split over ranks (run here one after another) and gathered
    back reproduce the single call bit for bit."""
    from paper_2104_10073_gb300 import shard

    tab = W.mixed(120, gen_seed=12, lo_exp=3.0, hi_exp=5.5)
    full = zmc.zmc_integrate(zctx.handle, tab)
    est = np.full(len(tab), np.nan)
    for rows in shard.partition_rows(tab, 3):
        part = zmc.zmc_integrate(zctx.handle, tab[rows])
        est[rows] = part["estimate"]
    assert np.array_equal(est, full["estimate"])


def test_plan_replay_is_bit_identical(zctx):
    tab = W.mixed(200, gen_seed=3, lo_exp=3, hi_exp=5)
    plan = zmc.zmc_plan_create(zctx.handle, tab)
    try:
        zmc.zmc_plan_run(plan)
        a = zmc.zmc_plan_results(plan, len(tab))
        for stages in (zmc.ZMC_STAGE_ALL, zmc.ZMC_STAGE_SAMPLE):
            zmc.zmc_plan_run(plan, stages)
            if stages == zmc.ZMC_STAGE_SAMPLE:
                zmc.zmc_plan_run(plan, zmc.ZMC_STAGE_MERGE)
            b = zmc.zmc_plan_results(plan, len(tab))
            assert np.array_equal(a["estimate"], b["estimate"])
            assert np.array_equal(a["stderr"], b["stderr"], equal_nan=True)
        one = zmc.zmc_integrate(zctx.handle, tab)
        assert np.array_equal(a["estimate"], one["estimate"])
    finally:
        zmc.zmc_plan_destroy(plan)


def test_autotune_keeps_results_and_caches(zctx, tmp_path):
    """The autotuner only picks launch geometry: results stay bit-identical, the
    choice is written to the JSON cache and reused by a later context."""
    import json

    tab = W.mixed(300, gen_seed=5, lo_exp=4.0, hi_exp=6.0)
    ref = zmc.zmc_integrate(zctx.handle, tab)
    path = str(tmp_path / "tune.json")
    infos = []
    for _ in range(2):
        with zmc.Context(arena_bytes=512 << 20, autotune=True, tune_cache_path=path) as c:
            plan = zmc.zmc_plan_create(c.handle, tab)
            try:
                infos.append(zmc.zmc_plan_info_get(plan))
                zmc.zmc_plan_run(plan)
                got = zmc.zmc_plan_results(plan, len(tab))
            finally:
                zmc.zmc_plan_destroy(plan)
        assert np.array_equal(got["estimate"], ref["estimate"])
        assert np.array_equal(got["stderr"], ref["stderr"], equal_nan=True)
    present = [b > 0 for b in infos[0]["family_block"]]
    assert [s for s, p in zip(infos[0]["tune_source"], present) if p] == [1] * sum(present)
    assert [s for s, p in zip(infos[1]["tune_source"], present) if p] == [2] * sum(present)
    assert infos[0]["family_grid"] == infos[1]["family_grid"]
    entries = json.load(open(path))["entries"]
    assert len(entries) == sum(present)
    assert all(e["block"] in (128, 256) and e["blocks_per_sm"] >= 1 for e in entries.values())


def test_chunk_length_changes_only_rounding():
    tab = W.random_table(30, np.random.default_rng(4), n_lo=100, n_hi=40000)
    want, _ = oracle.integrate(tab)
    for q in (1, 4, 64, 256):
        with zmc.Context(arena_bytes=256 << 20, quints_per_lane=q) as c:
            got = zmc.zmc_integrate(c.handle, tab)
        G.compare(tab, got, want)


def test_peaked_integrands_long_chunks():
    """Narrow Gaussians whose few large samples dominate the mean: the FP32 lane
    sums must not let a large first sample inflate the rounding error."""
    rng = np.random.default_rng(44)
    tab = W.empty(48)
    for i in range(48):
        d = 1 + i % 7
        lo = rng.uniform(-1, 0, size=d)
        hi = lo + rng.uniform(0.5, 2, size=d)
        W.gauss(tab[i], 1.0, rng.uniform(0.05, 0.2), rng.uniform(lo, hi), lo, hi,
                int(rng.integers(3000, 60000)), seed=i, stream_id=i)
    want, _ = oracle.integrate(tab)
    for q in (16, 64, 256):
        with zmc.Context(arena_bytes=256 << 20, quints_per_lane=q) as c:
            got = zmc.zmc_integrate(c.handle, tab)
        G.compare(tab, got, want)


def test_special_cases(zctx):
    t = W.empty(3)
    W.harmonic(t[0], 1.0, 2.0, [1.0, 2.0], [0.0, 0.0], [1.0, 1.0], 1)
    W.poly(t[1], [[1.75], [-0.5], [3.0]], [-1.0, 0.0, 0.5], [0.5, 2.0, 1.25], 100000, seed=3)
    W.gauss(t[2], 1.0, 0.2, [0.0], [0.0], [1.0], 2)
    got = zmc.zmc_integrate(zctx.handle, t)
    assert math.isnan(got["stderr"][0])
    assert got["stderr"][1] == 0.0
    assert abs(got["estimate"][1] - 1.5 * 2.0 * 0.75 * (1.75 * -0.5 * 3.0)) < 1e-6
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)


def test_empty_inputs(zctx):
    """An empty table is rejected by every call that integrates or plans it;
    zero-length test calls compute nothing; the context stays usable."""
    empty = W.empty(0)
    for call in (zmc.zmc_integrate, zmc.zmc_integrate_plain, zmc.zmc_plan_create):
        with pytest.raises(zmc.ZmcError) as e:
            call(zctx.handle, empty)
        assert e.value.status == zmc.ZMC_EINVAL
    words = zmc.zmc_philox4x32_10(zctx.handle, np.zeros((0, 4), np.uint32),
                                  np.zeros((0, 2), np.uint32))
    assert words.shape == (0, 4)
    t = W.harmonic_fig1(1000)[:1].copy()
    assert zmc.zmc_eval_samples(zctx.handle, t[0], 0, 0).shape == (0,)
    got = zmc.zmc_integrate(zctx.handle, t)
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)


def test_invalid_descriptor_is_rejected(zctx):
    t = W.harmonic_fig1(10)[:2].copy()
    t[1]["dim"] = 0
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_integrate(zctx.handle, t)
    assert e.value.status == zmc.ZMC_EINVAL
    # the context is still usable
    ok = zmc.zmc_integrate(zctx.handle, t[:1])
    assert ok["status"][0] == 0


# ------------------------------------------------------------------ full size
def _bench_config_results(tab, tmp_path):
    """Results of ``tab`` computed exactly as bench.py times it: autotuned
    context, device-resident plan, sampling and merge stages launched
    separately, then one more run as the captured graph (must agree)."""
    with zmc.Context(arena_bytes=2 << 30, autotune=True,
                     tune_cache_path=str(tmp_path / "tune.json")) as c:
        plan = zmc.zmc_plan_create(c.handle, tab)
        try:
            zmc.zmc_plan_run(plan, zmc.ZMC_STAGE_SAMPLE)
            zmc.zmc_plan_run(plan, zmc.ZMC_STAGE_MERGE)
            staged = zmc.zmc_plan_results(plan, len(tab))
            zmc.zmc_plan_run(plan)
            graph = zmc.zmc_plan_results(plan, len(tab))
        finally:
            zmc.zmc_plan_destroy(plan)
    assert np.array_equal(staged["estimate"], graph["estimate"])
    return graph


def test_fig1x10_full_size_bench_configuration(tmp_path):
    """The bench workload at full size (10^9 samples) in the bench's launch
    configuration; rows sampled across all keys recomputed by the oracle."""
    tab = W.harmonic_fig1(10**6, seeds=range(10))
    got = _bench_config_results(tab, tmp_path)
    assert np.array_equal(got["n"], tab["n_samples"]) and np.all(got["status"] == 0)
    pick = np.arange(3, 1000, 41)
    want, _ = oracle.integrate(tab[pick])
    G.compare(tab[pick], got[pick], want)


def test_mixed_1e4_full_size_sampled_rows(tmp_path):
    """The 10^4-integrand mix at full size in the bench's launch configuration;
    sampled rows of every family recomputed by the oracle one by one."""
    tab = W.mixed(10**4)
    got = _bench_config_results(tab, tmp_path)
    assert np.array_equal(got["n"], tab["n_samples"])
    assert np.all(np.isfinite(got["estimate"]))
    assert np.all(got["stderr"][tab["n_samples"] > 1] >= 0)
    rng = np.random.default_rng(0)
    pick = []
    for fam in range(4):
        rows = np.nonzero(tab["family"] == fam)[0]
        pick += list(rng.choice(rows, size=4, replace=False))
    pick = np.array(sorted(pick))
    want, _ = oracle.integrate(tab[pick])
    G.compare(tab[pick], got[pick], want)


def test_generator_rate_is_measured(zctx):
    """The generator-only kernel runs and reports a finite positive rate; its
    arguments are checked."""
    rate = zmc.zmc_philox_rate(zctx.handle, 1 << 28)
    assert math.isfinite(rate) and rate > 1e9
    for bad in (0, (1 << 40) + 1):
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_philox_rate(zctx.handle, bad)
        assert e.value.status == zmc.ZMC_EINVAL
