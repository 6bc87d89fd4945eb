"""The chunk tuner (zmc_options.autotune & ZMC_TUNE_CHUNK): per plan it picks
the chunk length among 26, 52, 104 and 208 quints per lane and each family
kernel's quint-loop unroll (1 or 2), caches the choice by the table's shape
class, and reports it in zmc_plan_info.  Both change results within rounding
only: every candidate agrees with the FP64 oracle, results are bit-identical
for one cached choice, and a choice with unroll 1 everywhere gives bit for bit
what an untuned context with that chunk length gives."""
import json

import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

CANDIDATES = (26, 52, 104, 208)
TUNE_ALL = zmc.ZMC_TUNE_GEOMETRY | zmc.ZMC_TUNE_CHUNK


def _table():
    """Every family, dimensions 1..7, sizes around the candidate chunk lengths
    (160 Q samples) and the quint boundaries."""
    rng = np.random.default_rng(31)
    sizes = [1, 4, 5, 6, 4159, 4160, 4161, 8319, 8321, 16640, 16641, 33279, 33281, 70001]
    rows = []
    for fam in (W.HARMONIC, W.ABSLIN, W.GAUSS, W.POLY):
        for k, n in enumerate(sizes):
            d = 1 + (k + fam) % 7
            t = W.random_table(1, rng, n_lo=n, n_hi=n, families=[fam], dims=[d], seed=k + 3)
            rows.append(t[0])
    tab = W.empty(len(rows))
    for i, r in enumerate(rows):
        tab[i] = r
        tab[i]["stream_id"] = i
    return tab


def _plan_results(ctx, tab):
    plan = zmc.zmc_plan_create(ctx.handle, tab)
    try:
        info = zmc.zmc_plan_info_get(plan)
        zmc.zmc_plan_run(plan)
        return zmc.zmc_plan_results(plan, len(tab)), info
    finally:
        zmc.zmc_plan_destroy(plan)


@pytest.fixture(scope="module")
def oracle_results():
    tab = _table()
    want, _ = oracle.integrate(tab)
    return tab, want


@pytest.fixture(scope="module")
def untuned(zctx, oracle_results):
    """Results of untuned contexts, one per candidate chunk length."""
    tab, _ = oracle_results
    out = {}
    for q in CANDIDATES:
        with zmc.Context(arena_bytes=256 << 20, quints_per_lane=q) as c:
            out[q] = zmc.zmc_integrate(c.handle, tab)
    return out


def test_every_candidate_chunk_matches_the_oracle(oracle_results, untuned):
    tab, want = oracle_results
    for q in CANDIDATES:
        G.compare(tab, untuned[q], want)


def test_tuner_picks_caches_and_keeps_results(oracle_results, untuned, tmp_path):
    tab, want = oracle_results
    path = str(tmp_path / "tune.json")
    infos, results = [], []
    for _ in range(2):
        with zmc.Context(arena_bytes=512 << 20, autotune=TUNE_ALL, tune_cache_path=path) as c:
            got, info = _plan_results(c, tab)
        infos.append(info)
        q = info["quints_per_lane"]
        assert q in CANDIDATES
        assert all(u in (1, 2) for u in info["family_unroll"])
        if info["family_unroll"] == [1, 1, 1, 1]:
            # bit-identical to an untuned context with the chosen chunk length
            for key in ("estimate", "stderr", "n", "status"):
                assert np.array_equal(got[key], untuned[q][key], equal_nan=True), key
        G.compare(tab, got, want)
        results.append(got)
    # the cached choice reproduces the measured one bit for bit
    for key in ("estimate", "stderr", "n", "status"):
        assert np.array_equal(results[0][key], results[1][key], equal_nan=True), key
    assert infos[0]["chunk_tune_source"] == 1 and infos[1]["chunk_tune_source"] == 2
    assert infos[0]["quints_per_lane"] == infos[1]["quints_per_lane"]
    assert infos[0]["family_unroll"] == infos[1]["family_unroll"]
    entries = json.load(open(path))["entries"]
    chunk = [e for k, e in entries.items() if k.startswith("chunk|")]
    assert len(chunk) == 1 and chunk[0]["quints"] == infos[0]["quints_per_lane"]
    geometry = [e for k, e in entries.items() if not k.startswith("chunk|")]
    assert len(geometry) == 4 and all(e["block"] in (128, 256) for e in geometry)


def test_every_chunk_and_unroll_choice_from_the_cache(oracle_results, untuned, tmp_path):
    """Each candidate chunk length with each unroll pattern, forced through the
    cache the tuner reads: unroll 1 everywhere equals the untuned context at that
    chunk length bit for bit; every choice agrees with the oracle and repeats
    bit for bit."""
    tab, want = oracle_results
    path = tmp_path / "tune.json"
    with zmc.Context(arena_bytes=512 << 20, autotune=zmc.ZMC_TUNE_CHUNK,
                     tune_cache_path=str(path)) as c:
        _plan_results(c, tab)
    doc = json.loads(path.read_text())
    (key,) = [k for k in doc["entries"] if k.startswith("chunk|")]
    for q in CANDIDATES:
        for unroll in ([1, 1, 1, 1], [2, 2, 2, 2], [1, 2, 1, 2]):
            doc["entries"][key] = {"quints": q, "unroll": unroll, "ms": 1.0}
            path.write_text(json.dumps(doc))
            runs = []
            for _ in range(2):
                with zmc.Context(arena_bytes=512 << 20, autotune=zmc.ZMC_TUNE_CHUNK,
                                 tune_cache_path=str(path)) as c:
                    got, info = _plan_results(c, tab)
                assert info["chunk_tune_source"] == 2
                assert info["quints_per_lane"] == q and info["family_unroll"] == unroll
                runs.append(got)
            for k in ("estimate", "stderr", "n", "status"):
                assert np.array_equal(runs[0][k], runs[1][k], equal_nan=True), (q, unroll, k)
                if unroll == [1, 1, 1, 1]:
                    assert np.array_equal(runs[0][k], untuned[q][k], equal_nan=True), (q, k)
            G.compare(tab, runs[0], want)


def test_unknown_tune_flags_are_rejected():
    with pytest.raises(zmc.ZmcError) as e:
        zmc.Context(arena_bytes=64 << 20, autotune=4)
    assert e.value.status == zmc.ZMC_EINVAL
