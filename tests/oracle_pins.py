"""Checks that tie the FP64 oracle to facts outside itself.

Each check takes an ``oracle.Oracle`` instance (and, for the generator checks,
an independent Philox implementation) and raises ``AssertionError`` when the
oracle disagrees with:

* ``philox_vs_independent`` -- PyTorch's header-only Philox4x32-10 engine on
  random and boundary 128-bit counters and 64-bit keys (bit-exact);
* ``word_layout`` -- the same independent engine at the counter each sample
  coordinate is defined to use (field c = s*d + i, block c div 5, bits
  23 (c mod 5) .. +22 of the block's 128 bits, word 0 least significant; counter
  (stream_id, block lo, block hi, 0), key = seed), including blocks past 2^32;
* ``bruteforce_small`` -- an exact rational / 40-digit recomputation of the
  estimate and standard error from those independent words for N <= 16;
* ``closed_forms`` -- the analytic integral of every family (paper, Fig. 1
  caption: estimates against analytic results), within 5 true standard
  deviations of the mean, with the true deviation known in closed form too;
* ``fig1`` -- the paper's 100 harmonics of Eq. 1 against their closed form;
* ``eq2`` -- the abs-linear set of Eq. 2 against its exact value;
* ``stderr_calibration`` -- the spread of independent repeats (Fig. 1 caption:
  mean and standard deviation of 10 independent evaluations) against the
  reported standard error;
* ``special_cases`` -- N = 1 gives an undefined (NaN) standard error; a
  constant integrand gives an exact estimate and zero standard error.
"""
from __future__ import annotations

import math
from fractions import Fraction

import mpmath
import numpy as np

from paper_2104_10073_gb300 import workloads as W
from tests import closed_forms as CF

mpmath.mp.dps = 40


# ------------------------------------------------------------------ generator
def philox_vs_independent(orc, indep, n_random=400):
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2**32, size=(n_random, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n_random, 2), dtype=np.uint64).astype(np.uint32)
    edge = [0, 1, 2**31, 2**32 - 2, 2**32 - 1]
    extra_c, extra_k = [], []
    for e in edge:
        extra_c += [[e, 0, 0, 0], [0, e, 0, 0], [0, 0, e, 0], [0, 0, 0, e], [e, e, e, e]]
        extra_k += [[0, 0], [e, 0], [0, e], [e, e], [e, 2**32 - 1 - e]]
    ctr = np.concatenate([ctr, np.array(extra_c, dtype=np.uint32)])
    key = np.concatenate([key, np.array(extra_k, dtype=np.uint32)])
    got = orc.philox4x32_10(ctr, key)
    c64 = ctr.astype(np.uint64)
    k64 = key.astype(np.uint64)
    triples = [(int(k64[j, 0] | (k64[j, 1] << np.uint64(32))),
                int(c64[j, 2] | (c64[j, 3] << np.uint64(32))),
                int(c64[j, 0] | (c64[j, 1] << np.uint64(32)))) for j in range(len(ctr))]
    want = indep(triples)
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    assert bad.size == 0, f"Philox mismatch at {bad[:5]}: {got[bad[:1]]} vs {want[bad[:1]]}"


def engine_triple(seed, stream_id, block):
    """(seed, subsequence, offset) of the independent engine for the block the
    sample stream draws from.  The engine's counter is (offset lo, offset hi,
    subsequence lo, subsequence hi); the stream's is (stream_id, block lo,
    block hi, 0), i.e. offset stream_id + 2^32 block lo in subsequence block hi."""
    return (seed, block >> 32, stream_id | ((block & 0xFFFFFFFF) << 32))


def engine_fields(indep, seed, stream_id, fields):
    """The 23-bit fields ``fields`` (field indices of one stream) from the
    independent engine: each block's four words joined into one Python integer
    (word 0 least significant), field k of it = bits 23k .. 23k + 22."""
    fields = [int(c) for c in fields]
    words = indep([engine_triple(seed, stream_id, c // 5) for c in fields])
    out = []
    for c, w in zip(fields, words):
        block = sum(int(w[j]) << (32 * j) for j in range(4))
        out.append((block >> (23 * (c % 5))) & 0x7FFFFF)
    return np.array(out, dtype=np.uint32)


def _layout_rows():
    rows = []
    for d, sid, seed in [(1, 0, 0), (2, 7, 1), (3, 12345, 2**40 + 3), (4, 99, 5),
                         (5, 2**31 + 5, 2**64 - 1), (7, 1, 77)]:
        t = W.empty(1)
        W.abslin(t[0], 1.0, [1.0] * d, [0.0] * d, [1.0] * d, 10, seed=seed, stream_id=sid)
        rows.append(t[0])
    return rows


def word_layout(orc, indep):
    for row in _layout_rows():
        d = int(row["dim"])
        seed = int(row["seed"])
        sid = int(row["stream_id"])
        # a window at the start and one whose blocks straddle 2^32
        for s0 in (0, (5 * 2**32) // d - 3):
            count = 6
            got, _, _ = orc.samples(row, s0, count)
            want = engine_fields(indep, seed, sid,
                                 [(s0 + t) * d + i for t in range(count) for i in range(d)])
            assert np.array_equal(got, want.reshape(count, d)), (d, s0, got, want)


# ------------------------------------------------------------------ brute force
def _bf_rows():
    rng = np.random.default_rng(5)
    t = W.empty(8)
    W.harmonic(t[0], 1.3, -0.7, [2.5, -11.0, 0.3], [-0.5, 0.1, -1.0], [0.7, 1.9, 0.2], 16,
               seed=3, stream_id=4)
    W.harmonic(t[1], 1.0, 1.0, [(1 + 50) / (2 * math.pi)] * 4, [0.0] * 4, [1.0] * 4, 16)
    W.abslin(t[2], 1.7, [1.0, 1.0, -1.0], [-0.9, -0.3, -0.6], [0.4, 1.5, 1.1], 16, seed=2**33,
             stream_id=9)
    W.abslin(t[3], 0.8, [2.0], [-1.0], [0.5], 16, seed=1, stream_id=0)
    W.gauss(t[4], 1.0, 0.3, [0.1, -0.2], [-0.5, -1.0], [1.0, 0.6], 16, seed=4, stream_id=2)
    W.gauss(t[5], 2.0, 0.05, [0.0] * 7, [-0.1] * 7, [0.1] * 7, 16, seed=4, stream_id=3)
    W.poly(t[6], rng.standard_normal((3, 5)), [-1.0, -0.2, 0.0], [0.5, 1.3, 2.0], 16, seed=6,
           stream_id=1)
    W.poly(t[7], [[0.5, -2.0], [1.5, 0.25]], [-0.3, -0.9], [0.9, 0.4], 16, seed=7, stream_id=5)
    return t


def _exact_f(row, xs):
    fam, d = int(row["family"]), int(row["dim"])
    p = [mpmath.mpf(float(v)) for v in row["p"]]
    if fam == 0:
        ph = sum(p[2 + i] * xs[i] for i in range(d))
        return p[0] * mpmath.cos(ph) + p[1] * mpmath.sin(ph)
    if fam == 1:
        return p[0] * abs(sum(p[1 + i] * xs[i] for i in range(d)))
    if fam == 2:
        r2 = sum((xs[i] - p[2 + i]) ** 2 for i in range(d))
        return p[0] * mpmath.exp(-r2 / (2 * p[1] ** 2))
    out = mpmath.mpf(1)
    for i in range(d):
        out *= sum(p[5 * i + j] * xs[i] ** j for j in range(int(row["deg"]) + 1))
    return out


def bruteforce_small(orc, indep, sizes=(1, 2, 3, 5, 16)):
    for row in _bf_rows():
        d = int(row["dim"])
        lo = [mpmath.mpf(float(v)) for v in row["lo"][:d]]
        # the box width is formed in binary64, as the method's volume is
        wd = [mpmath.mpf(float(row["hi"][i]) - float(row["lo"][i])) for i in range(d)]
        vol = mpmath.mpf(1)
        for v in wd:
            vol *= v
        nmax = max(sizes)
        r = engine_fields(indep, int(row["seed"]), int(row["stream_id"]),
                          range(nmax * d)).reshape(nmax, d)
        fs = []
        for s in range(nmax):
            xs = [lo[i] + wd[i] * mpmath.mpf(int(r[s, i]) & 0x7FFFFF) / 2**23
                  for i in range(d)]
            fs.append(_exact_f(row, xs))
        for n in sizes:
            t = W.empty(1)
            t[0] = row
            t[0]["n_samples"] = n
            res, _ = orc.integrate(t, threads=1)
            mean = sum(fs[:n]) / n
            m2 = sum((f - mean) ** 2 for f in fs[:n])
            est = float(vol * mean)
            mabs = float(sum(abs(f) for f in fs[:n]) / n)
            scale = float(vol) * max(mabs, 1e-300)
            assert abs(res["estimate"][0] - est) <= 1e-11 * scale, (row, n, res, est)
            assert abs(res["mean_abs"][0] - mabs) <= 1e-11 * max(mabs, 1e-300)
            if n == 1:
                assert math.isnan(res["stderr"][0])
            else:
                se = float(vol * mpmath.sqrt(m2 / (n * (n - 1))))
                assert abs(res["stderr"][0] - se) <= 1e-9 * max(se, 1e-12 * scale), (row, n,
                                                                                      res, se)


# ------------------------------------------------------------------ closed forms
def designed_rows(n_samples=200_000):
    """Rows whose integral is large against the estimator's spread, so that a
    dropped term, a wrong sign or a swapped parameter moves the estimate by
    many standard errors."""
    rng = np.random.default_rng(2104)
    rows = []
    for d in (1, 2, 3, 4, 7):
        t = W.empty(1)
        k = rng.uniform(0.4, 2.5, size=d) * rng.choice([-1, 1], size=d)
        lo = rng.uniform(-1.0, 0.0, size=d)
        W.harmonic(t[0], 1.3, -0.6, k, lo, lo + rng.uniform(0.5, 1.2, size=d), n_samples,
                   seed=d, stream_id=10 + d)
        rows.append(t[0])
    for d in (1, 2, 3, 5):
        t = W.empty(1)
        c = rng.uniform(0.3, 2.0, size=d) * rng.choice([-1, 1], size=d)
        lo = rng.uniform(-1.0, 0.0, size=d)
        W.abslin(t[0], 1.4, c, lo, lo + rng.uniform(0.8, 2.0, size=d), n_samples, seed=d,
                 stream_id=20 + d)
        rows.append(t[0])
    for d in (1, 2, 3, 4):
        t = W.empty(1)
        lo = rng.uniform(-1.0, 0.0, size=d)
        hi = lo + rng.uniform(0.8, 1.5, size=d)
        W.gauss(t[0], 1.5, 0.45, rng.uniform(lo, hi), lo, hi, n_samples, seed=d,
                stream_id=30 + d)
        rows.append(t[0])
    for d, deg in ((1, 4), (2, 3), (3, 2), (4, 1)):
        t = W.empty(1)
        lo = rng.uniform(-1.0, 0.0, size=d)
        coef = rng.standard_normal((d, deg + 1))
        coef[:, 0] += 2.0  # keep the integral well away from zero
        W.poly(t[0], coef, lo, lo + rng.uniform(0.5, 1.5, size=d), n_samples, seed=d,
               stream_id=40 + d)
        rows.append(t[0])
    # one strongly oscillating harmonic (the paper's regime, Eq. 1 test)
    t = W.empty(1)
    W.harmonic(t[0], 0.9, 1.6, [25.0, -17.0], [0.0, -0.5], [1.0, 0.5], n_samples, seed=1,
               stream_id=50)
    rows.append(t[0])
    tab = W.empty(len(rows))
    for i, r in enumerate(rows):
        tab[i] = r
    return tab


def closed_forms(orc, n_samples=200_000, sensitive=True):
    tab = designed_rows(n_samples)
    res, _ = orc.integrate(tab)
    for i, row in enumerate(tab):
        exact = CF.exact(row)
        sig = CF.sigma_f(row) * CF.volume(row) / math.sqrt(n_samples)
        est, se = res["estimate"][i], res["stderr"][i]
        assert abs(est - exact) <= 5.0 * sig, (i, int(row["family"]), est, exact, sig)
        # the reported standard error matches the true spread of the mean
        assert abs(se / sig - 1.0) < 0.05, (i, se, sig)
        if sensitive and i < len(tab) - 1:
            assert sig < 0.02 * abs(exact), (i, sig, exact)


def fig1(orc, n_samples=100_000):
    tab = W.harmonic_fig1(n_samples)
    res, _ = orc.integrate(tab)
    z = []
    for n in range(1, 101):
        exact = CF.fig1_closed_form(n)
        assert abs(exact - CF.exact(tab[n - 1])) < 1e-12
        sig = CF.sigma_f(tab[n - 1]) / math.sqrt(n_samples)
        z.append((res["estimate"][n - 1] - exact) / sig)
        assert abs(res["stderr"][n - 1] / sig - 1.0) < 0.02
    z = np.array(z)
    assert np.all(np.abs(z) < 5.0), z
    # 100 standard normal scores: mean and spread within generous bounds
    assert abs(z.mean()) < 0.5 and 0.7 < z.std(ddof=1) < 1.3, (z.mean(), z.std())


def eq2(orc, n_samples=100_000):
    tab = W.abslin_eq2(n_samples)
    res, _ = orc.integrate(tab)
    for i, row in enumerate(tab):
        exact = CF.exact(row)
        sig = CF.sigma_f(row) * CF.volume(row) / math.sqrt(n_samples)
        assert abs(res["estimate"][i] - exact) <= 5 * sig, (i, res["estimate"][i], exact)
        assert sig < 0.02 * abs(exact)


def stderr_calibration(orc, repeats=300, n_samples=2000):
    """Spread of independent repeats (distinct keys) against the reported error."""
    tab = W.empty(repeats)
    for r in range(repeats):
        W.harmonic(tab[r], 1.2, 0.4, [3.0, -1.5], [0.0, -0.5], [1.0, 1.0], n_samples, seed=r,
                   stream_id=3)
    res, _ = orc.integrate(tab)
    spread = np.std(res["estimate"], ddof=1)
    se = np.mean(res["stderr"])
    # (repeats-1) s^2 / sigma^2 ~ chi^2_{repeats-1}: 0.1%..99.9% band of the ratio
    lo, hi = math.sqrt(0.76), math.sqrt(1.27)
    assert lo < spread / se < hi, (spread, se)
    sig = CF.sigma_f(tab[0]) * CF.volume(tab[0]) / math.sqrt(n_samples)
    assert abs(se / sig - 1) < 0.02
    z = (res["estimate"] - CF.exact(tab[0])) / sig
    assert abs(z.mean()) < 4.0 / math.sqrt(repeats)


def special_cases(orc):
    t = W.empty(3)
    W.harmonic(t[0], 1.0, 2.0, [1.0, 2.0], [0.0, 0.0], [1.0, 1.0], 1)
    W.poly(t[1], [[1.75], [-0.5], [3.0]], [-1.0, 0.0, 0.5], [0.5, 2.0, 1.25], 1000, seed=3)
    W.gauss(t[2], 1.0, 0.2, [0.0], [0.0], [1.0], 2)
    res, _ = orc.integrate(t)
    assert math.isnan(res["stderr"][0]) and np.isfinite(res["estimate"][0])
    vol = 1.5 * 2.0 * 0.75
    assert res["estimate"][1] == vol * (1.75 * -0.5 * 3.0)
    assert res["stderr"][1] == 0.0
    # N = 2: the standard error is V |f1 - f2| / 2
    _, _, fx = orc.samples(t[2], 0, 2)
    assert abs(res["stderr"][2] - abs(fx[0] - fx[1]) / 2) < 1e-15


ALL_CHECKS = ("philox_vs_independent", "word_layout", "bruteforce_small", "closed_forms",
              "fig1", "eq2", "stderr_calibration", "special_cases")
