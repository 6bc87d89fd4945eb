"""The FP64 oracle against facts outside itself (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate as spi

import oracle
from paper_2104_10073_gb300 import workloads as W
from tests import closed_forms as CF
from tests import oracle_pins as P


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def test_philox_matches_independent_engine(orc, torch_philox):
    P.philox_vs_independent(orc, torch_philox)


def test_word_layout_matches_independent_engine(orc, torch_philox):
    P.word_layout(orc, torch_philox)


def test_bruteforce_exact_small_n(orc, torch_philox):
    P.bruteforce_small(orc, torch_philox)


def test_closed_forms_all_families(orc):
    P.closed_forms(orc)


def test_fig1_harmonics_closed_form(orc):
    P.fig1(orc)


def test_eq2_abslin_exact(orc):
    P.eq2(orc)


def test_stderr_matches_repeat_spread(orc):
    P.stderr_calibration(orc)


def test_special_cases(orc):
    P.special_cases(orc)


def test_moments_split_merge(orc):
    """Moments over sample ranges combine (Chan's pairwise form) to the whole."""
    t = W.random_table(6, np.random.default_rng(3), n_lo=50, n_hi=3000)
    for row in t:
        n = int(row["n_samples"])
        whole = orc.moments(row, 0, n)
        cut = n // 3
        a, b = orc.moments(row, 0, cut), orc.moments(row, cut, n)
        na, nb = a[0], b[0]
        delta = b[1] - a[1]
        mean = a[1] + delta * nb / n
        m2 = a[2] + b[2] + delta * delta * na * nb / n
        assert whole[0] == n
        assert abs(mean - whole[1]) <= 1e-12 * max(1.0, abs(whole[3] / n))
        assert abs(m2 - whole[2]) <= 1e-10 * max(whole[2], 1e-300)


# ---------------------------------------------------------- the closed forms themselves
def _quad(row):
    d = int(row["dim"])
    lo, hi = row["lo"][:d], row["hi"][:d]
    fam = int(row["family"])
    p = row["p"]

    def f(*x):
        x = np.array(x)
        if fam == 0:
            ph = np.dot(p[2:2 + d], x)
            return p[0] * math.cos(ph) + p[1] * math.sin(ph)
        if fam == 1:
            return p[0] * abs(np.dot(p[1:1 + d], x))
        if fam == 2:
            return p[0] * math.exp(-np.sum((x - p[2:2 + d]) ** 2) / (2 * p[1] ** 2))
        return float(np.prod([np.polyval(p[5 * i:5 * i + int(row["deg"]) + 1][::-1], x[i])
                              for i in range(d)]))

    opts = {"limit": 200, "epsabs": 1e-10, "epsrel": 1e-10}
    val, _ = spi.nquad(f, [[lo[i], hi[i]] for i in range(d)], opts=[opts] * d)
    val2, _ = spi.nquad(lambda *x: f(*x) ** 2, [[lo[i], hi[i]] for i in range(d)],
                        opts=[opts] * d)
    return val, val2


def test_closed_forms_against_quadrature():
    """The analytic integrals (and integrals of f^2) agree with adaptive quadrature
    (1-D and 2-D boxes; the formulas are the same for every dimension)."""
    rng = np.random.default_rng(8)
    t = W.empty(7)
    W.harmonic(t[0], 1.3, -0.6, [7.0, -3.0], [-0.4, -1.0], [0.8, 0.3], 1)
    W.harmonic(t[1], 0.5, 2.0, [0.0], [-1.0], [0.5], 1)
    W.abslin(t[2], 1.2, [1.0, -1.0], [-1.0, -0.5], [0.5, 1.0], 1)
    W.abslin(t[3], 0.7, [2.0], [-1.0], [0.25], 1)
    W.abslin(t[4], 0.7, [1.0, 0.0], [-1.0, 0.0], [0.5, 2.0], 1)
    W.gauss(t[5], 1.0, 0.2, [0.1, -0.3], [-0.5, -1.0], [0.5, 0.2], 1)
    W.poly(t[6], rng.standard_normal((2, 4)), [-1.0, 0.0], [0.5, 1.5], 1)
    for row in t:
        q1, q2 = _quad(row)
        assert abs(CF.exact(row) - q1) < 1e-7 * max(1.0, abs(q1)), (row["family"], q1)
        assert abs(CF.second_moment(row) - q2) < 1e-7 * max(1.0, abs(q2))


def test_abslin_1d_closed_form():
    """d = 1: int_l^h |c x| dx = (c h |c h| - c l |c l|) / (2 c)."""
    for c, l, h in [(1.0, -1.0, 0.5), (-2.0, 0.25, 1.5), (0.5, -2.0, -0.5)]:
        t = W.empty(1)
        W.abslin(t[0], 1.0, [c], [l], [h], 1)
        want = (c * h * abs(c * h) - c * l * abs(c * l)) / (2 * c)
        assert abs(CF.exact(t[0]) - want) < 1e-15


def test_golden_fig1_regression(orc):
    """The oracle reproduces its stored Fig. 1 values bit for bit."""
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "fig1_oracle_n1e5.json")
    g = json.load(open(path))
    res, _ = orc.integrate(W.harmonic_fig1(10**5))
    for key in ("estimate", "stderr", "mean_abs"):
        want = np.array([float.fromhex(v) for v in g[key]])
        assert np.array_equal(res[key], want), key
