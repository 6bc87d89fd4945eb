"""Pins of the stratified-sampling oracle (oracle/normal.py) against facts that do
not come from it: closed-form integrals, the partition the tree must form, the
exact behaviour of the split rule at its extremes, and the calibration of the
reported standard error over independent repetitions."""
import math

import numpy as np
import pytest
from scipy.special import erf

from oracle.normal import normal
from paper_2104_10073_gb300 import workloads as W


def gauss_prod(x, p):
    return np.exp(-np.sum((x - p[0]) ** 2, axis=1) / (2.0 * p[1] ** 2))


def gauss_prod_exact(lo, hi, mu, sigma):
    out = 1.0
    for a, b in zip(lo, hi):
        out *= sigma * math.sqrt(math.pi / 2) * (erf((b - mu) / (sigma * math.sqrt(2)))
                                                 - erf((a - mu) / (sigma * math.sqrt(2))))
    return out


@pytest.mark.parametrize("dim", [8, 10])
def test_closed_form_high_dimension(dim):
    lo, hi = [-1.0] * dim, [1.5] * dim
    p = np.array([0.2, 0.6])
    r = normal(dim, lo, hi, divisions=2, depth=2, samples_per_cell=1000, sigma_mult=1.5,
               seed=5, f=gauss_prod, p=p, max_leaves=4 * 2 ** dim)
    exact = gauss_prod_exact(lo, hi, 0.2, 0.6)
    assert r["rounds"] >= 1
    assert abs(r["estimate"] - exact) <= 5 * r["stderr"], (r["estimate"], exact, r["stderr"])


def test_builtin_family_cells_closed_form():
    """A 3-D Gaussian of the built-in family through the C oracle's cells."""
    row = W.empty(1)[0]
    W.gauss(row, 1.5, 0.3, [0.1, 0.4, 0.7], [-0.5, 0.0, 0.0], [1.0, 1.0, 1.2], 1)
    r = normal(3, row["lo"][:3], row["hi"][:3], divisions=3, depth=2, samples_per_cell=4096,
               sigma_mult=1.2, seed=2, row=row)
    exact = 1.5
    for a, b, m in zip([-0.5, 0.0, 0.0], [1.0, 1.0, 1.2], [0.1, 0.4, 0.7]):
        exact *= 0.3 * math.sqrt(math.pi / 2) * (erf((b - m) / (0.3 * math.sqrt(2)))
                                                 - erf((a - m) / (0.3 * math.sqrt(2))))
    assert abs(r["estimate"] - exact) <= 5 * r["stderr"]
    assert r["rounds"] >= 1 and r["n_leaves"] > 27


def test_leaves_partition_the_box():
    lo, hi = [-1.0, 0.5], [2.0, 3.0]
    r = normal(2, lo, hi, divisions=3, depth=3, samples_per_cell=64, sigma_mult=0.8, seed=1,
               f=lambda x, p: np.exp(3 * x[:, 0]) * np.cos(2 * x[:, 1]), p=None)
    leaves = r["leaves"]
    vol = sum((b[0] - a[0]) * (b[1] - a[1]) for a, b in leaves)
    assert abs(vol - 7.5) <= 1e-12 * 7.5
    rng = np.random.default_rng(0)
    pts = rng.uniform(lo, hi, size=(4000, 2))
    inside = np.zeros(len(pts), dtype=int)
    for a, b in leaves:
        inside += np.all((pts >= a) & (pts < b), axis=1)
    assert np.all(inside == 1)
    assert r["n_cells"] == 9 + (r["n_cells"] - 9)  # level 0 plus children
    assert (r["n_cells"] - 9) % 4 == 0 and r["n_leaves"] == 9 + 3 * (r["n_cells"] - 9) // 4


def test_split_rule_extremes():
    f = lambda x, p: 1.0 + x[:, 0] * x[:, 1]  # noqa: E731
    none = normal(2, [0, 0], [1, 1], divisions=2, depth=3, samples_per_cell=32, sigma_mult=1e9,
                  f=f, p=None)
    assert none["rounds"] == 0 and none["n_cells"] == 4 and none["n_leaves"] == 4
    # a threshold below every s_c splits every leaf of every round
    allr = normal(2, [0, 0], [1, 1], divisions=2, depth=2, samples_per_cell=32,
                  sigma_mult=1e-9, f=f, p=None)
    assert allr["rounds"] == 2 and allr["n_leaves"] == 4 * 4 * 4
    assert allr["n_cells"] == 4 + 16 + 64
    capped = normal(2, [0, 0], [1, 1], divisions=2, depth=2, samples_per_cell=32,
                    sigma_mult=1e-9, max_leaves=10, f=f, p=None)
    # 4 leaves: two splits fit (4 -> 7 -> 10), the third would exceed 10
    assert capped["n_leaves"] == 10 and capped["rounds"] == 1


def test_constant_integrand_is_exact():
    r = normal(4, [0] * 4, [2, 1, 1, 0.5], divisions=2, depth=2, samples_per_cell=16,
               f=lambda x, p: np.full(len(x), 3.0), p=None)
    assert r["stderr"] == 0.0 and r["rounds"] == 0
    assert abs(r["estimate"] - 3.0) <= 1e-15 * 3


def test_stderr_is_calibrated_over_repeats():
    """The spread of 200 independent stratified estimates matches the reported
    standard error (chi-square band for 199 degrees of freedom)."""
    f = lambda x, p: np.sin(3 * x[:, 0]) + x[:, 1] ** 2  # noqa: E731
    est, se = [], []
    for s in range(200):
        r = normal(2, [0, 0], [1, 1], divisions=2, depth=1, samples_per_cell=64,
                   sigma_mult=1.0, seed=s, f=f, p=None)
        est.append(r["estimate"])
        se.append(r["stderr"])
    ratio = np.var(est, ddof=1) / np.mean(np.square(se))
    assert 0.7 < ratio < 1.35, ratio


def test_plain_limit_is_direct_monte_carlo():
    """divisions 1, depth 0: one cell, the plain direct MC estimate of the box
    with stream stream_base; equals the oracle's integrate of that row."""
    import oracle

    row = W.harmonic_fig1(4096)[17]
    r = normal(4, row["lo"][:4], row["hi"][:4], divisions=1, depth=0, samples_per_cell=4096,
               seed=int(row["seed"]), stream_base=int(row["stream_id"]), row=row)
    want, _ = oracle.integrate(np.asarray(row).reshape(1))
    assert r["estimate"] == want["estimate"][0] and r["stderr"] == want["stderr"][0]


def test_numpy_cells_match_the_c_oracle():
    """The numpy cell path (mean and M2 by definition) against the C oracle's
    Welford on the same Eq. 1 integrand: one cell, the plain direct-MC limit."""
    import oracle

    row = W.harmonic_fig1(20000)[33]

    def harm(x, p):
        return p[0] * np.cos(x @ p[2:6]) + p[1] * np.sin(x @ p[2:6])

    r = normal(4, row["lo"][:4], row["hi"][:4], divisions=1, depth=0, samples_per_cell=20000,
               seed=int(row["seed"]), stream_base=int(row["stream_id"]), f=harm,
               p=np.asarray(row["p"]))
    want, _ = oracle.integrate(np.asarray(row).reshape(1))
    assert abs(r["estimate"] - want["estimate"][0]) <= 1e-12 * abs(want["mean_abs"][0])
    assert abs(r["stderr"] - want["stderr"][0]) <= 1e-10 * want["stderr"][0]


def test_children_draw_independent_samples():
    """After a split the halves' estimates must be independent: for f(x) = x on
    [0, 1] with the root always split, the spread of the estimate over 300
    repetitions matches sqrt(sum of the halves' s_c^2) (samples shared between
    the halves would double the variance)."""
    est, se = [], []
    for s in range(300):
        r = normal(1, [0.0], [1.0], divisions=1, depth=1, samples_per_cell=16, sigma_mult=0.5,
                   seed=1000 + s, f=lambda x, p: x[:, 0], p=None)
        assert r["rounds"] == 1 and r["n_leaves"] == 2
        est.append(r["estimate"])
        se.append(r["stderr"])
    ratio = np.var(est, ddof=1) / np.mean(np.square(se))
    assert 0.75 < ratio < 1.33, ratio
