"""Seeded random tables against the FP64 oracle (GPU): every family and every
evaluation form the library picks (general and equal-rate harmonics, 64- and
32-bit abs-linear sums, near and far Gaussians, polynomials of degree 0..4 in
coefficient and root form), dimensions 1..7, sample counts log-uniform over
1..2e5 mixed with sizes at the quint and chunk boundaries, random 64-bit keys,
stream ids up to 2^32 - 1, and the chunk length drawn per table from the
autotuner's candidates."""
import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

EDGES = [1, 2, 4, 5, 6, 255, 256, 257, 4159, 4160, 4161, 16639, 16640, 16641, 33281]


def _row(rng, r, i):
    fam = int(rng.integers(0, 4))
    d = int(rng.integers(1, 8))
    n = int(EDGES[rng.integers(0, len(EDGES))]) if rng.random() < 0.3 else \
        int(round(10 ** rng.uniform(0.0, np.log10(2e5))))
    lo = rng.uniform(-1.0, 0.0, size=d)
    w = rng.uniform(0.5, 2.0, size=d)
    key = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
    sid = int(rng.choice([rng.integers(0, 2**32), 2**32 - 1 - int(rng.integers(0, 4))]))
    if fam == W.HARMONIC:
        if d >= 2 and rng.random() < 0.4:  # equal rates: one wave number on a cube
            w = np.full(d, w[0])
            k = np.full(d, rng.uniform(-40.0, 40.0))
        else:
            k = rng.uniform(-40.0, 40.0, size=d)
        W.harmonic(r, rng.uniform(-2, 2), rng.uniform(-2, 2), k, lo, lo + w, n, key, sid)
    elif fam == W.ABSLIN:
        c = rng.choice([-1.0, 1.0], size=d) * 10 ** rng.uniform(-3, 3, size=d)
        W.abslin(r, rng.uniform(0.5, 2.0), c, lo, lo + w, n, key, sid)
    elif fam == W.GAUSS:
        far = rng.random() < 0.3
        mu = lo + w * (rng.uniform(2.5, 4.0, size=d) if far else rng.uniform(0, 1, size=d))
        W.gauss(r, rng.uniform(0.5, 2.0), rng.uniform(0.05, 0.8), mu, lo, lo + w, n, key, sid)
    else:
        deg = int(rng.integers(0, 5))
        coef = rng.standard_normal(size=(d, deg + 1))
        if deg >= 2 and rng.random() < 0.3:
            # a factor of lower degree than the row's keeps the coefficient form
            coef[int(rng.integers(0, d)), deg] = 0.0
        W.poly(r, coef, lo, lo + w, n, key, sid)


def table(seed):
    """The seed's table of 160 rows and the chunk length (quints per lane) it
    runs with."""
    rng = np.random.default_rng(10_000 + seed)
    t = W.empty(160)
    for i in range(len(t)):
        _row(rng, t[i], i)
    return t, int(rng.choice([26, 52, 104, 208]))


@pytest.mark.parametrize("seed", range(10))
def test_random_tables_match_the_oracle(zctx, seed):
    t, q = table(seed)
    with zmc.Context(arena_bytes=512 << 20, quints_per_lane=q) as c:
        got = zmc.zmc_integrate(c.handle, t)
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)
