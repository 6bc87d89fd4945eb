"""The bound the 32-bit abs-linear sum rests on (CPU, exact arithmetic): on any
box of up to 7 dimensions, mean |c.x| is at least a tenth of max |c.x|.

The library sums c.x in 32-bit integers for rows of >= 256 samples; its
per-sample error is below ~2e-8 of max |c.x|, so the estimate stays inside the
1e-6 mean|f| tolerance as long as mean |c.x| >= max |c.x| / 10 (with a margin
of five).  The density of c.x over a box is a convolution of uniform
densities; the mean of |c.x| is smallest relative to its maximum when the
hyperplane c.x = 0 passes through the box centre with equal widths |c_i| w_i
(0.17 for 7 dimensions).  Checked here with the exact closed form of the
integral of |c.x| over a box (the one that pins the oracle), for the worst
case in every dimension and for random boxes, coefficients and offsets."""
import itertools

import numpy as np

from paper_2104_10073_gb300 import workloads as W
from tests import closed_forms as CF


def _ratio(c, lo, hi):
    t = W.empty(1)
    W.abslin(t[0], 1.0, c, lo, hi, 10)
    mean = CF.abslin(t[0]) / CF.volume(t[0])
    smax = max(abs(sum(ci * (h if bit else l) for ci, l, h, bit in zip(c, lo, hi, corner)))
               for corner in itertools.product((0, 1), repeat=len(c)))
    return mean / smax


def test_worst_case_centred_equal_widths():
    for d in range(1, 8):
        r = _ratio([1.0] * d, [-0.5] * d, [0.5] * d)
        assert r >= 0.1, (d, r)
    # the 7-dimensional worst case is about 0.17
    assert 0.15 < _ratio([1.0] * 7, [-0.5] * 7, [0.5] * 7) < 0.2


def test_random_boxes():
    rng = np.random.default_rng(77)
    worst = 1.0
    for _ in range(400):
        d = int(rng.integers(1, 8))
        c = list(rng.choice([-1.0, 1.0], size=d) * 2.0 ** rng.integers(-3, 4, size=d))
        w = 2.0 ** rng.integers(-4, 3, size=d)
        # boxes centred on the hyperplane (two in three) or shifted along c
        shift = float(rng.choice([0.0, 0.0, rng.uniform(-1.0, 1.0)]))
        lo = list(-w / 2 + shift * np.sign(c) * w)
        hi = list(np.array(lo) + w)
        worst = min(worst, _ratio(c, lo, hi))
    assert worst >= 0.1, worst
