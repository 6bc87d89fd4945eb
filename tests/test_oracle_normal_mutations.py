"""Plausible mistakes planted in a copy of the stratified-sampling oracle
(oracle/normal.py) are each caught by at least one of its pins
(tests/test_oracle_normal.py), run against the mutated copy on the CPU."""
import importlib.util
import os
import sys

import numpy as np
import pytest

import oracle
from tests import test_oracle_normal as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "normal.py")

MUTANTS = [
    ("split threshold >= instead of >", "if not (s_c > tau and", "if not (s_c >= tau and"),
    ("variance sums s_c, not s_c^2", "var += res[c][1] * res[c][1]", "var += res[c][1]"),
    ("estimate over every cell, not the leaves", "    for c in leaves:\n        est += res[c][0]",
     "    for c in range(len(boxes)):\n        est += res[c][0]"),
    ("level-0 lower bound shifted by one cell", "cl.append(lo[i] + (w * idx) / k)",
     "cl.append(lo[i] + (w * (idx + 1)) / k)"),
    ("midpoint at the upper edge", "mid = cl0[i] + (ch0[i] - cl0[i]) * 0.5",
     "mid = cl0[i] + (ch0[i] - cl0[i])"),
    ("cell stderr divides by N^2", "math.sqrt(m2 / (n * (n - 1)))", "math.sqrt(m2 / (n * n))"),
    ("cell estimate without the volume", "out.append((V * mean,", "out.append((mean,"),
    ("threshold from the largest leaf error, not the mean",
     "tau = sigma_mult * (sum(res[c][1] for c in leaves) / len(leaves))",
     "tau = sigma_mult * max(res[c][1] for c in leaves)"),
    ("children keep the parent's stream", "streams.append(next_stream[0])\n                next_stream[0] += 1",
     "streams.append(streams[c])"),
]

PINS = [
    lambda: P.test_closed_form_high_dimension(8),
    P.test_builtin_family_cells_closed_form,
    P.test_leaves_partition_the_box,
    P.test_split_rule_extremes,
    P.test_constant_integrand_is_exact,
    P.test_stderr_is_calibrated_over_repeats,
    P.test_plain_limit_is_direct_monte_carlo,
    P.test_numpy_cells_match_the_c_oracle,
    P.test_children_draw_independent_samples,
]


def _load_mutant(old, new):
    text = open(SRC).read()
    assert old in text, old
    spec = importlib.util.spec_from_loader("oracle._normal_mutant", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    exec(compile(text.replace(old, new, 1), SRC, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(monkeypatch, name, old, new):
    mod = _load_mutant(old, new)
    monkeypatch.setattr(P, "normal", mod.normal)
    caught = []
    for pin in PINS:
        try:
            with np.errstate(invalid="ignore", divide="ignore"):
                pin()
        except AssertionError:
            caught.append(pin)
    assert caught, f"no pin catches: {name}"
