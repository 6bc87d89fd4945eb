"""Shared helpers of the GPU parity tests: the library context and the stated
tolerances.

Tolerances (per integrand, CUDA path against the FP64 oracle on the same
Philox samples):

* estimate: |est_gpu - est_oracle| <= 1e-6 * V * mean|f|_oracle, plus an
  absolute floor V * B * 2^-100, B an upper bound of |f| over the box: the FP32
  path works on 2^48-scaled values and resolves integrand values down to about
  2^-111 B (squares) and 2^-126 B (values); smaller ones are lost, which only
  shows when every sample of an integrand lies there (far Gaussian tails).
* standard error: |se_gpu - se_oracle| <= 1e-4 * se_oracle
  + 2e-6 * V * mean|f|_oracle / sqrt(N) (the second term covers tiny samples,
  where the spread is a difference of nearly equal FP32 values);
  N = 1 gives NaN on both sides.
* Philox words: bit-exact.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc

EST_REL = 1e-6
SE_REL = 1e-4


def volume(row) -> float:
    d = int(row["dim"])
    return float(np.prod(row["hi"][:d] - row["lo"][:d]))


def floor_abs(row) -> float:
    return volume(row) * sample_scale(row) * 2.0**-100


def compare(table, got, want, est_rel=EST_REL, se_rel=SE_REL):
    """Assert the GPU results ``got`` match oracle results ``want`` row by row.
    Returns the largest |d est| / (V mean|f|) seen (for reporting)."""
    worst = 0.0
    bad = []
    for i, row in enumerate(table):
        V = volume(row)
        N = int(row["n_samples"])
        scale = V * want["mean_abs"][i]
        d_est = abs(got["estimate"][i] - want["estimate"][i])
        tol = est_rel * scale + floor_abs(row)
        if scale > 0:
            worst = max(worst, d_est / scale)
        ok = d_est <= tol and int(got["n"][i]) == N and got["status"][i] == 0
        if N == 1:
            ok = ok and math.isnan(got["stderr"][i]) and math.isnan(want["stderr"][i])
        else:
            se_w = want["stderr"][i]
            tol_se = se_rel * se_w + 2e-6 * scale / math.sqrt(N) + floor_abs(row)
            ok = ok and abs(got["stderr"][i] - se_w) <= tol_se
        if not ok:
            bad.append((i, int(row["family"]), int(row["dim"]), int(row["deg"]), N,
                        got["estimate"][i], want["estimate"][i], got["stderr"][i],
                        want["stderr"][i], scale))
    assert not bad, f"{len(bad)} rows out of tolerance, first: {bad[:3]}"
    return worst


def sample_scale(row) -> float:
    """A bound on |f| over the box, for per-sample comparisons."""
    fam, d = int(row["family"]), int(row["dim"])
    lo, hi, p = row["lo"][:d], row["hi"][:d], row["p"]
    if fam == W.USER:  # no bound is known for a user-defined integrand
        return 0.0
    if fam == W.HARMONIC:
        return abs(p[0]) + abs(p[1])
    if fam == W.ABSLIN:
        return abs(p[0]) * float(np.sum(np.abs(p[1:1 + d]) * (np.abs(lo) + 2 * (hi - lo))))
    if fam == W.GAUSS:
        return abs(p[0])
    m = np.maximum(np.abs(lo), np.abs(hi))
    deg = int(row["deg"])
    return float(np.prod([np.sum(np.abs(p[5 * i:5 * i + deg + 1]) * m[i] ** np.arange(deg + 1))
                          for i in range(d)]))
