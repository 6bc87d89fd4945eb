"""FP64 oracle of stratified sampling with a heuristic tree search (test
infrastructure; only tests/ may import it).

The paper's ZMCintegral_normal (Sec. "Solution method", "Additional comments")
stratifies the integration domain and refines the strata by a heuristic tree
search, for integrands of 8 to 12 dimensions; it gives no steps.  This module
states the reading the library implements, one step at a time, in plain Python
over the oracle's own samples and FP64 integrand evaluations:

1. Level 0: the box is cut into k^d equal cells, k = ``divisions``; cell j has
   grid index (j // k**i) % k in dimension i, boundaries
   lo_i + ((hi_i - lo_i) * idx) / k, the last one hi_i.
2. Each cell is integrated by direct Monte Carlo with ``samples_per_cell``
   samples: the j-th cell created uses Philox stream ``stream_base + j`` under
   key ``seed``; e_c = V_c * mean, s_c = V_c * sqrt(M2 / (N (N - 1))).
3. Up to ``depth`` rounds: tau = sigma_mult * (sum of s_c over the leaves) /
   (number of leaves); in leaf order, each leaf with s_c > tau is split into its
   2^d halves (child b takes the upper half of dimension i when bit i of b is
   set; mid = lo + (hi - lo) * 0.5) while the leaf count stays within
   ``max_leaves``; children take their parent's place in the leaf order, get
   the next streams and are integrated as in step 2.  A round that splits
   nothing ends the search.
4. estimate = sum of e_c over the leaves (leaf order), stderr = sqrt(sum s_c^2).

The integrand is either a built-in family descriptor (its cells are integrated
by the C oracle, ``oracle.integrate``) or a numpy function f(x, p) evaluated at
the oracle's sample points (``oracle.points``), mean and M2 by their definitions.
"""
from __future__ import annotations

import math

import numpy as np

from . import integrate, points


def _cells_builtin(row, cells, n, seed):
    t = np.repeat(np.asarray(row).reshape(1), len(cells))
    d = int(row["dim"])
    for q, (lo, hi, stream) in enumerate(cells):
        t[q]["lo"][:d], t[q]["hi"][:d] = lo, hi
        t[q]["n_samples"], t[q]["seed"], t[q]["stream_id"] = n, seed, stream
    res, _ = integrate(t)
    return [(float(r["estimate"]), float(r["stderr"]), float(r["mean_abs"])) for r in res]


def _cells_numpy(f, p, cells, n, seed):
    out = []
    for lo, hi, stream in cells:
        x = points(len(lo), lo, hi, seed, stream, 0, n)
        fx = np.asarray(f(x, p), dtype=np.float64)
        V = float(np.prod(np.asarray(hi) - np.asarray(lo)))
        mean = float(fx.mean())
        m2 = float(np.sum((fx - mean) ** 2))
        out.append((V * mean, V * math.sqrt(m2 / (n * (n - 1))), float(np.abs(fx).mean())))
    return out


def normal(dim, lo, hi, divisions=2, depth=2, samples_per_cell=1 << 14, sigma_mult=2.0,
           seed=0, stream_base=0, max_leaves=1 << 20, row=None, f=None, p=None):
    """Returns a dict: estimate, stderr, n_samples, n_cells, n_leaves, rounds,
    scale (sum over leaves of V_c mean|f|_c), margin (the smallest |s_c - tau| / tau
    over every split decision taken), leaves (their (lo, hi) boxes)."""
    lo = [float(v) for v in lo]
    hi = [float(v) for v in hi]
    k = int(divisions)
    n = int(samples_per_cell)
    next_stream = [int(stream_base)]

    def evaluate(new):
        if row is not None:
            return _cells_builtin(row, new, n, seed)
        return _cells_numpy(f, p, new, n, seed)

    # step 1: level-0 grid
    boxes, streams = [], []
    for j in range(k ** dim):
        cl, ch = [], []
        r = j
        for i in range(dim):
            idx = r % k
            r //= k
            w = hi[i] - lo[i]
            cl.append(lo[i] + (w * idx) / k)
            ch.append(hi[i] if idx + 1 == k else lo[i] + (w * (idx + 1)) / k)
        boxes.append((cl, ch))
        streams.append(next_stream[0])
        next_stream[0] += 1
    # step 2
    res = evaluate([(b[0], b[1], s) for b, s in zip(boxes, streams)])
    leaves = list(range(len(boxes)))
    rounds = 0
    margin = math.inf
    # step 3
    for _ in range(depth):
        tau = sigma_mult * (sum(res[c][1] for c in leaves) / len(leaves))
        nxt, new = [], []
        n_leaves = len(leaves)
        for c in leaves:
            s_c = res[c][1]
            if tau > 0:
                margin = min(margin, abs(s_c - tau) / tau)
            if not (s_c > tau and n_leaves + 2 ** dim - 1 <= max_leaves):
                nxt.append(c)
                continue
            n_leaves += 2 ** dim - 1
            cl0, ch0 = boxes[c]
            for b in range(2 ** dim):
                cl, ch = [], []
                for i in range(dim):
                    mid = cl0[i] + (ch0[i] - cl0[i]) * 0.5
                    upper = (b >> i) & 1
                    cl.append(mid if upper else cl0[i])
                    ch.append(ch0[i] if upper else mid)
                boxes.append((cl, ch))
                streams.append(next_stream[0])
                next_stream[0] += 1
                new.append(len(boxes) - 1)
                nxt.append(len(boxes) - 1)
        if not new:
            break
        res += evaluate([(boxes[c][0], boxes[c][1], streams[c]) for c in new])
        leaves = nxt
        rounds += 1
    # step 4
    est = 0.0
    var = 0.0
    scale = 0.0
    for c in leaves:
        est += res[c][0]
        var += res[c][1] * res[c][1]
        V = float(np.prod(np.asarray(boxes[c][1]) - np.asarray(boxes[c][0])))
        scale += V * res[c][2]
    return {"estimate": est, "stderr": math.sqrt(var), "n_samples": len(boxes) * n,
            "n_cells": len(boxes), "n_leaves": len(leaves), "rounds": rounds, "scale": scale,
            "margin": margin, "leaves": [boxes[c] for c in leaves]}
