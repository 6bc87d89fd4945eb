"""Splitting one integration table over several ranks (host logic only).

The work of the method is embarrassingly parallel: integrands are independent,
and within an integrand every sample is addressed by its Philox counter, so any
partition of the samples reproduces exactly the same samples.  Two partitions:

* :func:`partition_rows` gives each rank whole integrands, balanced by sample
  budget (longest-processing-time greedy).  Each rank runs its rows through the
  library unchanged; since a row's result does not depend on which other rows
  share a launch, gathering the rows back in table order gives the same results
  as one rank running the whole table.  No collective touches the data path.
* :func:`partition_samples` cuts the global sample sequence (rows in table
  order, samples in order within a row) into contiguous, equally sized ranges,
  one per rank, so a single huge integrand can be spread too.  Each rank
  reports per-piece moments (n, mean, M2); :func:`merge_moments` combines the
  pieces of each row in rank order with Chan's pairwise update: the one
  exchange step (three numbers per piece).
"""
from __future__ import annotations

import heapq
import math

import numpy as np


def partition_rows(table, world: int) -> list[np.ndarray]:
    """Row indices per rank, balanced by ``n_samples`` (deterministic)."""
    n = np.asarray(table["n_samples"], dtype=np.float64)
    order = sorted(range(len(n)), key=lambda i: (-n[i], i))
    heap = [(0.0, r) for r in range(world)]
    rows = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        rows[r].append(i)
        heapq.heappush(heap, (load + n[i], r))
    return [np.array(sorted(r), dtype=np.int64) for r in rows]


def partition_samples(table, world: int, align: int = 1) -> list[list[tuple[int, int, int]]]:
    """Contiguous (row, s_begin, s_end) pieces per rank covering every sample once.

    Rank boundaries are rounded down to multiples of ``align`` within the global
    sample sequence; ``align`` = the library's chunk length (160 * quints_per_lane)
    makes each piece start on a chunk of its row whenever rows start on one
    (pieces then reproduce the unsplit chunk sums exactly)."""
    n = [int(v) for v in table["n_samples"]]
    total = sum(n)
    bounds = [(total * r // world) // align * align for r in range(world)] + [total]
    pieces = [[] for _ in range(world)]
    start = 0
    for row, cnt in enumerate(n):
        lo, hi = start, start + cnt
        for r in range(world):
            a, b = max(lo, bounds[r]), min(hi, bounds[r + 1])
            if a < b:
                pieces[r].append((row, a - start, b - start))
        start = hi
    return pieces


def chan_merge(a, b):
    """Combine two (n, mean, M2) summaries."""
    na, ma, qa = a
    nb, mb, qb = b
    n = na + nb
    if nb == 0:
        return a
    if na == 0:
        return b
    d = mb - ma
    return (n, ma + d * nb / n, qa + qb + d * d * na * nb / n)


def merge_moments(n_rows: int, pieces, volumes) -> np.ndarray:
    """Estimates from ``pieces`` = iterable of (row, n, mean, M2), taken in the
    order given (rank order); returns a structured array (estimate, stderr, n)."""
    acc = [(0.0, 0.0, 0.0) for _ in range(n_rows)]
    for row, n, mean, m2 in pieces:
        acc[row] = chan_merge(acc[row], (float(n), float(mean), float(m2)))
    out = np.zeros(n_rows, dtype=[("estimate", "f8"), ("stderr", "f8"), ("n", "u8")])
    for i, (n, mean, m2) in enumerate(acc):
        v = float(volumes[i])
        out["estimate"][i] = v * mean
        out["stderr"][i] = v * math.sqrt(m2 / (n * (n - 1))) if n > 1 else math.nan
        out["n"][i] = int(n)
    return out


def rank_moments(ctx_handle: int, table, pieces) -> list[tuple[int, float, float, float]]:
    """(row, n, mean, M2) of this rank's pieces computed by the library (the
    device counterpart of the CPU oracle's moments); piece starts must be
    multiples of 5 (whole quints)."""
    from . import zmc

    if not pieces:
        return []
    rows = np.array([p[0] for p in pieces], dtype=np.int64)
    m = zmc.zmc_integrate_moments(ctx_handle, table[rows], [p[1] for p in pieces],
                                  [p[2] for p in pieces])
    return [(int(r), float(k["n"]), float(k["mean"]), float(k["m2"])) for r, k in zip(rows, m)]
