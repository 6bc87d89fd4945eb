"""Multi-rank splitting on CPU: world_size 2 over gloo.

Each rank computes its share with the FP64 oracle (standing in for its GPU),
the shares are gathered, and the result must equal one rank doing everything:
bit for bit for the row partition (row results do not depend on the partition),
to rounding for the sample partition (Chan's merge of FP64 pieces).
"""
import math
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2104_10073_gb300 import shard
from paper_2104_10073_gb300 import workloads as W


def _table():
    t = W.random_table(23, np.random.default_rng(17), n_lo=1, n_hi=40000)
    big = W.empty(1)
    W.harmonic(big[0], 1.2, 0.7, [3.0, -2.0], [0.0, -0.5], [1.0, 0.5], 150000, seed=4,
               stream_id=99)
    return np.concatenate([t, big])


def _volumes(t):
    return [float(np.prod(r["hi"][:int(r["dim"])] - r["lo"][:int(r["dim"])])) for r in t]


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = _table()
    # row partition: whole integrands per rank
    mine = shard.partition_rows(t, world)[rank]
    res, _ = oracle.integrate(t[mine], threads=1)
    rows = [(int(i), float(e), float(s)) for i, e, s in zip(mine, res["estimate"], res["stderr"])]
    gathered = [None] * world
    dist.all_gather_object(gathered, rows)
    # sample partition: contiguous sample ranges, moments exchanged
    pieces = []
    for row, a, b in shard.partition_samples(t, world)[rank]:
        n, mean, m2, _ = oracle.moments(t[row], a, b)
        pieces.append((row, n, mean, m2))
    gp = [None] * world
    dist.all_gather_object(gp, pieces)
    if rank == 0:
        np.save(result_path, np.array([gathered, gp], dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def gathered(tmp_path_factory):
    path = str(tmp_path_factory.mktemp("shard") / "res.npy")
    mp.spawn(_worker, args=(2, _free_port(), path), nprocs=2, join=True)
    return np.load(path, allow_pickle=True)


def test_row_partition_matches_single_rank_bitwise(gathered):
    t = _table()
    rows_by_rank, _ = gathered
    est = np.full(len(t), np.nan)
    se = np.full(len(t), np.nan)
    seen = 0
    for rows in rows_by_rank:
        for i, e, s in rows:
            est[i], se[i] = e, s
            seen += 1
    assert seen == len(t)
    want, _ = oracle.integrate(t)
    assert np.array_equal(est, want["estimate"])
    assert np.array_equal(se, want["stderr"], equal_nan=True)


def test_sample_partition_merges_to_single_rank(gathered):
    t = _table()
    _, pieces_by_rank = gathered
    pieces = [p for rank in pieces_by_rank for p in rank]
    got = shard.merge_moments(len(t), pieces, _volumes(t))
    want, _ = oracle.integrate(t)
    assert np.array_equal(got["n"], t["n_samples"])
    for i in range(len(t)):
        scale = abs(want["estimate"][i]) + want["mean_abs"][i] * _volumes(t)[i]
        assert abs(got["estimate"][i] - want["estimate"][i]) <= 1e-12 * scale
        if t["n_samples"][i] > 1:
            assert abs(got["stderr"][i] - want["stderr"][i]) <= 1e-9 * want["stderr"][i] + 1e-15


def test_partitions_cover_everything_once():
    t = _table()
    for world in (1, 2, 3, 8):
        rows = shard.partition_rows(t, world)
        assert sorted(np.concatenate(rows).tolist()) == list(range(len(t)))
        loads = [int(np.sum(t["n_samples"][r])) for r in rows]
        assert max(loads) - min(loads) <= int(t["n_samples"].max())
        pieces = shard.partition_samples(t, world)
        cover = {}
        for rank in pieces:
            for row, a, b in rank:
                cover.setdefault(row, []).append((a, b))
        for row in range(len(t)):
            segs = sorted(cover[row])
            assert segs[0][0] == 0 and segs[-1][1] == int(t["n_samples"][row])
            assert all(segs[k][1] == segs[k + 1][0] for k in range(len(segs) - 1))
        sizes = [sum(b - a for _, a, b in rank) for rank in pieces]
        assert max(sizes) - min(sizes) <= 1
        assert math.isclose(sum(sizes), int(np.sum(t["n_samples"])))
