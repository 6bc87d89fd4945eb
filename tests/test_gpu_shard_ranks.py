"""The multi-rank path through the library: two gloo ranks, each a process of
its own with its own library context on cuda:0, integrate their share of one
table with libzmc (row partition: zmc_integrate on whole integrands; sample
partition: shard.rank_moments -> zmc_integrate_moments on contiguous sample
ranges), and the shares are gathered over gloo.  Gathered rows must equal one
process integrating the whole table bit for bit; merged sample pieces must
equal it to FP64 rounding of the merge; both must match the FP64 oracle.  The
ranks' kernels are independent of each other (no kernel waits on another rank);
only the host exchanges results."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2104_10073_gb300 import shard
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

CHUNK = 160 * zmc.DEFAULT_QUINTS_PER_LANE


def _table():
    t = W.mixed(60, gen_seed=41, lo_exp=3.5, hi_exp=5.5)
    # rows start on chunk boundaries of the global sample sequence, so that the
    # sample pieces reproduce the unsplit chunk sums
    t["n_samples"] = (t["n_samples"] + CHUNK - 1) // CHUNK * CHUNK
    return t


def _worker(rank, world, port, path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = _table()
    with zmc.Context(arena_bytes=512 << 20) as ctx:
        mine = shard.partition_rows(t, world)[rank]
        res = zmc.zmc_integrate(ctx.handle, t[mine])
        rows = [(int(i), float(e), float(s), int(n))
                for i, e, s, n in zip(mine, res["estimate"], res["stderr"], res["n"])]
        pieces = shard.rank_moments(ctx.handle, t,
                                    shard.partition_samples(t, world, align=CHUNK)[rank])
    g_rows, g_pieces = [None] * world, [None] * world
    dist.all_gather_object(g_rows, rows)
    dist.all_gather_object(g_pieces, pieces)
    if rank == 0:
        np.save(path, np.array([g_rows, g_pieces], dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def gathered(tmp_path_factory, zctx):
    path = str(tmp_path_factory.mktemp("ranks") / "res.npy")
    mp.spawn(_worker, args=(2, _free_port(), path), nprocs=2, join=True)
    return np.load(path, allow_pickle=True)


def test_row_partition_over_two_processes(gathered, zctx):
    t = _table()
    rows_by_rank, _ = gathered
    est = np.full(len(t), np.nan)
    se = np.full(len(t), np.nan)
    n = np.zeros(len(t), dtype=np.uint64)
    for rows in rows_by_rank:
        assert rows, "each rank got some rows"
        for i, e, s, k in rows:
            est[i], se[i], n[i] = e, s, k
    full = zmc.zmc_integrate(zctx.handle, t)
    assert np.array_equal(est, full["estimate"])
    assert np.array_equal(se, full["stderr"], equal_nan=True)
    assert np.array_equal(n, full["n"])
    want, _ = oracle.integrate(t)
    got = full.copy()
    got["estimate"], got["stderr"] = est, se
    G.compare(t, got, want)


def test_sample_partition_over_two_processes(gathered, zctx):
    t = _table()
    _, pieces_by_rank = gathered
    assert all(pieces_by_rank)
    pieces = [p for rank in pieces_by_rank for p in rank]
    vols = [G.volume(r) for r in t]
    got = shard.merge_moments(len(t), pieces, vols)
    full = zmc.zmc_integrate(zctx.handle, t)
    want, _ = oracle.integrate(t)
    assert np.array_equal(got["n"], t["n_samples"])
    for i in range(len(t)):
        scale = vols[i] * want["mean_abs"][i]
        assert abs(got["estimate"][i] - full["estimate"][i]) <= 1e-12 * scale + 1e-300
    res = full.copy()
    res["estimate"], res["stderr"] = got["estimate"], got["stderr"]
    G.compare(t, res, want)
