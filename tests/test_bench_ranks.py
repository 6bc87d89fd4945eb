"""The benchmark's multi-rank bookkeeping on CPU (2 gloo ranks): the step time
is the maximum over ranks, the sample count the sum (weak scaling: every rank
integrates its own 10 repeats, keys 10r .. 10r + 9)."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, path):
    import sys

    sys.path.insert(0, ROOT)
    import bench
    from paper_2104_10073_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tab = bench.fig1_table(rank)
    ms = bench.max_over_ranks(world, 3.0 + rank)
    total = bench.sum_over_ranks(world, float(W.total_samples(tab)))
    bench.barrier(world)
    keys = sorted(set(int(k) for k in tab["seed"]))
    if rank == 0:
        np.save(path, np.array([ms, total]))
    np.save(path + f".keys{rank}.npy", np.array(keys))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks(tmp_path):
    path = str(tmp_path / "r.npy")
    mp.spawn(_worker, args=(2, _free_port(), path), nprocs=2, join=True)
    ms, total = np.load(path)
    assert ms == 4.0 and total == 2 * 10**9
    k0 = np.load(path + ".keys0.npy")
    k1 = np.load(path + ".keys1.npy")
    assert list(k0) == list(range(10)) and list(k1) == list(range(10, 20))
