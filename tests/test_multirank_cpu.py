"""The multi-rank side of the benchmark on CPU: two gloo ranks combine their timings like the
NCCL ranks of a multi-GPU run (replicas: max of the timed seconds, sum of the particle-forces), and
every rank integrates a different seeded system."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_dev = 1.5 + rank          # rank 1 is the slow one
    sinks = 1000.0 * (rank + 1)
    t_max, sinks_all = bench.combine_ranks(t_dev, sinks, torch.device("cpu"), world)
    pos, _, _ = bench.workload("disk", 64, seed=1003 + rank)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([t_max, sinks_all]))
    np.save(os.path.join(out_dir, f"p{rank}.npy"), pos)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        t_max, sinks_all = np.load(tmp_path / f"r{r}.npy")
        assert t_max == 2.5 and sinks_all == 3000.0
    # replicas: each rank's system comes from its own seed
    assert not np.array_equal(np.load(tmp_path / "p0.npy"), np.load(tmp_path / "p1.npy"))


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(2.0, 10.0, torch.device("cpu"), 1) == (2.0, 10.0)
