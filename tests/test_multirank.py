"""Multi-rank host logic of the benchmark, run as two gloo ranks on the CPU.

Problems are independent, so ranks shard them (weak scaling) and exchange nothing on the data
path; every rank gates its own problems against its own oracle run, and the only collective is
the whole-job figures (slowest rank's time, sum of passed solves)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cpu = torch.device("cpu")
        t, passed = bench.reduce_over_ranks(10.0 + 5.0 * rank, 3 + rank, cpu)
        probs = bench.make_problems("C1", 2, rank)
        out[rank] = (t, passed, [P.t.tolist() for P in probs])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, passed, _ = out[r]
        assert t == 15.0                      # slowest rank
        assert passed == 7.0                  # 3 + 4 solves
    # every rank draws its own problems: no two ranks solve the same instance
    t0 = [np.asarray(x) for x in out[0][2]]
    t1 = [np.asarray(x) for x in out[1][2]]
    for a in t0:
        for b in t1:
            assert a.shape != b.shape or not np.allclose(a, b)
