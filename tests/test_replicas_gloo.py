"""The multi-GPU form is replicas only: every rank simulates its own network and the benchmark
reports the sum of the events over the slowest rank's time.  This checks that path on the CPU
with two gloo ranks, each running the oracle on its own replica."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from helpers import oracle_run
    from paper_2406_03762_gb300 import workloads as W
    spec = W.NetSpec(400, 100, 40, 10)
    seed = bench.replica_seed(W.CONFIGS["c0"]["seed"], rank)
    ref, s, i, _ = oracle_run(spec, seed, 300)
    ms = 10.0 + 5.0 * rank                       # stand-in for each rank's measured time
    ms_max, ev_all = bench.replica_aggregate(ms, ref.events, dist, "cpu")
    np.save(os.path.join(out, f"r{rank}.npy"), np.array([seed, ref.events, ms_max, ev_all, len(s)], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_events_and_take_the_slowest_time(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] != r1[0]                        # distinct replicas
    assert r0[1] != r1[1] or r0[4] != r1[4]      # ... with different activity
    for r in (r0, r1):
        assert r[2] == 15.0                      # max over ranks
        assert r[3] == r0[1] + r1[1]             # sum over ranks
