"""Multi-GPU host logic on CPU ranks (gloo, world size 2): the batch shards
are disjoint, complete and size-balanced, and the whole-job rate is the
units of all ranks over the slowest rank's time (the rule bench.py
applies at N GPUs)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2603_00035_gb300 import replicas  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard(sizes, rank, world)
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        flat = sorted(i for part in everyone for i in part)
        assert flat == list(range(len(sizes)))  # disjoint and complete
        loads = [sum(sizes[i] for i in part) for part in everyone]
        assert max(loads) - min(loads) <= max(sizes)  # greedy balance bound
        assert everyone[rank] == replicas.shard(sizes, rank, world)  # deterministic
        assert replicas.max_over_ranks(10.0 * rank + 5.0) == 15.0
        assert replicas.sum_over_ranks(rank + 1) == 3.0
        rate, ms = replicas.job_rate(units_local=rank + 1, ms_local=100.0 * (rank + 1))
        assert ms == 200.0 and abs(rate - 3 / 0.2) < 1e-9
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    sizes = [(64 + 37 * k % 960) * (32 + 11 * k % 480) for k in range(37)]
    mp.start_processes(_worker, args=(2, free_port(), sizes), nprocs=2, join=True, start_method="spawn")


def test_single_process_is_identity():
    assert replicas.shard([5, 3, 9], 0, 1) == [0, 1, 2]
    rate, ms = replicas.job_rate(4, 2000.0)
    assert ms == 2000.0 and rate == 2.0
