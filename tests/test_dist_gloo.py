"""The multi-rank host logic on CPU: two gloo ranks each take their share of a batch (no
data exchange), the shares cover every instance once and balance the N^3 cost, and the step
time is reduced to the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_2306_12616_gb300.dist import instance_cost, lpt_partition, rank_share, reduce_max


def test_lpt_partition_covers_and_balances():
    ns = [int(n) for n in synth.batch_sizes(512, 4000)]
    costs = [instance_cost(n) for n in ns]
    for world in (1, 2, 3, 8):
        parts = lpt_partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(ns)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT: the heaviest rank exceeds the mean by at most the largest single cost
        assert max(loads) <= sum(costs) / world + max(costs)
        assert max(loads) <= 1.05 * sum(costs) / world


def test_rank_share_is_deterministic_without_communication():
    ns = [64, 1024, 300, 300, 900, 128, 512]
    a = [rank_share(ns, r, 3) for r in range(3)]
    b = [rank_share(list(ns), r, 3) for r in range(3)]
    assert a == b and sorted(sum(a, [])) == list(range(len(ns)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ns, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    share = rank_share(ns, rank, world)
    # a stand-in for the rank's step time: proportional to its share of the work
    t = sum(instance_cost(ns[i]) for i in share) * 1e-9
    out[rank] = (share, t, reduce_max(t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ns = [int(n) for n in synth.batch_sizes(64, 7)]
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(2, port, ns, out), nprocs=2, join=True, start_method="spawn")
    shares = [out[r][0] for r in range(2)]
    assert sorted(shares[0] + shares[1]) == list(range(len(ns)))
    tmax = max(out[r][1] for r in range(2))
    assert out[0][2] == pytest.approx(tmax) and out[1][2] == pytest.approx(tmax)
