"""Replica bookkeeping with world-size-2 gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2506_20809_gb300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = R.shard(len(costs), rank, world, costs)
    load = float(sum(costs[k] for k in mine))
    dist.barrier()
    mx = R.max_over_ranks(load, world)
    out[rank] = (mine, load, mx)
    dist.destroy_process_group()


def test_shard_round_robin_and_lpt():
    assert R.shard(5, 0, 2) == [0, 2, 4] and R.shard(5, 1, 2) == [1, 3]
    costs = [10, 1, 1, 1, 9, 2]
    a, b = R.shard(6, 0, 2, costs), R.shard(6, 1, 2, costs)
    assert sorted(a + b) == list(range(6)) and not set(a) & set(b)
    la, lb = sum(costs[k] for k in a), sum(costs[k] for k in b)
    assert abs(la - lb) <= max(costs)
    with pytest.raises(ValueError):
        R.shard(3, 2, 2)


def test_two_gloo_ranks_split_and_max():
    costs = [float(c) for c in (400, 10, 120, 30, 250, 80, 60, 15)]
    manager = mp.Manager()
    out = manager.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, costs, out), nprocs=2, join=True)
    (m0, l0, x0), (m1, l1, x1) = out[0], out[1]
    assert sorted(m0 + m1) == list(range(len(costs))) and not set(m0) & set(m1)
    assert x0 == x1 == max(l0, l1)
