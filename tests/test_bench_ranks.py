"""The multi-rank path of bench.py (one replica per GPU under torchrun): the
whole-job value is the units all ranks processed over the slowest rank's
time.  Checked with two gloo ranks on the CPU (the reduction is host logic;
no GPU and no data-path collective are involved)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 1 + r seconds, 100 (r + 1) units
        value, t_max, total = bench.aggregate_ranks(1.0 + rank, 100.0 * (rank + 1), world, dist, "cpu")
        dist.barrier()
        results[rank] = (value, t_max, total)
    finally:
        dist.destroy_process_group()


def test_two_ranks_aggregate_on_cpu():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank, args=(world, port, results), nprocs=world, join=True)
        got = dict(results)
    assert sorted(got) == [0, 1]
    for r in range(world):
        value, t_max, total = got[r]
        assert t_max == 2.0 and total == 300.0
        assert value == 150.0                      # every rank reports the same whole-job value


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(2.0, 10.0, 1) == (5.0, 2.0, 10.0)
