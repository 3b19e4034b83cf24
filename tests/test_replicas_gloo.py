"""The replica path of bench.py on CPU: two gloo ranks with different step
times report the slowest rank's time and both ranks' points."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_ms = 100.0 * (rank + 1)                 # rank 1 is the slower one
    ms, value = bench.aggregate(t_ms, steps=10, n_points=1000, world=world,
                                device=torch.device("cpu"))
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_replicas_aggregate():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == pytest.approx(20.0)                 # max(100, 200) / 10 steps
        assert value == pytest.approx(2 * 1000 / 20e-3 / 1e6)
