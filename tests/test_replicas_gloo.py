"""The N > 1 path of bench.py (independent replicas) on CPU: two gloo ranks with different timed
durations report the max duration and the whole-job rate (iterations of all ranks over it)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, value = bench.aggregate_replicas(10.0 + 5.0 * rank, 20, world)
        out[rank] = (ms, value)
    finally:
        torch.distributed.destroy_process_group()


def test_two_replicas_take_the_max_time_and_the_total_rate():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 15.0
        assert value == pytest.approx(world * 20 / 0.015)


def test_single_replica_needs_no_collective():
    import bench
    ms, value = bench.aggregate_replicas(8.0, 10, 1)
    assert ms == 8.0 and value == pytest.approx(1250.0)
