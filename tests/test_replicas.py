"""The multi-GPU form is replicas only: N ranks run the same graph and the
job rate is N times one rank's cliques over the slowest rank's time. The
reduction is checked here on CPU with two gloo ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 100 + 50 r ms for 3 steps of 1000 cliques
        value, slowest = bench.replica_throughput(1000, 3, 100.0 + 50.0 * rank, dist, "cpu")
        out[rank] = (value, slowest)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for value, slowest in res.values():
        assert slowest == 150.0
        assert value == pytest.approx(1000 * 3 * 2 / 0.150)


def test_one_replica():
    sys.path.insert(0, ROOT)
    import bench
    value, slowest = bench.replica_throughput(500, 2, 40.0)
    assert slowest == 40.0 and value == pytest.approx(500 * 2 / 0.040)
