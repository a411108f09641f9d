"""Replica aggregation of bench.py on CPU ranks (gloo, world size 2): each rank
sorts its own copy, the whole-job rate is all ranks' keys over the slowest
rank's time, and nothing else crosses ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, tmax = bench.replica_throughput(2.0 + rank, 1000, dist, "cpu")
    q.put((rank, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    ps = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, tmax in got:
        assert tmax == 3.0                           # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 1000 / 3.0e-3)


def test_replica_throughput_single():
    import bench
    value, tmax = bench.replica_throughput(4.0, 1000, None, "cpu")
    assert (value, tmax) == (1000 / 4.0e-3, 4.0)
