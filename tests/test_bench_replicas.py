"""The multi-rank path of the benchmark on CPU: replicas on two gloo ranks
report the units of all ranks over the slowest rank's time (no GPU)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    units = 1000.0 * (rank + 1)          # ranks that did different amounts of work
    secs = 2.0 + rank                    # and took different times
    value, slowest = bench.replica_throughput(units, secs, dist, "cpu")
    out.put((rank, value, slowest))
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, slowest in got:
        assert slowest == 3.0
        assert value == pytest.approx(3000.0 / 3.0)


def test_replica_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    value, secs = bench.replica_throughput(500.0, 0.5)
    assert (value, secs) == (1000.0, 0.5)
