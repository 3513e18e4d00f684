"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) agree on the
job time (the slowest rank's) and on the replica throughput."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 250.0][rank]                    # each rank's own timed region
    ms_max = bench.reduce_max(ms, world, dist, torch.device("cpu"))
    value = bench.replica_throughput(world, 5, 32, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    results[rank] = (ms_max, value)


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank, args=(2, port, results), nprocs=2, join=True)
        got = dict(results)
    assert got[0] == got[1]
    ms_max, value = got[0]
    assert ms_max == 250.0
    assert value == pytest.approx(2 * 5 * 32 / 0.25)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.replica_throughput(1, 10, 32, 1000.0) == pytest.approx(320.0)
