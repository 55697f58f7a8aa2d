"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own replica, report the
slowest rank's time and the units of both ranks (weak scaling, no collective on the data path)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [40.0, 55.0][rank]                       # rank 1 is the slow replica
    max_ms = bench.max_over_ranks(dist, ms, "cpu")
    rate = bench.whole_job_rate(world, 1000, 4, max_ms)
    dist.barrier()
    out.put((rank, max_ms, rate))
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_rate():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, rate in res:
        assert max_ms == 55.0                      # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * 1000 * 4 / 0.055)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    pytest.importorskip("torch")
    import bench
    assert bench.max_over_ranks(None, 12.5, "cpu") == 12.5
    assert bench.whole_job_rate(1, 10, 2, 1.0) == pytest.approx(20000.0)
