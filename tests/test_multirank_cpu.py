"""The N > 1 path of bench.py: ranks are replicas (each solves its own copy),
the timed region is the maximum over ranks, and the reported value is the
work of all ranks over that time.  Run as world_size-2 gloo ranks on CPU."""
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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [100.0, 250.0][rank]          # rank 1 is the slow one
    ms_max, value = bench.whole_job(ms_local, units_per_rank=5, world=world)
    out.put((rank, ms_max, value))
    dist.destroy_process_group()


def test_whole_job_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 250.0                   # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 5 / 0.25)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(50.0, 3, 1) == (50.0, pytest.approx(60.0))
