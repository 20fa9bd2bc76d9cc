"""The multi-process path of bench.py on CPU: N replicas (gloo, world size 2) each time their own
work; the job takes the slowest rank's time and the whole-job throughput counts every rank's units.
No GPU is used and no data-path collective exists (only the timing reduction)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_seconds = 2.0 if rank == 1 else 1.0  # rank 1 is the slow one
    sec, ups = bench.replica_throughput(dist, local_seconds, units_per_step=1000.0, steps=5, device="cpu")
    out.put((rank, sec, ups))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, sec, ups in res:
        assert sec == 2.0  # max over ranks
        assert ups == pytest.approx(2 * 1000.0 * 5 / 2.0)  # both ranks' units over the job time


def test_single_process_has_no_reduction():
    import bench

    assert bench.replica_throughput(None, 4.0, 10.0, 3) == (4.0, 7.5)
