"""The N > 1 replica path of bench.py on CPU: two gloo ranks (127.0.0.1)
take the max of their step times and report the whole-job rate from it, as
the NCCL run on N GPUs does."""
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


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                      # rank 1 is the slower replica
        mx = bench.max_over_ranks(ms, dist)
        dist.barrier()
        q.put((rank, mx, bench.whole_job_rate(1000.0, world, mx / 1e3)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_report_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, mx, rate in got:
        assert mx == 15.0                              # max over ranks, on every rank
        assert abs(rate - 2 * 1000.0 / 0.015) < 1e-6  # all ranks' units / slowest time


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
