"""The multi-GPU form of the bench is replicas: each rank searches its own batch
on its own copy of the index, and the only exchange is the timing (barrier and
max over ranks).  That host logic runs here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(5.0 + 2.5 * rank, "cpu")  # rank 1 is the slowest
        qps = bench.job_throughput(10_000, world, ms)
        out[rank] = (ms, qps)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert res[0] == res[1] == (7.5, 2 * 10_000 / 7.5e-3)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.0, "cpu") == 3.0
    assert bench.job_throughput(10_000, 1, 5.0) == pytest.approx(2_000_000.0)
