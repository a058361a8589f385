"""The bench's multi-rank host logic on the CPU (gloo, world size 2): the whole-job rate is
bounded by the slowest rank, every rank agrees on it, and the reference arm runs on rank 0
only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rate, t = bench.job_rate(1.0 + rank, 10, world, dist, device="cpu")
    out.put((rank, rate, t))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_is_bounded_by_the_slowest_rank():
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
    assert [r for r, _, _ in res] == [0, 1]
    for _, rate, t in res:
        assert t == 2.0                       # max over ranks
        assert rate == 2 * 10 / 2.0           # all ranks' units over the slowest time


def test_job_rate_single_rank():
    import bench
    assert bench.job_rate(0.5, 10, 1) == (20.0, 0.5)


def test_reference_arm_only_on_rank_zero(capsys):
    import bench

    class A:
        steps, gpus = 1, 2
    assert bench.run_reference(A(), 1, 2) is None
    assert capsys.readouterr().out == ""
