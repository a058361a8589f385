"""Instance sharding of the task-parallel batch (paper_2601_05709_gb300.shard) on the CPU with
gloo ranks: the partition covers every instance once, and the rank-ordered sum of the ranks'
cost and shape-derivative right-hand side (each rank's part computed here by the oracle for
its own instances, the volume term on rank 0 only) is the same bits on every rank, equals the
explicit rank-order sum bitwise, and equals the oracle's whole-batch J and b to rounding."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_05709_gb300 import shard


def test_partition_covers_instances_in_order():
    for n, world in ((64, 1), (64, 2), (64, 3), (10, 4), (5, 5)):
        ranges = [shard.partition(n, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0
        sizes = [b - a for a, b in ranges]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        shard.partition(3, 4, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from oracle.batch import Batch
    from oracle.mesh import BoxMesh
    from paper_2601_05709_gb300 import workloads
    m = BoxMesh(2, (12, 10), (0.0, 0.0), (1.0, 1.0))
    k, om, amp = workloads.batch_parameters(7, 3)
    f = workloads.fourier_loads(m.coords, amp)
    phi = workloads.phi_cos(m.coords)
    return m, k, om, f, phi


def _part(rank, world, lam):
    """This rank's (J, b) from the oracle, for its own instances."""
    from oracle.batch import Batch
    m, k, om, f, phi = _problem()
    i0, i1 = shard.partition(len(k), world, rank)
    b = Batch(m, k[i0:i1], om[i0:i1], f[i0:i1], dirichlet_faces=[(0, 0)], volume_target=0.4)
    U, A, chi = b.state(phi)
    return b.cost(U, A), b.rhs(U, A, chi, lam if rank == 0 else 0.0)


def _rank_main(rank, world, port, lam, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    J_r, b_r = _part(rank, world, lam)
    J = shard.ordered_sum(np.array([J_r]), dist)[0]
    b = shard.ordered_sum(b_r, dist)
    out.put((rank, float(J), b))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sum_matches_whole_batch(world):
    import torch.multiprocessing as mp
    from oracle.batch import Batch
    lam = 0.37
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, lam, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank holds the same bits
    for _, J, b in res[1:]:
        assert J == res[0][1] and np.array_equal(b, res[0][2])
    # the explicit rank-order sum of the parts, bitwise
    parts = [_part(r, world, lam) for r in range(world)]
    Jx, bx = parts[0][0], parts[0][1].copy()
    for J_r, b_r in parts[1:]:
        Jx = Jx + J_r
        bx += b_r
    assert res[0][1] == Jx and np.array_equal(res[0][2], bx)
    # the whole batch in one process, to rounding (different summation grouping)
    m, k, om, f, phi = _problem()
    whole = Batch(m, k, om, f, dirichlet_faces=[(0, 0)], volume_target=0.4)
    U, A, chi = whole.state(phi)
    assert abs(res[0][1] - whole.cost(U, A)) <= 1e-13 * abs(whole.cost(U, A))
    bw = whole.rhs(U, A, chi, lam)
    assert np.max(np.abs(res[0][2] - bw)) <= 1e-13 * np.max(np.abs(bw))
