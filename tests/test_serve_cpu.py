"""Host logic of the request server, without a GPU: executors in dry-run mode sleep instead
of touching the device, so the queue, FIFO admission, the memory budget, back-pressure and
the bounded waits can be checked on the CPU."""
import time

import numpy as np
import pytest

from paper_2601_05709_gb300 import api, _lib


def _req(n, kind=api.FO_HEAT, dim=2):
    desc = api.model_desc(kind, dirichlet=[(0, 0)], f_nodal=None)
    centers = np.full((1, dim), 0.5)
    return api.ServedRequest(dim, (n,) * dim, desc, centers=centers)


def test_footprint_grows_with_size_and_precision():
    b16 = _req(16).device_bytes()
    b32 = _req(32).device_bytes()
    assert 0 < b16 < b32
    e32 = _req(32, api.FO_ELASTIC).device_bytes()
    r = _req(32, api.FO_ELASTIC)
    r.struct.state.precision = _lib.FO_MIXED
    assert r.device_bytes() > e32            # the refinement keeps 11 state vectors instead of 8
    assert _req(8, api.FO_ELASTIC, 3).device_bytes() > _req(8, api.FO_HEAT, 3).device_bytes()


def test_fifo_admission_and_budget():
    small, big = _req(16), _req(64)
    bs, bb = small.device_bytes(), big.device_bytes()
    budget = bb + bs                          # a big one and one small one fit together, not two big
    srv = api.Server(None, executors=4, mem_budget=budget, dry_run_ms=20.0)
    order = [big, small, big, small, small, big]
    tickets = [srv.submit(r)[1] for r in order]
    res = [srv.wait(t, 30.0) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(r is not None and r.status == 0 for r in res)
    starts = [r.start_ms for r in res]
    assert starts == sorted(starts)            # admitted in submission order
    assert st.peak_bytes <= budget
    assert st.completed == len(order) and st.failed == 0
    # the second big request cannot start before the first has finished
    assert res[2].start_ms >= res[0].end_ms - 1e-6


def test_concurrency_and_rejections():
    r = _req(16)
    srv = api.Server(None, executors=3, mem_budget=100 * r.device_bytes(), queue_capacity=2, dry_run_ms=200.0)
    ok = []
    for _ in range(3):                        # each executor takes one as it arrives
        time.sleep(0.05)
        st, t = srv.submit(r)
        assert st == 0
        ok.append(t)
    time.sleep(0.05)
    st = None
    for _ in range(20):                       # 2 more fit in the queue, then back-pressure
        st, t = srv.submit(r)
        if st != 0:
            break
        ok.append(t)
    assert st == _lib.FO_EBUSY and len(ok) == 5, (st, len(ok))
    assert srv.wait(ok[-1], 0.01) is None      # bounded wait: not done yet
    res = [srv.wait(t, 30.0) for t in ok]
    assert all(x is not None for x in res)
    assert srv.stats().peak_in_flight == 3
    too_big = api.Server(None, executors=1, mem_budget=r.device_bytes() - 1, dry_run_ms=1.0)
    assert too_big.submit(r)[0] == _lib.FO_ENOMEM_BUDGET
    too_big.close()
    done, got = srv.poll(ok[0])
    assert done and got.status == 0
    srv.release(ok[0])
    with pytest.raises(_lib.FormoptError):
        srv.poll(ok[0])
    srv.close()


def test_destroy_cancels_queued():
    """Destroy waits for the running request only; the queued ones are cancelled."""
    r = _req(16)
    srv = api.Server(None, executors=1, mem_budget=10 * r.device_bytes(), dry_run_ms=300.0)
    for _ in range(4):
        assert srv.submit(r)[0] == 0
    time.sleep(0.05)
    t0 = time.time()
    srv.close()
    dt = time.time() - t0
    assert dt < 0.6, dt                      # one running request (<= 300 ms), not four


def test_footprint_counts_multigrid_only_where_it_applies():
    def req(n, pc):
        r = _req(n, api.FO_ELASTIC)
        r.struct.state.precond = pc
        r.struct.velocity.precond = pc
        return r.device_bytes()
    assert req(64, api.FO_PC_MG) > req(64, api.FO_PC_JACOBI)    # 64 halves down to a small coarsest grid
    assert req(63, api.FO_PC_MG) > req(63, api.FO_PC_JACOBI)    # odd: non-nested ceil(n/2) levels
    assert req(2, api.FO_PC_MG) == req(2, api.FO_PC_JACOBI)     # too small to coarsen: Jacobi fallback


def test_smallest_first_admission():
    """FO_SERVE_SMALLEST_FIRST: with one executor busy, the queued requests start smallest
    footprint first (ties in submission order); FIFO keeps submission order."""
    sizes = [64, 16, 48, 16, 32]
    reqs = [_req(n) for n in sizes]
    for smallest, expect in ((True, [0, 1, 3, 4, 2]), (False, [0, 1, 2, 3, 4])):
        srv = api.Server(None, executors=1, mem_budget=1 << 40, dry_run_ms=60.0, smallest_first=smallest)
        tickets = [srv.submit(reqs[0])[1]]
        time.sleep(0.015)                            # the first has started; the rest queue behind it
        tickets += [srv.submit(r)[1] for r in reqs[1:]]
        res = [srv.wait(t, 30.0) for t in tickets]
        srv.close()
        order = sorted(range(len(res)), key=lambda i: res[i].start_ms)
        assert order == expect, (smallest, order)
