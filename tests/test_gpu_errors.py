"""Bounded waits on the GPU, without a fault: a grid barrier that one block never reaches must
release the others at its time limit with FO_ETIMEOUT, and the context must stay usable."""
import time

import numpy as np
import pytest

from paper_2601_05709_gb300 import api, _lib
from tests.helpers import HEAT2D, case, gpu_problem

pytestmark = pytest.mark.gpu


def test_barrier_releases_when_all_arrive():
    ctx = api.Context(0)
    st, gave_up = ctx.selftest_barrier(16, -1, 1000.0)
    assert st == _lib.FO_OK and gave_up == 0
    ctx.close()


def test_barrier_gives_up_at_its_limit_and_context_survives():
    ctx = api.Context(0)
    t0 = time.perf_counter()
    st, gave_up = ctx.selftest_barrier(16, 5, 50.0)
    dt = time.perf_counter() - t0
    assert st == _lib.FO_ETIMEOUT and gave_up == 15
    assert 0.05 <= dt < 5.0, dt
    # the same context still runs a solve
    mesh, prob = gpu_problem(ctx, case(**HEAT2D))
    _, coords = mesh.copy_out()
    prob.set_levelset(np.cos(4 * np.pi * coords[:, 0]) * np.cos(4 * np.pi * coords[:, 1]) + 0.3)
    s = prob.state_solve(api.solve_opts(rtol=1e-10))
    assert s.iterations > 0
    ctx.close()
