"""fo_state_solve_noalloc: the state solve for callers that cannot let the library allocate.

Such callers (a loop that cannot afford the device-wide synchronisation cudaMalloc/cudaFree
may cause, a process whose device memory belongs to another framework's allocator or to a
fixed budget) pass their own input and output buffers; the solver's
working memory is a fixed array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test.

The check: through the C ABI, two calls in a row give the result of the ordinary entry
point fo_state_solve on the same problem under the solve criterion of the parity tests (the
two solvers sum in different orders, and the 128 x 64 cantilever's Skeel condition is ~1e9:
1e-10 where the conditioning allows it, else a componentwise backward error at the rounding
level and a forward difference within the perturbation bound), the context's device-memory
count does not move, and a problem larger than the array is refused with FO_EINVAL.
"""
import ctypes as C

import numpy as np
import pytest

from tests.helpers import HEAT2D, assert_solve_parity, cantilever2d, case, gpu_problem, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_05709_gb300 import api as a
    return a


def _noalloc(api, prob, b, x, opts):
    st = api._lib.SolveStats()
    s = prob.lib.fo_state_solve_noalloc(prob.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                        C.byref(opts), C.byref(st))
    return s, st


@pytest.mark.parametrize("c", [case(**HEAT2D), cantilever2d((128, 64))])
def test_noalloc_matches_state_solve(api, c):
    import torch
    from paper_2601_05709_gb300 import workloads
    ctx = api.Context(0)
    try:
        mesh, prob = gpu_problem(ctx, c)
        _, coords = mesh.copy_out()
        prob.set_levelset(workloads.phi_cos(coords))
        opts = api.solve_opts(rtol=1e-12)
        prob.state_solve(opts)                                  # the ordinary entry point
        u_ref = prob.get(api._lib.FO_FIELD_U)
        op = oracle_problem(c)
        _, A, _ = op.state(workloads.phi_cos(op.mesh.coords))
        K, F, free = op.stiffness(A), op.load(), op.dirichlet() == 0
        b = torch.from_numpy(prob.get(api._lib.FO_FIELD_LOAD)).cuda()
        torch.cuda.synchronize()
        before = ctx.memory()
        for call in range(2):                                   # the second call finds the array used
            x = torch.full_like(b, float("nan") if call else 7.0)   # stale output must not matter
            s, st = _noalloc(api, prob, b, x, opts)
            assert s == 0, api._lib.STATUS_NAMES.get(s, s)
            u = x.cpu().numpy()
            assert_solve_parity(K, F, free, u, u_ref, 1e-10, omega_max=1e-12)
            assert st.iterations > 0 and st.rel_residual <= 1e-12
        assert ctx.memory() == before                           # nothing allocated by the calls
    finally:
        ctx.close()


def test_noalloc_refuses_oversized_problem(api):
    import torch
    ctx = api.Context(0)
    try:
        # 3D heat on 64^3 cells: 274,625 DOFs > FO_NOALLOC_MAX_DOFS = 258,048
        mesh, prob = gpu_problem(ctx, case(dim=3, n=(64, 64, 64), kind=0, f=lambda X: np.ones(X.shape[0])))
        b = torch.zeros(mesh.num_nodes, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        s, _ = _noalloc(api, prob, b, x, api.solve_opts())
        assert s == api._lib.FO_EINVAL
        assert b"no-allocation limit" in prob.lib.fo_last_error(ctx.handle)
    finally:
        ctx.close()
