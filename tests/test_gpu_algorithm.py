"""Whole Algorithm-1 iterations on the GPU (fo_opt_step) against the oracle, plus the error
paths of the ABI (non-convergence, NaN input, memory budget, call order)."""
import numpy as np
import pytest

from oracle import algorithm as oalg, levelset, ppl as oppl
from paper_2601_05709_gb300 import workloads
from tests.helpers import HEAT2D, cantilever2d, cantilever3d, case, close_scaled, gpu_problem, oracle_problem, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_05709_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context(0)
    yield c
    c.close()


def tight_run(api, **kw):
    so = api.solve_opts(rtol=1e-13, maxit=400000)
    return api.run_options(state=so, velocity=so, transport=so, **kw)


def test_heat2d_iteration(ctx, api):
    """The 64 x 64 heat-compliance workload: one full iteration."""
    c = case(**HEAT2D)
    mesh, prob = gpu_problem(ctx, c)
    op = oracle_problem(c)
    phi0 = workloads.phi_cos(op.mesh.coords)
    prob.set_levelset(phi0)
    log = prob.opt_step(0, tight_run(api, dfactor=1e-2))
    phi1 = prob.get(api._lib.FO_FIELD_PHI)
    ophi1, olog = oalg.opt_step(op, phi0, 0, oppl.PPL(0), oalg.RunOptions(dfactor=1e-2))
    assert abs(log.J - olog["J"]) <= 1e-10 * abs(olog["J"])
    assert abs(log.Btt - olog["Btt"]) <= 1e-9 * abs(olog["Btt"])
    assert log.nsteps == olog["nsteps"] and log.t_end == pytest.approx(olog["t_end"], rel=1e-9)
    assert close_scaled(prob.get(api._lib.FO_FIELD_THETA), olog["theta"], 1e-10)
    assert close_scaled(phi1, ophi1, 1e-10), np.max(np.abs(phi1 - ophi1))


@pytest.mark.parametrize("c,iters", [(cantilever2d((64, 32)), 5), (cantilever3d((12, 6, 6)), 2)])
def test_cantilever_iterations_with_ppl_and_reinit(ctx, api, c, iters):
    mesh, prob = gpu_problem(ctx, c)
    op = oracle_problem(c)
    cen, rad = workloads.hole_lattice() if c["dim"] == 2 else (np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5]]), np.array([0.2, 0.2]))
    phi = levelset.initial_level(op.mesh.coords, cen, rad)
    prob.set_levelset(phi)
    run = tight_run(api, dfactor=1e-1, smooth=True, reinit_step=2, reinit_pars=(6, 0.05))
    ppl = api.PPL(1)
    oppl_state = oppl.PPL(1)
    oopts = oalg.RunOptions(dfactor=1e-1, smooth=True, reinit_step=2, reinit_pars=(6, 0.05))
    for i in range(iters):
        log = prob.opt_step(i, run, ppl)
        phi, olog = oalg.opt_step(op, phi, i, oppl_state, oopts)
        assert abs(log.J - olog["J"]) <= 1e-9 * abs(olog["J"]), (i, log.J, olog["J"])
        assert abs(log.C - olog["C"]) <= 1e-12
        assert abs(log.lam - olog["lam"]) <= 1e-9 * max(1.0, abs(olog["lam"]))
        assert log.nsteps == olog["nsteps"] and bool(log.reinit) == olog["reinit"]
        # element decisions must agree for the iterates to stay comparable
        gphi = prob.get(api._lib.FO_FIELD_PHI)
        assert close_scaled(gphi, phi, 1e-8), (i, np.max(np.abs(gphi - phi)))


def test_mixed_precision_iteration(ctx, api):
    c = cantilever2d((128, 64))
    mesh, prob = gpu_problem(ctx, c)
    op = oracle_problem(c)
    cen, rad = workloads.hole_lattice()
    phi = levelset.initial_level(op.mesh.coords, cen, rad)
    prob.set_levelset(phi)
    so = api.solve_opts(precision=api.FO_MIXED, rtol=1e-12)
    run = api.run_options(dfactor=1e-1, smooth=True, state=so)
    log = prob.opt_step(0, run, api.PPL(1))
    _, olog = oalg.opt_step(op, phi, 0, oppl.PPL(1), oalg.RunOptions(dfactor=1e-1, smooth=True))
    assert abs(log.J - olog["J"]) <= 1e-8 * abs(olog["J"])
    assert close_scaled(prob.get(api._lib.FO_FIELD_U), olog["u"], 1e-8)


# ------------------------------------------------------------------------- error paths
def test_noconv_reports_and_keeps_result(ctx, api):
    mesh, prob = gpu_problem(ctx, case(**HEAT2D))
    _, coords = mesh.copy_out()
    prob.set_levelset(workloads.phi_cos(coords))
    st = prob.state_solve(api.solve_opts(maxit=3), allow_noconv=True)
    assert st.iterations == 3 and st.rel_residual > 1e-6
    with pytest.raises(api.FormoptError) as e:
        prob.state_solve(api.solve_opts(maxit=3))
    assert e.value.status == api._lib.FO_ENOCONV


def test_nan_input_detected(ctx, api):
    mesh, prob = gpu_problem(ctx, case(dim=2, n=(8, 8), kind=0, f=lambda X: np.ones(X.shape[0])))
    f = np.ones(mesh.num_nodes)
    phi = -np.ones(mesh.num_nodes)
    prob.set_levelset(phi)
    prob.state_solve()
    u = prob.get(api._lib.FO_FIELD_U)
    u[10] = np.nan
    prob.set(api._lib.FO_FIELD_U, u)
    with pytest.raises(api.FormoptError) as e:
        prob.functionals()
    assert e.value.status == api._lib.FO_ENAN


def test_memory_budget_refuses(api):
    small = api.Context(0, mem_budget=1 << 16)
    with pytest.raises(api.FormoptError) as e:
        small.mesh_box(2, (256, 256), (0, 0), (1, 1))
    assert e.value.status == api._lib.FO_ENOMEM_BUDGET
    small.close()


def test_call_order_checked(ctx, api):
    mesh, prob = gpu_problem(ctx, case(dim=2, n=(4, 4), kind=0))
    with pytest.raises(api.FormoptError) as e:
        prob.descent()
    assert e.value.status == api._lib.FO_ESTATE


def test_deterministic(ctx, api):
    outs = []
    for _ in range(2):
        c = cantilever2d((64, 32))
        mesh, prob = gpu_problem(ctx, c)
        _, coords = mesh.copy_out()
        cen, rad = workloads.hole_lattice()
        prob.initial_level(cen, rad)
        log = prob.opt_step(0, api.run_options(dfactor=0.1, smooth=True), api.PPL(1))
        outs.append((log.J, log.Btt, prob.get(api._lib.FO_FIELD_PHI)))
        prob.close()
    assert outs[0][0] == outs[1][0] and outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][2], outs[1][2])
