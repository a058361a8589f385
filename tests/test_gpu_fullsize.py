"""GPU checks at the full sizes of the measured workloads, in the launch configuration the
bench times: the 3D cantilever on 96x48x48 (1,327,104 tetrahedra, 698,691 DOFs) and the
64-instance screened Helmholtz batch on 512x512.  The oracle cannot solve these sizes in
seconds, so the checks are what holds at any size -- the element coefficients against the
oracle's rule, the true FP64 residual of the solutions through the library's own operator,
the explicit adjoint against its closed form -- plus a sample of the batch's loads."""
import numpy as np
import pytest

from oracle import shape as oshape
from paper_2601_05709_gb300 import api, workloads
from tests.helpers import batch_case, cantilever3d, gpu_batch, gpu_problem, oracle_batch, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _phi_c3(coords):
    # 20 Gaussian bumps of width 0.1 minus 0.2, centres uniform in the box (seed 0)
    return workloads.phi_bumps(coords, workloads.bump_centres((0, 0, 0), (2, 1, 1), 20, seed=0), 0.1, 0.2)


@pytest.mark.parametrize("precision", [api.FO_MIXED, api.FO_FP64])
def test_cantilever3d_fullsize_state(ctx, precision):
    c = cantilever3d((96, 48, 48))
    mesh, prob = gpu_problem(ctx, c)
    cells, coords = mesh.copy_out()
    phi = _phi_c3(coords)
    prob.set_levelset(phi)
    prob.coefficients()
    A_ref, chi_ref = oshape.coefficient(phi, cells, c["a_in"], c["a_out"])
    assert np.array_equal(prob.get(api.FO_FIELD_COEF), A_ref)
    assert np.array_equal(prob.get(api.FO_FIELD_CHI), chi_ref)
    st = prob.state_solve(api.solve_opts(precision=precision, rtol=1e-8, precond=api.FO_PC_MG))
    assert 0 < st.iterations < 400, st.iterations
    u = prob.get(api.FO_FIELD_U)
    F = prob.get(api.FO_FIELD_LOAD)
    r = F - prob.apply(api.FO_OP_STATE, u)        # Dirichlet rows are identity with zero load
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(F), np.linalg.norm(r) / np.linalg.norm(F)
    prob.close()


def test_cantilever3d_fullsize_opt_step(ctx):
    """One Algorithm-1 iteration at full size through the multigrid path: the cost is the
    compliance F . u of the state it solved, the step moved phi, everything finite."""
    c = cantilever3d((96, 48, 48))
    mesh, prob = gpu_problem(ctx, c)
    _, coords = mesh.copy_out()
    phi0 = _phi_c3(coords)
    prob.set_levelset(phi0)
    ro = api.run_options(state=api.solve_opts(rtol=1e-11, precond=api.FO_PC_MG),
                         velocity=api.solve_opts(rtol=1e-10, precond=api.FO_PC_MG))
    log = prob.opt_step(0, ro)
    assert 0 < log.state.iterations < 400 and 0 < log.velocity.iterations < 400
    u = prob.get(api.FO_FIELD_U)
    F = prob.get(api.FO_FIELD_LOAD)
    assert abs(log.J - float(F @ u)) <= 1e-8 * abs(log.J)
    assert np.isfinite(log.Btt) and log.Btt > 0 and log.nsteps >= 1
    phi1 = prob.get(api.FO_FIELD_PHI)
    assert np.all(np.isfinite(phi1)) and rel(phi1, phi0) > 0
    prob.close()


def test_batch_fullsize(ctx):
    """The 64-instance batch on 512x512 as the bench runs it (FP64 refinement around the FP32
    multigrid CG): every instance's true residual, the explicit adjoint, and the loads of a
    sample of instances against the oracle."""
    c = batch_case(dim=2, n=(512, 512), n_inst=64, seed=1)
    mesh, prob = gpu_batch(ctx, c)
    _, coords = mesh.copy_out()
    prob.set_levelset(workloads.phi_cos(coords))
    prob.coefficients()
    opts = api.solve_opts(precision=api.FO_MIXED, rtol=1e-8, inner_rtol=1e-3, maxit=2000, inner_maxit=1000,
                          precond=api.FO_PC_MG)
    st = prob.state_solve(opts)
    assert st.iterations < 300 and st.outer_iterations <= 6, (st.iterations, st.outer_iterations)
    U = prob.get(api.FO_FIELD_U)
    F = prob.get(api.FO_FIELD_LOAD)
    R = F - prob.apply(api.FO_OP_STATE, U)
    for i in range(64):
        assert np.linalg.norm(R[:, i]) <= 1.5e-8 * np.linalg.norm(F[:, i]), i
    prob.adjoint_solve(opts)
    assert rel(prob.get(api.FO_FIELD_P), -U) <= 1e-6
    # loads of three instances from the oracle (its per-instance definition)
    sub = [0, 29, 63]
    cs = dict(c, n_inst=len(sub), k=c["k"][sub], omega=c["omega"][sub], amp=c["amp"][sub])
    Fref = oracle_batch(cs).loads()
    scale = np.max(np.abs(Fref))
    assert np.max(np.abs(F[:, sub] - Fref)) <= 1e-13 * scale
    prob.close()
