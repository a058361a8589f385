"""The logistic population model (Sec. 6.4) on the GPU against the oracle: Newton state,
adjoint, cost and constraint, shape-derivative right-hand side and one Algorithm-1 iteration."""
import numpy as np
import pytest

from oracle import algorithm as oalg, levelset, logistic, ppl as oppl, velocity as ovel
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads
from tests.helpers import close_scaled

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


def _phi(m, dim):
    if dim == 2:
        return workloads.phi_cos(m.coords)
    return workloads.phi_bumps(m.coords, workloads.bump_centres((0,) * dim, (1,) * dim, 6, seed=4), 0.25, 0.3)


def _setup(ctx, api, dim, n, r, volume=0.5):
    m = BoxMesh(dim, n, (0.0,) * dim, (1.0,) * dim)
    mesh = ctx.mesh_box(dim, n, (0.0,) * dim, (1.0,) * dim)
    u0 = workloads.u0_logistic(m.coords)
    desc = api.model_desc(api.FO_LOGISTIC, a_in=1.0, a_out=1e-2, dirichlet=[], volume=volume, alpha_mass=0.0,
                          normal_penalty=1e4, growth_rate=r, u_init=u0)
    prob = mesh.problem(desc)
    phi = _phi(m, dim)
    prob.set_levelset(phi)
    op = oalg.Problem(mesh=m, kind=oalg.LOGISTIC, a_in=1.0, a_out=1e-2, volume_target=volume, growth_rate=r,
                      u_init=u0, vform=ovel.VelocityForm(alpha_mass=0.0, normal_penalty=1e4))
    return m, mesh, prob, op, phi


def _opts(api, **kw):
    return api.solve_opts(rtol=1e-13, maxit=400000, precond=api.FO_PC_JACOBI, **kw)


@pytest.mark.parametrize("dim,n,r", [(2, (40, 32), 10.0), (2, (33, 47), 100.0), (3, (9, 8, 7), 40.0)])
def test_newton_state_adjoint_functionals(ctx, api, dim, n, r):
    m, mesh, prob, op, phi = _setup(ctx, api, dim, n, r)
    st = prob.state_solve(_opts(api))
    u = prob.get(api.FO_FIELD_U)
    u_ref, K, chi = op.state(phi)
    assert close_scaled(u, u_ref, 1e-10), np.max(np.abs(u - u_ref))
    assert 2 <= st.outer_iterations <= 30, st.outer_iterations
    prob.adjoint_solve(_opts(api))
    p = prob.get(api.FO_FIELD_P)
    p_ref = logistic.adjoint(m.coords, m.cells, K, r, u_ref)
    assert close_scaled(p, p_ref, 1e-10), np.max(np.abs(p - p_ref)) / np.max(np.abs(p_ref))
    J, C = prob.functionals()
    assert abs(J - logistic.cost(m.coords, m.cells, u_ref)) <= 1e-12 * abs(J)
    assert abs(C - op.constraint(chi)) <= 1e-13 * abs(C)


def test_constant_equilibrium(ctx, api):
    """All inside: u = K = 1 exactly is the root Newton reaches from the paper's guess."""
    m = BoxMesh(2, (24, 24), (0, 0), (1, 1))
    mesh = ctx.mesh_box(2, (24, 24), (0, 0), (1, 1))
    prob = mesh.problem(api.model_desc(api.FO_LOGISTIC, a_in=1.0, a_out=1e-2, dirichlet=[], growth_rate=40.0,
                                       u_init=workloads.u0_logistic(m.coords)))
    prob.set_levelset(-np.ones(m.num_nodes))
    prob.state_solve(_opts(api))
    assert np.max(np.abs(prob.get(api.FO_FIELD_U) - 1.0)) < 1e-13


@pytest.mark.parametrize("dim,n", [(2, (24, 20)), (3, (7, 6, 5))])
def test_shape_rhs_elementwise(ctx, api, dim, n):
    """b from the oracle's own u and p (set on the device), element by element, with lambda."""
    r, lam = 25.0, 0.37
    m, mesh, prob, op, phi = _setup(ctx, api, dim, n, r)
    u_ref, K, chi = op.state(phi)
    p_ref = logistic.adjoint(m.coords, m.cells, K, r, u_ref)
    prob.coefficients()
    prob.set(api.FO_FIELD_U, u_ref)
    prob.set(api.FO_FIELD_P, p_ref)
    b = prob.shape_derivative(lam)
    b_ref = logistic.rhs(m.coords, m.cells, K, r, u_ref, p_ref, lam, chi.astype(np.float64), 0.5)
    assert close_scaled(b, b_ref, 1e-12), np.max(np.abs(b - b_ref)) / np.max(np.abs(b_ref))


def test_mixed_newton_steps(ctx, api):
    """FP32 inner CG with FP64 refinement in each Newton step: the same root to 1e-10."""
    m, mesh, prob, op, phi = _setup(ctx, api, 2, (48, 40), 40.0)
    prob.state_solve(api.solve_opts(precision=api.FO_MIXED, rtol=1e-13, inner_rtol=1e-4, precond=api.FO_PC_JACOBI))
    u_ref, _, _ = op.state(phi)
    assert close_scaled(prob.get(api.FO_FIELD_U), u_ref, 1e-10)


def test_algorithm_iteration(ctx, api):
    """One Algorithm-1 iteration of the population example (V = 0.5, B = Dtheta:Dxi + 1e4 normal
    penalty on H^1): J, C, lambda, B(theta, theta), theta and the transported phi."""
    r = 40.0
    m, mesh, prob, op, phi = _setup(ctx, api, 2, (32, 32), r)
    so = _opts(api)
    ro = api.run_options(dfactor=1e-2, lv_time=(1e-3, 1e-1), lv_iter=(8, 16), smooth=False, state=so, velocity=so,
                         transport=so)
    ppl = api.PPL(1)
    log = prob.opt_step(0, ro, ppl)
    ophi, olog = oalg.opt_step(op, phi, 0, oppl.PPL(1), oalg.RunOptions(dfactor=1e-2))
    assert abs(log.J - olog["J"]) <= 1e-11 * abs(olog["J"])
    assert abs(log.C - olog["C"]) <= 1e-13 * abs(olog["C"])
    assert abs(log.lam - olog["lam"]) <= 1e-10 * max(1.0, abs(olog["lam"]))
    assert abs(log.Btt - olog["Btt"]) <= 1e-10 * abs(olog["Btt"])
    assert log.nsteps == olog["nsteps"]
    assert close_scaled(prob.get(api.FO_FIELD_THETA), olog["theta"], 1e-10)
    assert close_scaled(prob.get(api.FO_FIELD_PHI), ophi, 1e-10)
    assert log.newton_steps >= 2 and log.adjoint.iterations > 0
