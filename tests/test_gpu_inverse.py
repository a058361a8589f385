"""Inverse elasticity (Sec. 3, Sec. 6.1) on the GPU against the oracle: both states, the cost,
both adjoints, the shape-derivative right-hand side element by element, two force-displacement
pairs, and one Algorithm-1 iteration; the zero of the cost at the true inclusion."""
import numpy as np
import pytest

from oracle import fem, inverse, levelset, ppl as oppl, shape, velocity as ovel
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads
from tests.helpers import close_scaled

pytestmark = pytest.mark.gpu

LAM, MU = fem.lame(1.0, 0.3)
ALPHA, BETA = 3.0, 2.0


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


def _faces(dim):
    return [(0, 0)], [(a, s) for a in range(dim) for s in (0, 1) if (a, s) != (0, 0)]


def _tractions(dim, npairs):
    ts = [np.array([0.3, -1.0, 0.2][:dim]), np.array([-0.5, 0.2, 0.7][:dim])]
    faces = [(0, 1), (1, 1)]
    return [(faces[k][0], faces[k][1], ts[k]) for k in range(npairs)]


def _phi(m, seed):
    return workloads.phi_bumps(m.coords, workloads.bump_centres((0.2,) * m.dim, (0.8,) * m.dim, 3, seed), 0.15, 0.5)


def _oracle(m, phi, meas, npairs):
    dim = m.dim
    f0, f1 = _faces(dim)
    dir0 = m.dirichlet_mask(f0, dim)
    A, chi = shape.coefficient(phi, m.cells, 10.0, 1.0)
    K = inverse.elastic_matrix(m.coords, m.cells, A, LAM, MU)
    M = inverse.vector_mass(m.coords, m.cells)
    Mg = inverse.facet_vector_mass(m.coords, inverse.gamma_facets(m, f1))
    out = []
    for k, (ax, sd, t) in enumerate(_tractions(dim, npairs)):
        F = fem.facet_load(m.coords, m.boundary_facets(ax, sd), t, dim)
        F[dir0 == 1] = 0.0
        g = meas[k]
        u, v = inverse.states(m, K, F, g, dir0)
        p, q = inverse.adjoints(m, K, M, Mg, u, v, g, ALPHA, BETA, dir0)
        out.append(dict(F=F, g=g, u=u, v=v, p=p, q=q, J=inverse.cost(M, Mg, u, v, g, ALPHA, BETA)))
    return A, chi, out


def _gpu(ctx, api, m, phi, meas, npairs, vel=None):
    dim = m.dim
    f0, f1 = _faces(dim)
    mesh = ctx.mesh_box(dim, m.n, m.lo, m.hi)
    cases = [([], [(ax, sd, tuple(t))]) for (ax, sd, t) in _tractions(dim, npairs)]
    vkw = vel or dict(alpha_mass=0.1, velocity_dirichlet=True)
    desc = api.model_desc(api.FO_ELASTIC, a_in=10.0, a_out=1.0, E=1.0, nu=0.3, dirichlet=f0, load_cases=cases,
                          inverse=True, gamma1=f1, meas=np.stack(meas), kv_alpha=ALPHA, kv_beta=BETA, **vkw)
    prob = mesh.problem(desc)
    prob.set_levelset(phi)
    return mesh, prob


def _opts(api, **kw):
    return api.solve_opts(rtol=1e-13, maxit=400000, precond=api.FO_PC_JACOBI, **kw)


def _meas(m, npairs, seed=6):
    return [0.5 * workloads.smooth_field(m.coords, m.dim, seed + k) for k in range(npairs)]


@pytest.mark.parametrize("dim,n,npairs,pc", [(2, (24, 20), 1, 0), (2, (17, 23), 2, 0), (3, (6, 5, 5), 1, 0),
                                           (2, (32, 24), 2, 1), (3, (8, 8, 4), 1, 1)])
def test_states_cost_adjoints(ctx, api, dim, n, npairs, pc):
    """Jacobi (pc 0) or multigrid (pc 1; the boundary-clamped systems on a hierarchy of their own)."""
    m = BoxMesh(dim, n, (0.0,) * dim, (1.0,) * dim)
    phi = _phi(m, 1)
    meas = _meas(m, npairs)
    A, chi, ref = _oracle(m, phi, meas, npairs)
    mesh, prob = _gpu(ctx, api, m, phi, meas, npairs)
    so = api.solve_opts(rtol=1e-13, maxit=400000, precond=pc)
    st = prob.state_solve(so)
    if pc == 1:
        assert st.iterations < 600, st.iterations
    U = prob.get(api.FO_FIELD_U).reshape(npairs, -1)
    V = prob.get(api._lib.FO_FIELD_V).reshape(npairs, -1)
    for k in range(npairs):
        assert close_scaled(U[k], ref[k]["u"], 1e-10), (k, np.max(np.abs(U[k] - ref[k]["u"])))
        assert close_scaled(V[k], ref[k]["v"], 1e-10), (k, np.max(np.abs(V[k] - ref[k]["v"])))
    J, _ = prob.functionals()
    J_ref = sum(r["J"] for r in ref)
    assert abs(J - J_ref) <= 1e-10 * abs(J_ref), (J, J_ref)
    prob.adjoint_solve(so)
    P = prob.get(api.FO_FIELD_P).reshape(npairs, -1)
    Q = prob.get(api._lib.FO_FIELD_Q).reshape(npairs, -1)
    for k in range(npairs):
        assert close_scaled(P[k], ref[k]["p"], 1e-10), (k, np.max(np.abs(P[k] - ref[k]["p"])))
        assert close_scaled(Q[k], ref[k]["q"], 1e-10), (k, np.max(np.abs(Q[k] - ref[k]["q"])))


@pytest.mark.parametrize("dim,n,npairs", [(2, (20, 16), 2), (3, (5, 4, 4), 1)])
def test_shape_rhs_elementwise(ctx, api, dim, n, npairs):
    """b from the oracle's own states and adjoints (set on the device), element by element."""
    m = BoxMesh(dim, n, (0.0,) * dim, (1.0,) * dim)
    phi = _phi(m, 2)
    meas = _meas(m, npairs, 3)
    A, chi, ref = _oracle(m, phi, meas, npairs)
    mesh, prob = _gpu(ctx, api, m, phi, meas, npairs)
    prob.coefficients()
    prob.set(api.FO_FIELD_U, np.concatenate([r["u"] for r in ref]))
    prob.set(api._lib.FO_FIELD_V, np.concatenate([r["v"] for r in ref]))
    prob.set(api.FO_FIELD_P, np.concatenate([r["p"] for r in ref]))
    prob.set(api._lib.FO_FIELD_Q, np.concatenate([r["q"] for r in ref]))
    b = prob.shape_derivative(0.0)
    b_ref = sum(inverse.rhs(m.coords, m.cells, A, LAM, MU, r["u"], r["v"], r["p"], r["q"], r["g"], ALPHA) for r in ref)
    assert close_scaled(b, b_ref, 1e-12), np.max(np.abs(b - b_ref)) / np.max(np.abs(b_ref))


def test_zero_at_the_true_inclusion(ctx, api):
    """Measurement = the displacement at the true inclusion: J and b vanish there on the GPU."""
    m = BoxMesh(2, (20, 16), (0.0, 0.0), (1.0, 1.0))
    phi = _phi(m, 4)
    f0, f1 = _faces(2)
    dir0 = m.dirichlet_mask(f0, 2)
    A, _ = shape.coefficient(phi, m.cells, 10.0, 1.0)
    K = inverse.elastic_matrix(m.coords, m.cells, A, LAM, MU)
    ax, sd, t = _tractions(2, 1)[0]
    F = fem.facet_load(m.coords, m.boundary_facets(ax, sd), t, 2)
    F[dir0 == 1] = 0.0
    g = inverse.states(m, K, F, np.zeros(m.coords.size), dir0)[0]
    mesh, prob = _gpu(ctx, api, m, phi, [g], 1)
    prob.state_solve(_opts(api))
    J, _ = prob.functionals()
    assert J <= 1e-20, J
    prob.adjoint_solve(_opts(api))
    b = prob.shape_derivative(0.0)
    assert np.max(np.abs(b)) <= 1e-10, np.max(np.abs(b))


def test_algorithm_iteration(ctx, api):
    """One Algorithm-1 iteration (velocity 0.1 mass + Laplacian on H^1_0, as the paper's example):
    J, B(theta, theta), theta and the transported phi."""
    m = BoxMesh(2, (24, 24), (0.0, 0.0), (1.0, 1.0))
    phi = _phi(m, 5)
    meas = _meas(m, 2, 8)
    A, chi, ref = _oracle(m, phi, meas, 2)
    mesh, prob = _gpu(ctx, api, m, phi, meas, 2)
    so = _opts(api)
    ro = api.run_options(dfactor=1e-2, lv_time=(1e-3, 1e-1), lv_iter=(8, 16), smooth=False, state=so, velocity=so,
                         transport=so)
    log = prob.opt_step(0, ro, api.PPL(0))
    b = sum(inverse.rhs(m.coords, m.cells, A, LAM, MU, r["u"], r["v"], r["p"], r["q"], r["g"], ALPHA) for r in ref)
    form = ovel.VelocityForm(alpha_mass=0.1, dirichlet=True)
    theta, Btt = ovel.solve(m, form, b)
    t_end, ns = oppl.adaptime(Btt, 1e-2, (1e-3, 1e-1), (8, 16))
    phi1 = levelset.transport(m, phi, theta, t_end, ns, m.diameter(), False)
    J_ref = sum(r["J"] for r in ref)
    assert abs(log.J - J_ref) <= 1e-10 * abs(J_ref)
    assert abs(log.Btt - Btt) <= 1e-9 * abs(Btt), (log.Btt, Btt)
    assert log.nsteps == ns
    assert close_scaled(prob.get(api.FO_FIELD_THETA), theta, 1e-9)
    assert close_scaled(prob.get(api.FO_FIELD_PHI), phi1, 1e-9)


@pytest.mark.parametrize("dim,n", [(2, (23, 17)), (3, (6, 5, 4))])
def test_dirichlet_extension(ctx, api, dim, n):
    """fo_dirichlet_extension against the oracle's (Sec. 5.7): values kept on the faces, the
    harmonic extension elsewhere; linear data extend to the linear field."""
    m = BoxMesh(dim, n, (0.0,) * dim, (1.0,) * dim)
    mesh = ctx.mesh_box(dim, n, (0.0,) * dim, (1.0,) * dim)
    faces = [(0, 1), (1, 0), (1, 1)]
    vals = workloads.smooth_field(m.coords, dim, 3)
    eta = mesh.dirichlet_extension(faces, vals, api.solve_opts(rtol=1e-13, maxit=100000))
    ref = inverse.dirichlet_extension(m, vals, faces)
    assert close_scaled(eta, ref, 1e-10), np.max(np.abs(eta - ref))
    G = np.random.default_rng(1).standard_normal((dim, dim))
    lin = (m.coords @ G.T).reshape(-1)
    eta = mesh.dirichlet_extension([(a, s) for a in range(dim) for s in (0, 1)], lin,
                                   api.solve_opts(rtol=1e-13, maxit=100000))
    assert close_scaled(eta, lin, 1e-10)
