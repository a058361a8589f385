"""General simplicial meshes given as arrays (fo_mesh_from_arrays) on the GPU against the
FP64 oracle on the same arrays: jittered meshes with shuffled numbering, a 2D mesh with
alternating diagonals (a connectivity the box path cannot produce) and a 3D one.

Tolerances as for the box path: element flags and masks bit-exact; loads 1e-14 and
operator applies / shape RHS / transport matrices 1e-12 of the vector's scale; solves 1e-10
(or the perturbation bound, tests/helpers.assert_solve_parity), mixed 1e-8; transport steps
1e-11 and reinitialisation 1e-10 element by element; whole iterations 1e-9 on J and 1e-8 on phi.
"""
import numpy as np
import pytest

from oracle import algorithm as oalg, fem, levelset, ppl as oppl, shape, velocity as ovel
from oracle.mesh import ArrayMesh
from paper_2601_05709_gb300 import workloads
from tests.helpers import (assert_solve_parity, case, close_scaled, gpu_problem, gpu_umesh_problem, node_at,
                           oracle_problem, oracle_umesh_problem, umesh)

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


def tight(api, precision=None):
    return api.solve_opts(precision=api.FO_FP64 if precision is None else precision, rtol=1e-13, maxit=400000)


MESHES = {
    "2d_alternate": dict(dim=2, n=(12, 8), hi=(2.0, 1.0), jitter=0.3, seed=1, pattern="alternate"),
    "2d_kuhn": dict(dim=2, n=(16, 8), hi=(2.0, 1.0), jitter=0.3, seed=2),
    "3d_kuhn": dict(dim=3, n=(5, 3, 3), hi=(2.0, 1.0, 1.0), jitter=0.25, seed=3),
}


def mesh_arrays(name):
    return umesh(**MESHES[name])


def phi_of(coords):
    d = coords.shape[1]
    if d == 2:
        return workloads.phi_cos(coords)
    return workloads.phi_bumps(coords, workloads.bump_centres((0, 0, 0), (2, 1, 1), 5, 4), 0.3, 0.4)


def elastic_case(dim, **kw):
    tip = (2.0, 0.5) if dim == 2 else (2.0, 0.5 + 1.0 / 6.0, 0.5 + 1.0 / 6.0)
    base = dict(dim=dim, kind=1, dirichlet=[(0, 0)], point_loads=[(tip, (0.0, -1.0, 0.0)[:dim])],
                tractions=[(1, 1, (0.2, -0.1, 0.05)[:dim])], volume=1.0, alpha_mass=0.1, normal_penalty=1e4,
                omega0_weight=1e4, omega0_boxes=[((1.6,) + (0.3,) * (dim - 1), (np.inf,) + (0.7,) * (dim - 1))])
    base.update(kw)
    return case(**base)


def heat_case(dim, **kw):
    base = dict(dim=dim, kind=0, dirichlet=[(0, 0)], f=lambda X: 1.0 + X[:, 1] - 0.3 * X[:, 0], volume=0.8,
                alpha_mass=0.01, velocity_dirichlet=True)
    base.update(kw)
    return case(**base)


@pytest.mark.parametrize("name", list(MESHES))
def test_umesh_query_and_copy_out(ctx, name):
    coords, cells = mesh_arrays(name)
    m = ctx.mesh_from_arrays(coords, cells)
    om = ArrayMesh(coords, cells)
    c2, x2 = m.copy_out()
    assert np.array_equal(c2, cells) and np.array_equal(x2, coords)
    assert m.num_nodes == om.num_nodes and m.num_elems == om.num_elems
    assert abs(m.volume - om.volume()) <= 1e-13 * om.volume()
    assert abs(m.h - om.diameter()) <= 1e-14 * om.diameter()


@pytest.mark.parametrize("name", list(MESHES))
def test_umesh_coefficients_and_masks_bit_exact(ctx, api, name):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    c = elastic_case(dim)
    _, prob = gpu_umesh_problem(ctx, coords, cells, c)
    op = oracle_umesh_problem(coords, cells, c)
    phi = phi_of(coords)
    phi[:30] = 0.0                                       # planted ties: a zero sum is outside
    prob.set_levelset(phi)
    prob.coefficients()
    A, chi = shape.coefficient(phi, cells, c["a_in"], c["a_out"])
    assert np.array_equal(prob.get(api._lib.FO_FIELD_CHI).astype(np.uint8), chi)
    assert np.array_equal(prob.get(api._lib.FO_FIELD_COEF), A)
    assert np.array_equal(prob.get(api._lib.FO_FIELD_OMEGA0).astype(np.uint8),
                          op.mesh.subdomain_mask(c["omega0_boxes"]))


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("kind", [0, 1])
def test_umesh_loads(ctx, api, name, kind):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    c = elastic_case(dim) if kind == 1 else heat_case(dim, dirichlet=[(0, 0), (1, 1)])
    _, prob = gpu_umesh_problem(ctx, coords, cells, c)
    op = oracle_umesh_problem(coords, cells, c)
    assert close_scaled(prob.get(api._lib.FO_FIELD_LOAD), op.load(), 1e-14)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_umesh_state_apply(ctx, api, name, kind):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    c = {0: heat_case(dim), 1: elastic_case(dim), 2: heat_case(dim, kind=2, k=1.3, omega=2.7)}[kind]
    _, prob = gpu_umesh_problem(ctx, coords, cells, c)
    op = oracle_umesh_problem(coords, cells, c)
    phi = phi_of(coords)
    prob.set_levelset(phi)
    A, _ = shape.coefficient(phi, cells, c["a_in"], c["a_out"])
    K = op.stiffness(A)
    dmask = op.dirichlet()
    x = workloads.random_field(K.shape[0], 9)
    y = prob.apply(api._lib.FO_OP_STATE, x)
    ref = K @ np.where(dmask == 1, 0.0, x)
    ref[dmask == 1] = 0.0
    assert close_scaled(y, ref, 1e-12)
    y32 = prob.apply(api._lib.FO_OP_STATE_FP32, x)
    assert close_scaled(y32, ref, 2e-5)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("kind", [0, 1])
def test_umesh_state_solve(ctx, api, name, kind):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    c = elastic_case(dim) if kind == 1 else heat_case(dim)
    _, prob = gpu_umesh_problem(ctx, coords, cells, c)
    op = oracle_umesh_problem(coords, cells, c)
    phi = phi_of(coords)
    prob.set_levelset(phi)
    prob.state_solve(tight(api))
    u = prob.get(api._lib.FO_FIELD_U)
    u_ref, A, chi = op.state(phi)
    K, F, free = op.stiffness(A), op.load(), op.dirichlet() == 0
    fwd, om, skeel = assert_solve_parity(K, F, free, u, u_ref, 1e-10, omega_max=1e-12)
    J, C = prob.functionals()
    J_ref = op.cost(u_ref, A)
    assert abs(J - J_ref) <= max(1e-10, 4 * fwd) * abs(J_ref)
    assert abs(C - op.constraint(chi)) <= 1e-13 * abs(op.constraint(chi))
    # FP32 inner solves in FP64 refinement: 1e-8
    prob.state_solve(api.solve_opts(precision=api.FO_MIXED, rtol=1e-12, inner_rtol=1e-3))
    assert close_scaled(prob.get(api._lib.FO_FIELD_U), u_ref, 1e-8)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("kind,lam", [(0, 0.6), (1, 0.35)])
def test_umesh_shape_rhs(ctx, api, name, kind, lam):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    c = elastic_case(dim) if kind == 1 else heat_case(dim)
    _, prob = gpu_umesh_problem(ctx, coords, cells, c)
    op = oracle_umesh_problem(coords, cells, c)
    phi = phi_of(coords)
    prob.set_levelset(phi)
    prob.coefficients()
    u = workloads.smooth_field(coords, op.ncomp, 17)
    u[op.dirichlet() == 1] = 0.0
    prob.set(api._lib.FO_FIELD_U, u)
    b = prob.shape_derivative(lam)
    A, chi = shape.coefficient(phi, cells, c["a_in"], c["a_out"])
    assert close_scaled(b, op.rhs(u, A, chi, lam), 1e-12)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("kind", [0, 1])
def test_umesh_velocity(ctx, api, name, kind):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    c = elastic_case(dim) if kind == 1 else heat_case(dim)
    _, prob = gpu_umesh_problem(ctx, coords, cells, c)
    op = oracle_umesh_problem(coords, cells, c)
    prob.set_levelset(-np.ones(coords.shape[0]))
    prob.coefficients()
    free = ovel.free_nodes(op.mesh, op.vform)
    x = workloads.random_field(dim * coords.shape[0], 4)
    y = prob.apply(api._lib.FO_OP_VELOCITY, x).reshape(-1, dim)
    x2 = x.reshape(-1, dim)
    for a in range(dim):
        B = ovel.component_matrix(op.mesh, op.vform, a)
        ref = B @ np.where(free, x2[:, a], 0.0)
        assert close_scaled(y[free, a], ref[free], 1e-12)
    b = workloads.smooth_field(coords, dim, 23)
    prob.set(api._lib.FO_FIELD_RHS, b)
    Btt, st = prob.descent(tight(api))
    theta_ref, Btt_ref = ovel.solve(op.mesh, op.vform, b)
    assert close_scaled(prob.get(api._lib.FO_FIELD_THETA), theta_ref, 1e-10)
    assert abs(Btt - Btt_ref) <= 1e-10 * abs(Btt_ref)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("smooth", [False, True])
def test_umesh_transport(ctx, api, name, smooth):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    c = heat_case(dim)
    _, prob = gpu_umesh_problem(ctx, coords, cells, c)
    m = ArrayMesh(coords, cells)
    theta = workloads.smooth_field(coords, dim, 31)
    phi = phi_of(coords)
    prob.set(api._lib.FO_FIELD_THETA, theta)
    prob.set_levelset(phi)
    h, t_end, ns = m.diameter(), 0.05, 9
    dt = t_end / ns
    prob.transport_assemble(dt, h, smooth)
    L, R = levelset.transport_matrices(m, theta, dt, h, smooth)
    x = workloads.random_field(m.num_nodes, 3)
    assert close_scaled(prob.apply(api._lib.FO_OP_TRANSPORT_L, x), L @ x, 1e-12)
    assert close_scaled(prob.apply(api._lib.FO_OP_TRANSPORT_R, x), R @ x, 1e-12)
    prob.levelset_step(t_end, ns, h, smooth, tight(api))
    ref = levelset.transport(m, phi, theta, t_end, ns, h, smooth)
    out = prob.get(api._lib.FO_FIELD_PHI)
    assert close_scaled(out, ref, 1e-11), np.max(np.abs(out - ref))


@pytest.mark.parametrize("name", list(MESHES))
def test_umesh_reinit(ctx, api, name):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    _, prob = gpu_umesh_problem(ctx, coords, cells, heat_case(dim))
    m = ArrayMesh(coords, cells)
    phi = 2.5 * levelset.initial_level(coords, [(0.9,) + (0.5,) * (dim - 1), (0.3,) * dim], [0.3, 0.15])
    prob.set_levelset(phi)
    h = m.diameter()
    prob.reinit(6, 0.05, h, tight(api))
    ref = levelset.reinit(m, phi, 6, 0.05, h)
    out = prob.get(api._lib.FO_FIELD_PHI)
    assert close_scaled(out, ref, 1e-10), np.max(np.abs(out - ref))


@pytest.mark.parametrize("name,iters", [("2d_alternate", 3), ("3d_kuhn", 2)])
def test_umesh_iterations_with_ppl_and_reinit(ctx, api, name, iters):
    coords, cells = mesh_arrays(name)
    dim = coords.shape[1]
    c = elastic_case(dim)
    _, prob = gpu_umesh_problem(ctx, coords, cells, c)
    op = oracle_umesh_problem(coords, cells, c)
    cen = np.array([[0.5] + [0.5] * (dim - 1), [1.3] + [0.5] * (dim - 1)])
    phi = levelset.initial_level(coords, cen, [0.2, 0.2])
    prob.set_levelset(phi)
    so = api.solve_opts(rtol=1e-13, maxit=400000)
    run = api.run_options(dfactor=1e-1, smooth=True, reinit_step=2, reinit_pars=(6, 0.05), state=so, velocity=so,
                          transport=so)
    ppl, oppl_state = api.PPL(1), oppl.PPL(1)
    oopts = oalg.RunOptions(dfactor=1e-1, smooth=True, reinit_step=2, reinit_pars=(6, 0.05))
    for i in range(iters):
        log = prob.opt_step(i, run, ppl)
        phi, olog = oalg.opt_step(op, phi, i, oppl_state, oopts)
        assert abs(log.J - olog["J"]) <= 1e-9 * abs(olog["J"]), (i, log.J, olog["J"])
        assert abs(log.C - olog["C"]) <= 1e-12
        assert log.nsteps == olog["nsteps"] and bool(log.reinit) == olog["reinit"]
        gphi = prob.get(api._lib.FO_FIELD_PHI)
        assert close_scaled(gphi, phi, 1e-8), (i, np.max(np.abs(gphi - phi)))


def test_umesh_on_kuhn_arrays_matches_box_path(ctx, api):
    """The box mesh's own arrays, renumbered, through the general path: the same state, cost,
    shape derivative and descent direction as the structured path (solved to 1e-13)."""
    c = elastic_case(2, n=(16, 8), lo=(0, 0), hi=(2, 1), point_loads=[((16, 4), (0.0, -1.0))], tractions=[],
                     omega0_boxes=[((1.6, 0.3), (np.inf, 0.7))])
    bm, bprob = gpu_problem(ctx, c)
    cells, coords = bm.copy_out()
    rng = np.random.default_rng(11)
    newid = rng.permutation(coords.shape[0])
    inv = np.empty_like(newid)
    inv[newid] = np.arange(newid.size)
    ucoords, ucells = coords[inv], newid[cells].astype(np.int32)
    cu = dict(c, point_loads=[((2.0, 0.5), (0.0, -1.0))])
    _, uprob = gpu_umesh_problem(ctx, ucoords, ucells, cu)
    phi = workloads.phi_cos(coords)
    for p, ph in ((bprob, phi), (uprob, phi[inv])):
        p.set_levelset(ph)
        p.state_solve(tight(api))
    J0, C0 = bprob.functionals()
    J1, C1 = uprob.functionals()
    assert abs(J1 - J0) <= 1e-10 * abs(J0) and abs(C1 - C0) <= 1e-14 * abs(C0)
    idx = (inv[:, None] * 2 + np.arange(2)[None, :]).ravel()
    u0 = bprob.get(api._lib.FO_FIELD_U)
    assert close_scaled(uprob.get(api._lib.FO_FIELD_U), u0[idx], 1e-10)
    b0, b1 = bprob.shape_derivative(0.3), uprob.shape_derivative(0.3)
    assert close_scaled(b1, b0[idx], 1e-10)
    t0, _ = bprob.descent(tight(api))
    t1, _ = uprob.descent(tight(api))
    assert abs(t1 - t0) <= 1e-10 * abs(t0)
    assert close_scaled(uprob.get(api._lib.FO_FIELD_THETA), bprob.get(api._lib.FO_FIELD_THETA)[idx], 1e-10)
