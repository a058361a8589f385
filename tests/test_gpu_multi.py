"""Several load cases (eq. compli_plus) and several region volume constraints (Sec. 5.4 with
N_c > 1) on the GPU against the oracle: per-case states, the summed cost, the constraint vector,
the shape derivative with one multiplier per constraint, and whole iterations with one PPL
update of the vector C -- on the box path and on a general mesh."""
import numpy as np
import pytest

from oracle import algorithm as oalg, levelset, ppl as oppl, shape, velocity as ovel
from oracle.mesh import ArrayMesh, BoxMesh
from paper_2601_05709_gb300 import workloads
from tests.helpers import assert_solve_parity, close_scaled, node_at, umesh

pytestmark = pytest.mark.gpu

REGIONS = [((-np.inf, -np.inf), (1.0, np.inf), 0.35), ((1.0, -np.inf), (np.inf, np.inf), 0.55)]


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


def _setup(api, ctx, kind, general, regions=True):
    """(gpu problem, oracle problem, coords) of a two-load-case problem on (0,2) x (0,1)."""
    if general:
        coords, cells = umesh(dim=2, n=(24, 12), hi=(2.0, 1.0), jitter=0.3, seed=6)
        om = ArrayMesh(coords, cells)
        mesh = ctx.mesh_from_arrays(coords, cells)
    else:
        om = BoxMesh(2, (32, 16), (0.0, 0.0), (2.0, 1.0))
        coords = om.coords
        mesh = ctx.mesh_box(2, (32, 16), (0.0, 0.0), (2.0, 1.0))
    tip, top = node_at(coords, (2.0, 0.5)), node_at(coords, (1.25, 1.0))
    if kind == 1:
        cases = [([(tip, (0.0, -1.0))], []), ([(top, (0.4, -0.6))], [(1, 0, (0.0, 0.3))])]
        f = None
    else:   # heat: source f in case 0, a flux on the top face in case 1
        cases = [([], []), ([(top, (1.0,))], [(1, 1, (0.5,))])]
        f = 1.0 + coords[:, 1]
    vr = REGIONS if regions else None
    desc = api.model_desc(kind, dirichlet=[(0, 0)], f_nodal=f, load_cases=cases, volume=1.0, volume_regions=vr,
                          alpha_mass=0.1, normal_penalty=1e4 if kind == 1 else 0.0,
                          velocity_dirichlet=kind == 0)
    prob = mesh.problem(desc)
    op = oalg.Problem(mesh=om, kind=kind, dirichlet_faces=[(0, 0)], f_nodal=f, load_cases=cases,
                      volume_target=1.0, volume_regions=vr,
                      vform=ovel.VelocityForm(alpha_mass=0.1, normal_penalty=1e4 if kind == 1 else 0.0,
                                              dirichlet=kind == 0))
    return prob, op, coords


@pytest.mark.parametrize("general", [False, True], ids=["box", "arrays"])
@pytest.mark.parametrize("kind", [0, 1])
def test_cases_states_cost_constraints_and_rhs(ctx, api, general, kind):
    prob, op, coords = _setup(api, ctx, kind, general)
    phi = workloads.phi_cos(coords)
    prob.set_levelset(phi)
    np.testing.assert_array_equal(prob.get(api._lib.FO_FIELD_LOAD).shape, (2, op.ncomp * coords.shape[0]))
    assert close_scaled(prob.get(api._lib.FO_FIELD_LOAD).ravel(),
                        np.concatenate([op.case_load(0), op.case_load(1)]), 1e-14)
    st = prob.state_solve(api.solve_opts(rtol=1e-13, maxit=400000))
    U = prob.get(api._lib.FO_FIELD_U)
    U_ref, A, chi = op.states(phi)
    K, free = op.stiffness(A), op.dirichlet() == 0
    for k in range(2):
        assert_solve_parity(K, op.case_load(k), free, U[k], U_ref[k], 1e-10, omega_max=1e-12)
    J, C = prob.functionals_v()
    assert abs(J - op.total_cost(U_ref, A)) <= 1e-9 * abs(J)
    assert np.allclose(C, op.constraints(chi), rtol=1e-13, atol=0)
    # shape derivative with one multiplier per constraint, on the oracle's states
    prob.set(api._lib.FO_FIELD_U, U_ref.ravel())
    lams = np.array([0.4, -0.7])
    b = prob.shape_derivative_v(lams)
    ref = op.total_rhs(U_ref, A, chi, lams)
    # the states of the ersatz-1e-3 material are large (|u| ~ 1e4) and a node's element terms
    # cancel to a much smaller sum: elementwise 1e-10 of the vector's scale
    assert close_scaled(b, ref, 1e-10), np.max(np.abs(b - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("general", [False, True], ids=["box", "arrays"])
def test_iterations_with_two_cases_and_two_constraints(ctx, api, general):
    prob, op, coords = _setup(api, ctx, 1, general)
    cen, rad = workloads.hole_lattice()
    phi = levelset.initial_level(coords, cen, rad)
    prob.set_levelset(phi)
    so = api.solve_opts(rtol=1e-13, maxit=400000)
    run = api.run_options(dfactor=1e-1, smooth=True, state=so, velocity=so, transport=so)
    ppl, ost = api.PPL(2), oppl.PPL(2)
    oopts = oalg.RunOptions(dfactor=1e-1, smooth=True)
    for i in range(3):
        log = prob.opt_step(i, run, ppl)
        phi, olog = oalg.opt_step(op, phi, i, ost, oopts)
        assert log.nc == 2
        assert abs(log.J - olog["J"]) <= 1e-9 * abs(olog["J"]), (i, log.J, olog["J"])
        assert np.allclose(list(log.Cv)[:2], olog["C"], rtol=1e-12, atol=0)
        assert np.allclose(list(log.lambdav)[:2], olog["lam"], rtol=1e-9, atol=1e-12)
        assert log.nsteps == olog["nsteps"]
        assert close_scaled(prob.get(api._lib.FO_FIELD_PHI), phi, 1e-8)


def test_ppl_size_must_match(ctx, api):
    prob, op, coords = _setup(api, ctx, 1, False)
    prob.set_levelset(workloads.phi_cos(coords))
    with pytest.raises(api.FormoptError) as e:
        prob.opt_step(0, api.run_options(), api.PPL(1))
    assert e.value.status == api._lib.FO_EINVAL
