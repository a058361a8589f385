"""GPU tests of the request server: results in a concurrent mix equal the same requests run
alone (same bits), served results equal the direct API, the memory estimate is exact, and a
served heat request matches the oracle."""
import numpy as np
import pytest

from paper_2601_05709_gb300 import api, workloads
from paper_2601_05709_gb300.api import FO_ELASTIC, FO_HEAT
from tests.helpers import close_scaled, oracle_problem, case, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _desc(kind, dim):
    if kind == FO_HEAT:
        return api.model_desc(FO_HEAT, dirichlet=[(0, 0)], f_nodal=None, alpha_mass=0.01, velocity_dirichlet=True)
    face_vec = (0.0, -1.0) if dim == 2 else (0.0, 0.0, -1.0)
    return api.model_desc(FO_ELASTIC, dirichlet=[(0, 0)], tractions=[(0, 1, face_vec)], volume=0.5,
                          alpha_mass=0.1, normal_penalty=1e4)


def _mix():
    rng = np.random.default_rng(11)
    out = []
    for i, (dim, n, kind) in enumerate([(2, 16, FO_HEAT), (2, 24, FO_ELASTIC), (3, 6, FO_HEAT), (2, 20, FO_HEAT),
                                        (3, 5, FO_ELASTIC), (2, 12, FO_ELASTIC), (3, 7, FO_HEAT), (2, 28, FO_HEAT),
                                        (2, 18, FO_ELASTIC), (3, 6, FO_ELASTIC)]):
        centers = rng.random((6, dim))
        lam = 0.3 if kind == FO_ELASTIC else 0.0
        out.append((dim, n, kind, centers, lam))
    return out


def _request(dim, n, kind, centers, lam, phi=None):
    opts = api.solve_opts(rtol=1e-10)
    if phi is not None:
        return api.ServedRequest(dim, (n,) * dim, _desc(kind, dim), phi=phi, lam=lam, state=opts, want_theta=True)
    return api.ServedRequest(dim, (n,) * dim, _desc(kind, dim), centers=centers, width=0.15, offset=0.2, lam=lam,
                             state=opts, want_theta=True)


def _serve(ctx, items, executors):
    srv = api.Server(ctx, executors=executors)
    reqs = [_request(*it) for it in items]
    tickets = [srv.submit(r)[1] for r in reqs]
    res = [srv.wait(t, 120.0) for t in tickets]
    st = srv.stats()
    srv.close()
    return reqs, res, st


def test_mix_equals_alone(ctx):
    items = _mix()
    reqs_mix, res_mix, st = _serve(ctx, items, executors=4)
    assert st.failed == 0 and st.completed == len(items)
    assert st.peak_in_flight >= 2                       # requests did overlap
    for it, rq_m, r_m in zip(items, reqs_mix, res_mix):
        assert r_m is not None and r_m.status == 0, r_m.message
        (rq_a,), (r_a,), _ = _serve(ctx, [it], executors=1)
        assert (r_m.J, r_m.C, r_m.Btt) == (r_a.J, r_a.C, r_a.Btt), it
        assert np.array_equal(rq_m.theta, rq_a.theta), it
        assert r_m.state.iterations == r_a.state.iterations


def test_served_equals_direct_api(ctx):
    dim, n, kind, centers, lam = _mix()[1]
    (rq,), (r,), _ = _serve(ctx, [(dim, n, kind, centers, lam)], executors=2)
    mesh = ctx.mesh_box(dim, (n,) * dim, (0.0,) * dim, (1.0,) * dim)
    prob = mesh.problem(_desc(kind, dim))
    prob._chk(prob.lib.fo_levelset_bumps(prob.handle, len(centers), api._dp(np.ascontiguousarray(centers).reshape(-1)),
                                         0.15, 0.2), "fo_levelset_bumps")
    opts = api.solve_opts(rtol=1e-10)
    prob.coefficients()
    prob.state_solve(opts)
    prob.adjoint_solve(opts)
    J, C = prob.functionals()
    prob.shape_derivative(lam, copy=False)
    Btt, _ = prob.descent(api.solve_opts())
    assert (J, C, Btt) == (r.J, r.C, r.Btt)
    assert np.array_equal(prob.get(api.FO_FIELD_THETA), rq.theta)


@pytest.mark.parametrize("kind,dim,n,prec,pc", [(FO_HEAT, 2, 20, api.FO_FP64, 0), (FO_ELASTIC, 2, 16, api.FO_MIXED, 0),
                                                (FO_ELASTIC, 3, 5, api.FO_FP64, 0),
                                                (FO_ELASTIC, 2, 64, api.FO_FP64, api.FO_PC_MG),
                                                (FO_HEAT, 3, 16, api.FO_FP64, api.FO_PC_MG),
                                                (FO_HEAT, 2, 63, api.FO_FP64, api.FO_PC_MG)])
def test_request_footprint_exact(kind, dim, n, prec, pc):
    """The estimate equals what the request allocates, multigrid hierarchies included (the
    odd 63x63 grid coarsens to non-nested levels)."""
    c2 = api.Context(0)
    phi = workloads.phi_cos(np.random.default_rng(0).random((int((n + 1) ** dim), dim)))
    rq = api.ServedRequest(dim, (n,) * dim, _desc(kind, dim), phi=phi,
                           state=api.solve_opts(precision=prec, rtol=1e-9, precond=pc),
                           velocity=api.solve_opts(precond=pc))
    mesh = c2.mesh_box(dim, (n,) * dim, (0.0,) * dim, (1.0,) * dim)
    prob = mesh.problem(_desc(kind, dim))
    prob.set_levelset(phi)
    prob.coefficients()
    prob.state_solve(rq.struct.state, allow_noconv=True)
    prob.adjoint_solve(rq.struct.state)
    prob.shape_derivative(0.0, copy=False)
    prob.descent(rq.struct.velocity)
    assert c2.memory() == rq.device_bytes()
    c2.close()


def test_served_heat_matches_oracle(ctx):
    n = 24
    c = case(dim=2, n=(n, n), kind=FO_HEAT, f=lambda X: np.ones(X.shape[0]), dirichlet=[(0, 0)], alpha_mass=0.01,
             velocity_dirichlet=True)
    op = oracle_problem(c)
    phi = workloads.phi_cos(op.mesh.coords)
    desc = api.model_desc(FO_HEAT, dirichlet=[(0, 0)], f_nodal=np.ones(op.mesh.num_nodes), alpha_mass=0.01,
                          velocity_dirichlet=True)
    rq = api.ServedRequest(2, (n, n), desc, phi=phi, state=api.solve_opts(rtol=1e-13),
                           velocity=api.solve_opts(rtol=1e-13), want_theta=True)
    srv = api.Server(ctx, executors=2)
    st, t = srv.submit(rq)
    r = srv.wait(t, 60.0)
    srv.close()
    assert r.status == 0
    u, A, chi = op.state(phi)
    J = op.cost(u, A)
    assert abs(r.J - J) <= 1e-10 * abs(J)
    from oracle import velocity as ovel
    theta, Btt = ovel.solve(op.mesh, op.vform, op.rhs(u, A, chi, 0.0))
    assert close_scaled(rq.theta, theta, 1e-10), np.max(np.abs(rq.theta - theta))
    assert abs(r.Btt - Btt) <= 1e-10 * abs(Btt)


@pytest.mark.parametrize("prec", [api.FO_FP64, api.FO_MIXED])
def test_concurrent_multigrid_requests_of_distinct_sizes(ctx, prec):
    """Eight executors launching multigrid solves whose staged shared memory differs from request
    to request (the kernel's shared-memory limit is process-wide state): every request runs, and
    in-mix results equal the same request served alone (same bits)."""
    rng = np.random.default_rng(5)
    items = []
    for i, n in enumerate([40, 72, 96, 130, 64, 100, 150, 84, 112, 56, 140, 90, 120, 48, 160, 76, 33, 45]):
        kind = FO_HEAT if i % 2 == 0 else FO_ELASTIC
        items.append((2, n, kind, rng.random((6, 2))))

    def req(dim, n, kind, centers):
        return api.ServedRequest(dim, (n,) * dim, _desc(kind, dim), centers=centers, width=0.15, offset=0.2,
                                 state=api.solve_opts(precision=prec, rtol=1e-9, precond=api.FO_PC_MG),
                                 velocity=api.solve_opts(rtol=1e-9, precond=api.FO_PC_MG), want_theta=True)

    def serve(its, executors):
        srv = api.Server(ctx, executors=executors)
        reqs = [req(*it) for it in its]
        res = [srv.wait(srv.submit(r)[1], 300.0) for r in reqs]
        st = srv.stats()
        srv.close()
        return reqs, res, st

    reqs, res, st = serve(items, 8)
    assert st.failed == 0 and st.completed == len(items)
    for it, r in zip(items, res):
        assert r is not None and r.status == 0, (it[:3], r.message)
        if it[2] == FO_ELASTIC:   # (the heat requests here have no source: a zero state)
            assert r.state.iterations > 0
    for k in (0, 3, 6):
        (rq_a,), (r_a,), _ = serve([items[k]], 1)
        assert (res[k].J, res[k].C, res[k].Btt) == (r_a.J, r_a.C, r_a.Btt), items[k][:3]
        assert np.array_equal(reqs[k].theta, rq_a.theta)


def test_grid_share_agrees_with_full_grid(ctx):
    """A context whose persistent launches take half the co-resident blocks solves the same
    system to the solve tolerance (the grid changes only the order of the block sums)."""
    c2 = api.Context(0)
    c2.set_grid_share(2)
    out = []
    for c in (ctx, c2):
        mesh = c.mesh_box(3, (24, 12, 12), (0.0, 0.0, 0.0), (2.0, 1.0, 1.0))
        _, coords = mesh.copy_out()
        prob = mesh.problem(_desc(FO_ELASTIC, 3))
        prob.set_levelset(workloads.phi_bumps(coords, workloads.bump_centres((0, 0, 0), (2, 1, 1), 6, seed=3), 0.2, 0.2))
        st = prob.state_solve(api.solve_opts(rtol=1e-12, precond=api.FO_PC_MG))
        out.append((prob.get(api.FO_FIELD_U), st.iterations))
    assert close_scaled(out[1][0], out[0][0], 1e-10)
    with pytest.raises(api.FormoptError):
        c2.set_grid_share(0)
    c2.close()
