"""The exact cut-cell coefficient (FO_COEF_CUT) on the GPU against the oracle's convex-hull
volumes: the fraction, A_e and chi_e per element (1e-14), and a whole Algorithm-1 iteration
(cost, constraint, shape derivative, velocity, transport) on the box path and on a general
mesh."""
import numpy as np
import pytest

from oracle import algorithm as oalg, ppl as oppl, shape, levelset
from paper_2601_05709_gb300 import workloads
from tests.helpers import (cantilever2d, case, close_scaled, gpu_problem, gpu_umesh_problem, oracle_problem,
                           oracle_umesh_problem, umesh)

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


def _cut(api, ctx, c, coords=None, cells=None):
    c = dict(c, coef_rule=1)
    return gpu_problem(ctx, c) if coords is None else gpu_umesh_problem(ctx, coords, cells, c)


@pytest.mark.parametrize("dim,n", [(2, (31, 17)), (3, (9, 7, 5))])
def test_cut_fraction_per_element(ctx, api, dim, n):
    c = case(dim=dim, n=n, hi=(2.0,) + (1.0,) * (dim - 1), kind=0, a_in=1.0, a_out=1e-3, coef_rule=1)
    mesh, prob = _cut(api, ctx, c)
    op = oracle_problem(c)
    m = op.mesh
    phi = workloads.phi_cos(m.coords) if dim == 2 else workloads.phi_bumps(
        m.coords, workloads.bump_centres((0,) * 3, (2, 1, 1), 6, 1), 0.3, 0.4)
    phi[:25] = 0.0                                         # vertices exactly on the interface
    prob.set_levelset(phi)
    prob.coefficients()
    A_ref, f_ref = shape.coefficient_cut(phi, m.cells, 1.0, 1e-3)
    f = prob.get(api._lib.FO_FIELD_CHI)
    assert np.max(np.abs(f - f_ref)) <= 1e-14
    assert np.max(np.abs(prob.get(api._lib.FO_FIELD_COEF) - A_ref)) <= 1e-14
    assert 0 < np.count_nonzero((f_ref > 0) & (f_ref < 1))   # cut elements are present


@pytest.mark.parametrize("general", [False, True], ids=["box", "arrays"])
def test_cut_rule_iteration(ctx, api, general):
    if general:
        coords, cells = umesh(dim=2, n=(24, 12), hi=(2.0, 1.0), jitter=0.3, seed=5, pattern="alternate")
        c = case(dim=2, kind=1, dirichlet=[(0, 0)], point_loads=[((2.0, 0.5), (0.0, -1.0))], volume=1.0,
                 alpha_mass=0.1, normal_penalty=1e4)
        mesh, prob = _cut(api, ctx, c, coords, cells)
        op = oracle_umesh_problem(coords, cells, dict(c, coef_rule=1))
    else:
        c = cantilever2d((48, 24))
        mesh, prob = _cut(api, ctx, c)
        op = oracle_problem(dict(c, coef_rule=1))
    cen, rad = workloads.hole_lattice()
    phi = levelset.initial_level(op.mesh.coords, cen, rad)
    prob.set_levelset(phi)
    so = api.solve_opts(rtol=1e-13, maxit=400000)
    run = api.run_options(dfactor=1e-1, smooth=True, state=so, velocity=so, transport=so)
    ppl, ost = api.PPL(1), oppl.PPL(1)
    oopts = oalg.RunOptions(dfactor=1e-1, smooth=True)
    for i in range(2):
        log = prob.opt_step(i, run, ppl)
        phi, olog = oalg.opt_step(op, phi, i, ost, oopts)
        assert abs(log.C - olog["C"]) <= 1e-13 * abs(olog["C"])
        assert abs(log.J - olog["J"]) <= 1e-9 * abs(olog["J"]), (i, log.J, olog["J"])
        if i == 0:
            assert close_scaled(prob.get(api._lib.FO_FIELD_RHS), olog["rhs"], 1e-9)
        assert log.nsteps == olog["nsteps"]
        assert close_scaled(prob.get(api._lib.FO_FIELD_PHI), phi, 1e-8)
