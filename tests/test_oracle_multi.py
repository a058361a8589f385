"""Pins of the oracle's several-load-case compliance (eq. compli_plus), several volume
constraints (Sec. 5.4 with N_c > 1) and stopping criterion (Sec. 5.7): the parallelogram law
of compliance, a Taylor test of the summed cost against the moved mesh, the exact derivative
of a region's volume, the regions' volumes adding up to |Omega|, and hand-made histories."""
import numpy as np
import pytest

from oracle import algorithm as oalg, fem, ppl, shape
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads


def _mesh_phi():
    m = BoxMesh(2, (16, 8), (0.0, 0.0), (2.0, 1.0))
    phi = workloads.phi_bumps(m.coords, workloads.bump_centres((0, 0), (2, 1), 6, seed=4), 0.15, 0.5)
    return m, phi


def _elastic(m, cases, **kw):
    return oalg.Problem(mesh=m, kind=oalg.ELASTIC, dirichlet_faces=[(0, 0)], load_cases=cases, **kw)


def test_parallelogram_law_of_compliance():
    m, phi = _mesh_phi()
    tip, top = int(m.node_id(np.array([16, 4]))), int(m.node_id(np.array([10, 8])))
    g1 = [(tip, (0.0, -1.0))]
    g2 = [(top, (0.3, -0.5))]
    two = _elastic(m, [(g1, []), (g2, [])])
    U, A, _ = two.states(phi)
    J12 = two.total_cost(U, A)

    def single(pts):
        p = _elastic(m, [(pts, [])])
        Us, As, _ = p.states(phi)
        return p.total_cost(Us, As)
    Jp = single(g1 + g2)
    Jm = single(g1 + [(top, (-0.3, 0.5))])
    assert abs((Jp + Jm) - 2.0 * J12) <= 1e-11 * abs(J12)
    assert abs(J12 - (single(g1) + single(g2))) <= 1e-13 * abs(J12)


def test_taylor_of_summed_compliance():
    m, phi = _mesh_phi()
    A, chi = shape.coefficient(phi, m.cells, 1.0, 1e-2)
    tip = int(m.node_id(np.array([16, 4])))
    cases = [([(tip, (0.0, -1.0))], []), ([], [(1, 1, (0.2, -0.4))])]
    prob = _elastic(m, cases, a_out=1e-2)
    U, _, _ = prob.states(phi)
    b = prob.total_rhs(U, A, chi, [])
    # a velocity vanishing on the whole boundary moves no load or support
    d = 2
    t0 = workloads.smooth_field(m.coords, d, 5).reshape(-1, d)
    w = (m.coords[:, 0] * (2 - m.coords[:, 0])) * (m.coords[:, 1] * (1 - m.coords[:, 1]))
    theta = (t0 * w[:, None]).reshape(-1)
    dJ = b @ theta
    lam_e, mu_e = fem.lame(1.0, 0.3)

    def J_at(t):
        X = m.coords + t * theta.reshape(-1, d)
        mm = oalg.BoxMesh(2, (16, 8), (0.0, 0.0), (2.0, 1.0))
        mm.coords = X
        p = _elastic(mm, cases, a_out=1e-2)
        vol, g = fem.geometry(X, m.cells)
        K = fem.assemble(fem.elastic_stiffness(vol, g, A, lam_e, mu_e), fem.element_dofs(m.cells, 2), X.size)
        free = p.dirichlet() == 0
        from oracle import solvers
        tot = 0.0
        for k in range(2):
            u = solvers.solve_free(K, p.case_load(k), free)
            tot += shape.elastic_cost(vol, g, A, u, m.cells, lam_e, mu_e)
        return tot
    errs = [abs((J_at(t) - J_at(-t)) / (2 * t) - dJ) / abs(dJ) for t in (1e-2, 1e-3, 1e-4)]
    assert errs[1] < errs[0] / 50 and min(errs) < 1e-7, errs


def test_region_constraints_volume_and_exact_derivative():
    m, phi = _mesh_phi()
    regions = [((-np.inf, -np.inf), (1.0, np.inf), 0.4), ((1.0, -np.inf), (np.inf, np.inf), 0.6)]
    prob = _elastic(m, None, volume_regions=regions, volume_target=1.0)
    A, chi = shape.coefficient(phi, m.cells, 1.0, 1e-3)
    C = prob.constraints(chi)
    vol, _ = fem.geometry(m.coords, m.cells)
    total = shape.volume(vol, chi)
    # the two regions partition D (no centroid lies on x = 1): their volumes add up to |Omega|
    assert abs(C[0] * 0.4 + C[1] * 0.6 - total) <= 1e-14 * total
    # exact derivative of region 1's volume: chi and the region flags move with the elements
    r = m.subdomain_mask([regions[1][:2]]).astype(float)
    b = shape.volume_rhs(m.coords, m.cells, chi * r, 0.6)
    theta = workloads.smooth_field(m.coords, 2, 9)
    dV = b @ theta

    def V_at(t):
        vt, _ = fem.geometry(m.coords + t * theta.reshape(-1, 2), m.cells)
        return np.sum(chi * r * vt) / 0.6
    fd = (V_at(1e-3) - V_at(-1e-3)) / 2e-3                 # the measure is quadratic in t in 2D
    assert abs(fd - dV) <= 1e-12 * abs(dV)


def test_total_rhs_adds_each_constraint_with_its_multiplier():
    m, phi = _mesh_phi()
    regions = [((-np.inf, -np.inf), (1.0, np.inf), 0.4), ((1.0, -np.inf), (np.inf, np.inf), 0.6)]
    tip = int(m.node_id(np.array([16, 4])))
    prob = _elastic(m, [([(tip, (0.0, -1.0))], [])], volume_regions=regions, volume_target=1.0)
    U, A, chi = prob.states(phi)
    b0 = prob.total_rhs(U, A, chi, [0.0, 0.0])
    b1 = prob.total_rhs(U, A, chi, [0.7, -0.2])
    for (lo, hi, V), lam in zip(regions, [0.7, -0.2]):
        r = m.subdomain_mask([(lo, hi)]).astype(float)
        b0 = b0 + lam * shape.volume_rhs(m.coords, m.cells, chi * r, V)
    assert np.max(np.abs(b1 - b0)) <= 1e-13 * np.max(np.abs(b1))


def test_stop_check_hand_histories():
    flat = [10.0] * 25 + [1.0 + 1e-4 * k for k in range(20)]          # i = 44
    assert ppl.stop_check(flat, start_to_check=30)
    assert not ppl.stop_check(flat[:31], start_to_check=30)            # i = 30 is not > 30
    moving = [1.0 + 0.05 * k for k in range(45)]                       # 10 steps back differ by ~25 %
    assert not ppl.stop_check(moving, start_to_check=30)
    assert ppl.stop_check(flat, C=[1.005, 0.996], start_to_check=30)
    assert not ppl.stop_check(flat, C=[1.02], start_to_check=30)       # constraint error 2e-2
    # the spread is taken over exactly the previous `prev` values
    h = [5.0] * 40 + [1.0] * 11
    assert ppl.stop_check(h, start_to_check=30, prev=10)
    assert not ppl.stop_check(h, start_to_check=30, prev=11)
