"""Pins of the oracle's shape derivative and velocity: Taylor tests against the
moved-mesh cost, exact volume derivative, descent identity, special cases."""
import numpy as np
import pytest

from oracle import fem, shape, solvers, velocity
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads


def _bubble_theta(m, seed):
    """Smooth P1 field vanishing on the whole boundary of D (so no boundary data moves)."""
    d = m.dim
    t = workloads.smooth_field(m.coords, d, seed).reshape(-1, d)
    w = np.ones(m.num_nodes)
    for a in range(d):
        lo, hi = m.lo[a], m.hi[a]
        w *= (m.coords[:, a] - lo) * (hi - m.coords[:, a]) * 4 / (hi - lo) ** 2
    return (t * w[:, None]).reshape(-1)


def _heat_J(coords, cells, A, f_fun, dir_mask):
    vol, g = fem.geometry(coords, cells)
    K = fem.assemble(fem.scalar_stiffness(vol, g, A), cells.astype(np.int64), coords.shape[0])
    F = fem.body_load(coords, cells, f_fun(coords))
    F[dir_mask] = 0.0
    u = solvers.solve_free(K, F, ~dir_mask)
    return shape.heat_cost(vol, g, A, u, cells), u


def _elastic_J(coords, cells, A, lam, mu, F, dir_mask):
    vol, g = fem.geometry(coords, cells)
    K = fem.assemble(fem.elastic_stiffness(vol, g, A, lam, mu), fem.element_dofs(cells, coords.shape[1]),
                     coords.size)
    u = solvers.solve_free(K, F, ~dir_mask)
    return shape.elastic_cost(vol, g, A, u, cells, lam, mu), u


def _helm_J(coords, cells, A, k, om, f_fun, dir_mask):
    vol, g = fem.geometry(coords, cells)
    Ke = fem.scalar_stiffness(vol, g, A * k) + om * om * fem.mass(vol, coords.shape[1])
    K = fem.assemble(Ke, cells.astype(np.int64), coords.shape[0])
    F = fem.body_load(coords, cells, f_fun(coords))
    F[dir_mask] = 0.0
    u = solvers.solve_free(K, F, ~dir_mask)
    return float(F @ u), u


def _taylor(Jfun, theta, dJ, d):
    errs = []
    for t in (1e-2, 1e-3, 1e-4, 1e-5):
        fd = (Jfun(t) - Jfun(-t)) / (2 * t)
        errs.append(abs(fd - dJ) / abs(dJ))
    return errs


@pytest.mark.parametrize("dim", [2, 3])
def test_taylor_heat(dim):
    n = (12, 12) if dim == 2 else (5, 4, 4)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    phi = workloads.phi_bumps(m.coords, workloads.bump_centres((0,) * dim, (1,) * dim, 5, seed=3), 0.2, 0.5)
    A, chi = shape.coefficient(phi, m.cells, 1.0, 1e-2)
    gvec = np.array([0.5, -0.3, 0.2][:dim])

    def f_fun(X):
        return 1.0 + X @ gvec

    dir_mask = m.face_nodes(0, 0)
    J0, u = _heat_J(m.coords, m.cells, A, f_fun, dir_mask)
    b = shape.heat_rhs(m.coords, m.cells, A, u, f_fun(m.coords))
    theta = _bubble_theta(m, 11)
    dJ = b @ theta
    errs = _taylor(lambda t: _heat_J(m.coords + t * theta.reshape(-1, dim), m.cells, A, f_fun, dir_mask)[0],
                   theta, dJ, dim)
    assert errs[0] < 1e-2
    assert errs[1] < errs[0] / 50                      # second order in t
    assert min(errs) < 1e-7


@pytest.mark.parametrize("dim", [2, 3])
def test_taylor_elastic(dim):
    n = (12, 6) if dim == 2 else (6, 3, 3)
    hi = (2.0, 1.0) if dim == 2 else (2.0, 1.0, 1.0)
    m = BoxMesh(dim, n, (0,) * dim, hi)
    phi = workloads.phi_bumps(m.coords, workloads.bump_centres((0,) * dim, hi, 6, seed=4), 0.25, 0.4)
    A, chi = shape.coefficient(phi, m.cells, 1.0, 1e-2)
    lam, mu = fem.lame(1.0, 0.3)
    F = np.zeros(m.coords.size)
    corner = np.zeros(dim, dtype=np.int64)
    corner[0] = n[0]
    corner[1] = n[1] // 2
    F[dim * int(m.node_id(corner)) + 1] = -1.0
    dir_mask = np.repeat(m.face_nodes(0, 0), dim)
    J0, u = _elastic_J(m.coords, m.cells, A, lam, mu, F, dir_mask)
    b = shape.elastic_rhs(m.coords, m.cells, A, u, lam, mu)
    theta = _bubble_theta(m, 12)
    dJ = b @ theta
    errs = _taylor(lambda t: _elastic_J(m.coords + t * theta.reshape(-1, dim), m.cells, A, lam, mu, F,
                                        dir_mask)[0], theta, dJ, dim)
    assert errs[1] < errs[0] / 50
    assert min(errs) < 1e-7


def test_taylor_helmholtz():
    m = BoxMesh(2, (12, 12), (0, 0), (1, 1))
    phi = workloads.phi_cos(m.coords)
    A, chi = shape.coefficient(phi, m.cells, 1.0, 1e-2)
    k, om = 1.3, 2.5
    gvec = np.array([0.7, -0.4])

    def f_fun(X):
        return 0.5 + X @ gvec

    dir_mask = m.face_nodes(0, 0)
    J0, u = _helm_J(m.coords, m.cells, A, k, om, f_fun, dir_mask)
    b = shape.helmholtz_rhs(m.coords, m.cells, A, k, om, u, f_fun(m.coords))
    theta = _bubble_theta(m, 13)
    dJ = b @ theta
    errs = _taylor(lambda t: _helm_J(m.coords + t * theta.reshape(-1, 2), m.cells, A, k, om, f_fun, dir_mask)[0],
                   theta, dJ, 2)
    assert errs[1] < errs[0] / 50
    assert min(errs) < 1e-7


@pytest.mark.parametrize("dim", [2, 3])
def test_volume_derivative_exact(dim):
    n = (8, 8) if dim == 2 else (4, 4, 4)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    phi = workloads.phi_cos(m.coords)
    _, chi = shape.coefficient(phi, m.cells, 1.0, 1e-3)
    V = 0.4
    theta = workloads.smooth_field(m.coords, dim, 5)        # any P1 field: the identity is algebraic
    b = shape.volume_rhs(m.coords, m.cells, chi, V)

    def C(t):
        vol, _ = fem.geometry(m.coords + t * theta.reshape(-1, dim), m.cells)
        return shape.volume(vol, chi) / V

    t = 1e-3
    fd = (C(t) - C(-t)) / (2 * t)
    tol = 1e-10 if dim == 2 else 1e-5                       # vol(t) quadratic in 2D, cubic in 3D
    assert abs(fd - b @ theta) <= tol * abs(b @ theta)


def test_descent_identity_and_spd():
    m = BoxMesh(2, (10, 5), (0, 0), (2, 1))
    form = velocity.VelocityForm(alpha_mass=0.1, normal_penalty=1e4, omega0_weight=1e4,
                                 omega0_boxes=[((1.5, 0.4), (np.inf, 0.6))])
    b = workloads.random_field(2 * m.num_nodes, 7)
    theta, Btt = velocity.solve(m, form, b)
    assert Btt > 0
    assert abs(Btt - velocity.bilinear(m, form, theta)) < 1e-9 * Btt
    for a in range(2):
        ev = np.linalg.eigvalsh(velocity.component_matrix(m, form, a).toarray())
        assert ev.min() > 0
    # the normal penalty acts on theta_a only on the faces normal to e_a
    B0 = velocity.component_matrix(m, velocity.VelocityForm(alpha_mass=0.0, normal_penalty=1.0), 0)
    B0n = velocity.component_matrix(m, velocity.VelocityForm(alpha_mass=0.0, normal_penalty=0.0), 0)
    diff = (B0 - B0n).toarray()
    on = m.face_nodes(0, 0) | m.face_nodes(0, 1)
    assert np.all(diff[~on] == 0) and np.all(diff[:, ~on] == 0)
    assert abs(diff.sum() - 2.0) < 1e-13                    # two faces of length 1


def test_volume_only_h10_gives_zero_velocity():
    m = BoxMesh(2, (8, 8), (0, 0), (1, 1))
    chi = np.ones(m.num_elems)
    b = shape.volume_rhs(m.coords, m.cells, chi, 0.5)
    form = velocity.VelocityForm(alpha_mass=0.01, dirichlet=True)
    theta, Btt = velocity.solve(m, form, b)
    assert np.max(np.abs(theta)) < 1e-14
