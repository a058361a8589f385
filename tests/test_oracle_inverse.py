"""Pins of the oracle's inverse-elasticity model (Sec. 3, Sec. 6.1): Taylor tests of the shape
derivative against the moved-mesh cost (2D, 3D), the zero of the cost and of its derivative at
the true inclusion, finite-difference checks of both adjoints through the traction and the
extended measurement, and the Dirichlet extension's patch test."""
import numpy as np
import pytest

from oracle import fem, inverse, shape
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads

LAM, MU = fem.lame(1.0, 0.3)
ALPHA, BETA = 3.0, 2.0


def _setup(dim, n):
    m = BoxMesh(dim, n, (0.0,) * dim, (1.0,) * dim)
    faces0 = [(0, 0)]
    faces1 = [(a, s) for a in range(dim) for s in (0, 1) if (a, s) != (0, 0)]
    dir0 = m.dirichlet_mask(faces0, dim)
    t = np.array([0.3, -1.0, 0.2][:dim])
    F = fem.facet_load(m.coords, m.boundary_facets(0, 1), t, dim)
    F[dir0 == 1] = 0.0
    Mg = inverse.facet_vector_mass(m.coords, inverse.gamma_facets(m, faces1))
    return m, dir0, F, Mg


def _phi(m, seed):
    return workloads.phi_bumps(m.coords, workloads.bump_centres((0.2,) * m.dim, (0.8,) * m.dim, 3, seed), 0.15, 0.5)


def _J(coords, m, A, F, g, dir0, Mg):
    K = inverse.elastic_matrix(coords, m.cells, A, LAM, MU)
    M = inverse.vector_mass(coords, m.cells)
    u, v = inverse.states(m, K, F, g, dir0)
    return inverse.cost(M, Mg, u, v, g, ALPHA, BETA), (K, M, u, v)


def _bubble(m, seed):
    d = m.dim
    t = workloads.smooth_field(m.coords, d, seed).reshape(-1, d)
    w = np.ones(m.num_nodes)
    for a in range(d):
        w *= m.coords[:, a] * (1 - m.coords[:, a]) * 4
    return (t * w[:, None]).reshape(-1)


@pytest.mark.parametrize("dim", [2, 3])
def test_taylor_shape_derivative(dim):
    m, dir0, F, Mg = _setup(dim, (10, 8) if dim == 2 else (4, 4, 3))
    A, _ = shape.coefficient(_phi(m, 1), m.cells, 10.0, 1.0)
    rng = np.random.default_rng(3)
    G, c0 = rng.standard_normal((dim, dim)) * 0.3, rng.standard_normal(dim) * 0.1

    def g_at(X):                       # a linear measurement field: exact in P1, evaluated at moved nodes
        return (X @ G.T + c0).reshape(-1)

    J0, (K, M, u, v) = _J(m.coords, m, A, F, g_at(m.coords), dir0, Mg)
    g = g_at(m.coords)
    p, q = inverse.adjoints(m, K, M, Mg, u, v, g, ALPHA, BETA, dir0)
    b = inverse.rhs(m.coords, m.cells, A, LAM, MU, u, v, p, q, g, ALPHA)
    theta = _bubble(m, 5)
    dJ = b @ theta

    def J(t):
        X = m.coords + t * theta.reshape(-1, dim)
        return _J(X, m, A, F, g_at(X), dir0, Mg)[0]

    errs = [abs((J(t) - J(-t)) / (2 * t) - dJ) / abs(dJ) for t in (1e-2, 1e-3, 1e-4, 1e-5)]
    assert errs[1] < errs[0] / 50 or errs[1] < 1e-8, errs
    assert min(errs) < 1e-7, errs


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_at_the_true_inclusion(dim):
    """With the measurement generated at the true inclusion (g = its displacement), the cost,
    the second state, both adjoints and the shape derivative vanish there."""
    m, dir0, F, Mg = _setup(dim, (12, 10) if dim == 2 else (5, 4, 4))
    A, _ = shape.coefficient(_phi(m, 2), m.cells, 10.0, 1.0)
    K = inverse.elastic_matrix(m.coords, m.cells, A, LAM, MU)
    g = inverse.states(m, K, F, np.zeros(m.coords.size), dir0)[0]
    J, (K, M, u, v) = _J(m.coords, m, A, F, g, dir0, Mg)
    scale = float(g @ (M @ g))
    assert J <= 1e-24 * max(scale, 1.0), J
    assert np.max(np.abs(v)) <= 1e-12 * np.max(np.abs(g))
    p, q = inverse.adjoints(m, K, M, Mg, u, v, g, ALPHA, BETA, dir0)
    assert np.max(np.abs(p)) <= 1e-12 and np.max(np.abs(q)) <= 1e-12
    b = inverse.rhs(m.coords, m.cells, A, LAM, MU, u, v, p, q, g, ALPHA)
    assert np.max(np.abs(b)) <= 1e-12
    # and a different inclusion gives a positive cost
    A2, _ = shape.coefficient(_phi(m, 7), m.cells, 10.0, 1.0)
    assert _J(m.coords, m, A2, F, g, dir0, Mg)[0] > 1e-8 * max(scale, 1.0)


def test_adjoints_by_finite_differences():
    """dJ/dF(dF) = -p . dF; dJ/dg(dg) = -alpha w.M dg - beta (u - g).M_G1 dg + dg.K q (w = u - v - g)."""
    m, dir0, F, Mg = _setup(2, (10, 9))
    A, _ = shape.coefficient(_phi(m, 4), m.cells, 10.0, 1.0)
    rng = np.random.default_rng(8)
    g = workloads.smooth_field(m.coords, 2, 6) * 0.5
    J0, (K, M, u, v) = _J(m.coords, m, A, F, g, dir0, Mg)
    p, q = inverse.adjoints(m, K, M, Mg, u, v, g, ALPHA, BETA, dir0)
    dF = rng.standard_normal(F.size)
    dF[dir0 == 1] = 0.0
    t = 1e-6
    fd = (_J(m.coords, m, A, F + t * dF, g, dir0, Mg)[0] - _J(m.coords, m, A, F - t * dF, g, dir0, Mg)[0]) / (2 * t)
    assert abs(fd - (-p @ dF)) <= 1e-7 * abs(p @ dF)
    dg = workloads.smooth_field(m.coords, 2, 9)
    w = u - v - g
    pred = -ALPHA * (w @ (M @ dg)) - BETA * ((u - g) @ (Mg @ dg)) + dg @ (K @ q)
    fd = (_J(m.coords, m, A, F, g + t * dg, dir0, Mg)[0] - _J(m.coords, m, A, F, g - t * dg, dir0, Mg)[0]) / (2 * t)
    assert abs(fd - pred) <= 1e-7 * abs(pred)


@pytest.mark.parametrize("dim", [2, 3])
def test_dirichlet_extension_patch(dim):
    """Linear boundary data extend to the linear field (P1 reproduces harmonic linears); the
    extension keeps the given values on its faces."""
    m = BoxMesh(dim, (7, 5) if dim == 2 else (4, 3, 3), (0.0,) * dim, (1.0,) * dim)
    rng = np.random.default_rng(2)
    G = rng.standard_normal((dim, dim))
    lin = (m.coords @ G.T).reshape(-1)
    faces = [(a, s) for a in range(dim) for s in (0, 1)]
    eta = inverse.dirichlet_extension(m, lin, faces)
    assert np.max(np.abs(eta - lin)) < 1e-12
    vals = workloads.smooth_field(m.coords, dim, 4)
    eta = inverse.dirichlet_extension(m, vals, [(0, 1), (1, 0)])
    on = (m.face_nodes(0, 1) | m.face_nodes(1, 0))
    assert np.array_equal(eta.reshape(-1, dim)[on], vals.reshape(-1, dim)[on])
