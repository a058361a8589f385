"""Pins of the oracle's logistic population model (Sec. 6.4): the cubic integrals against a
collapsed-coordinate Gauss product rule, the residual against per-element quadrature, the
Jacobian against central differences of the residual, constant equilibria in closed form,
quadratic Newton convergence, the adjoint against a finite-difference source derivative and
the shape derivative against the moved-mesh cost (Taylor test)."""
import math

import numpy as np
import pytest

from oracle import fem, logistic, shape
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads


def _collapsed_rule(d, n=4):
    """Gauss-Legendre product rule on the unit square / cube mapped onto the reference simplex
    (Duffy collapse); exact for polynomials of degree <= 2n - 1 - (d - 1) on the simplex.
    Returns barycentric points [Q, d+1] and weights summing to 1 / d!."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    pts, wts = [], []
    if d == 2:
        for xi, wi in zip(x, w):
            for eta, we in zip(x, w):
                p = np.array([xi, (1 - xi) * eta])
                pts.append(p)
                wts.append(wi * we * (1 - xi))
    else:
        for xi, wi in zip(x, w):
            for eta, we in zip(x, w):
                for ze, wz in zip(x, w):
                    p = np.array([xi, (1 - xi) * eta, (1 - xi) * (1 - eta) * ze])
                    pts.append(p)
                    wts.append(wi * we * wz * (1 - xi) ** 2 * (1 - eta))
    P = np.array(pts)
    bary = np.hstack([1.0 - P.sum(axis=1, keepdims=True), P])
    return bary, np.array(wts)


@pytest.mark.parametrize("d", [2, 3])
def test_cubic_tensor_against_quadrature(d):
    bary, w = _collapsed_rule(d)
    assert abs(w.sum() - 1.0 / math.factorial(d)) < 1e-15
    ref = np.einsum("q,qa,qb,qc->abc", w, bary, bary, bary) * math.factorial(d)
    assert np.max(np.abs(logistic.cubic_tensor(d) - ref)) < 1e-15
    # the sum rule over one index gives the consistent mass
    M = fem.mass(np.ones(1), d)[0]
    assert np.allclose(logistic.cubic_tensor(d).sum(axis=2), M, atol=1e-16)


def _jittered(dim, n, seed):
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    rng = np.random.default_rng(seed)
    X = m.coords.copy()
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    X[interior] += 0.2 / max(n) * (rng.random((interior.sum(), dim)) - 0.5)
    return m, X


@pytest.mark.parametrize("d", [2, 3])
def test_residual_against_pointwise_quadrature(d):
    """F(u)_a assembled from per-element integrals evaluated at the collapsed-rule points."""
    m, X = _jittered(d, (4, 3) if d == 2 else (2, 2, 2), 3)
    rng = np.random.default_rng(5)
    u = 0.5 + rng.random(m.num_nodes)
    K = np.where(rng.random(m.num_elems) < 0.5, 1.0, 1e-2)
    r = 7.0
    F = logistic.residual(X, m.cells, K, r, u)
    vol, g = fem.geometry(X, m.cells)
    bary, w = _collapsed_rule(d)
    ref = np.zeros(m.num_nodes)
    for e, cell in enumerate(m.cells):
        ue = u[cell]
        gu = g[e].T @ ue
        for a in range(d + 1):
            uq = bary @ ue
            react = np.sum(w * r * uq * (1 - uq / K[e]) * bary[:, a]) * math.factorial(d) * vol[e]
            ref[cell[a]] += vol[e] * gu @ g[e, a] - react
    assert np.max(np.abs(F - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("d", [2, 3])
def test_jacobian_is_derivative_of_residual(d):
    m, X = _jittered(d, (5, 4) if d == 2 else (3, 2, 2), 4)
    rng = np.random.default_rng(6)
    u = 0.3 + rng.random(m.num_nodes)
    v = rng.standard_normal(m.num_nodes)
    K = np.where(rng.random(m.num_elems) < 0.5, 1.0, 1e-2)
    r = 40.0
    Jv = logistic.jacobian(X, m.cells, K, r, u) @ v
    errs = []
    for t in (1e-2, 1e-3):
        fd = (logistic.residual(X, m.cells, K, r, u + t * v) - logistic.residual(X, m.cells, K, r, u - t * v)) / (2 * t)
        errs.append(np.max(np.abs(fd - Jv)) / np.max(np.abs(Jv)))
    # the residual is quadratic in u, so the central difference is exact up to rounding
    assert max(errs) < 1e-9, errs
    # symmetric (the adjoint uses DF itself)
    Jm = logistic.jacobian(X, m.cells, K, r, u)
    assert abs(Jm - Jm.T).max() < 1e-13 * abs(Jm).max()


@pytest.mark.parametrize("kin,inside", [(1.0, True), (1e-2, False)])
def test_constant_equilibrium(kin, inside):
    """With K constant the discrete problem has the exact root u = K (grad u = 0, 1 - u/K = 0);
    Newton from the paper's initial guess reaches it."""
    m = BoxMesh(2, (16, 16), (0, 0), (1, 1))
    phi = -np.ones(m.num_nodes) if inside else np.ones(m.num_nodes)
    K, chi = logistic.carrying_capacity(phi, m.cells)
    assert np.all(K == kin)
    u0 = workloads.u0_logistic(m.coords) * (1.0 if inside else 1e-2)
    u, hist = logistic.newton(m.coords, m.cells, K, 10.0, u0)
    assert np.max(np.abs(u - kin)) < 1e-13 * kin, np.max(np.abs(u - kin))
    assert np.max(np.abs(logistic.residual(m.coords, m.cells, K, 10.0, np.full(m.num_nodes, kin)))) < 1e-16


def test_newton_converges_quadratically():
    m = BoxMesh(2, (24, 24), (0, 0), (1, 1))
    phi = workloads.phi_cos(m.coords)
    K, _ = logistic.carrying_capacity(phi, m.cells)
    u, hist = logistic.newton(m.coords, m.cells, K, 40.0, workloads.u0_logistic(m.coords))
    assert hist[-1] <= 1e-13 * hist[0]
    # once in the basin, each error is about the square of the previous one
    ratios = [hist[k + 1] / hist[k] ** 2 for k in range(len(hist) - 1) if hist[k] < 1e-2 * hist[0] and hist[k + 1] > 1e-14]
    assert ratios and max(ratios) < 1e4 / hist[0], (hist, ratios)
    assert np.all(u > 0)


def test_adjoint_is_source_derivative():
    """dJ/de of F(u) = e M g at e = 0 equals -p . (M g)  (J = -int u, DF p = int psi)."""
    m = BoxMesh(2, (12, 10), (0, 0), (1, 1))
    phi = workloads.phi_cos(m.coords)
    K, _ = logistic.carrying_capacity(phi, m.cells)
    r = 10.0
    u0 = workloads.u0_logistic(m.coords)
    u, _ = logistic.newton(m.coords, m.cells, K, r, u0)
    p = logistic.adjoint(m.coords, m.cells, K, r, u)
    g = fem.body_load(m.coords, m.cells, np.sin(3 * m.coords[:, 0]) + m.coords[:, 1])
    dJ = -p @ g
    t = 1e-5
    Jp = logistic.cost(m.coords, m.cells, logistic.newton(m.coords, m.cells, K, r, u, extra=t * g)[0])
    Jm = logistic.cost(m.coords, m.cells, logistic.newton(m.coords, m.cells, K, r, u, extra=-t * g)[0])
    assert abs((Jp - Jm) / (2 * t) - dJ) <= 1e-7 * abs(dJ)


def test_cost_closed_form():
    m = BoxMesh(3, (3, 2, 2), (0, 0, 0), (2, 1, 1))
    u = 1.0 + 0.5 * m.coords[:, 0] - m.coords[:, 2]              # linear: int u = |D| u(centre)
    assert abs(logistic.cost(m.coords, m.cells, u) + 2.0 * (1.0 + 0.5 - 0.5)) < 1e-14


def _bubble_theta(m, seed):
    d = m.dim
    t = workloads.smooth_field(m.coords, d, seed).reshape(-1, d)
    w = np.ones(m.num_nodes)
    for a in range(d):
        w *= m.coords[:, a] * (1 - m.coords[:, a]) * 4
    return (t * w[:, None]).reshape(-1)


@pytest.mark.parametrize("dim", [2, 3])
def test_taylor_shape_derivative(dim):
    """Central differences of J(Omega_t) on the mesh moved by t theta (K carried with the
    elements) converge to b . theta at second order."""
    n = (10, 10) if dim == 2 else (4, 4, 3)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    phi = workloads.phi_bumps(m.coords, workloads.bump_centres((0,) * dim, (1,) * dim, 4, seed=2), 0.25, 0.4)
    K, chi = logistic.carrying_capacity(phi, m.cells)
    r = 10.0
    u0 = workloads.u0_logistic(m.coords)
    u, _ = logistic.newton(m.coords, m.cells, K, r, u0)
    p = logistic.adjoint(m.coords, m.cells, K, r, u)
    b = logistic.rhs(m.coords, m.cells, K, r, u, p)
    theta = _bubble_theta(m, 9)
    dJ = b @ theta

    def J(t):
        X = m.coords + t * theta.reshape(-1, dim)
        return logistic.cost(X, m.cells, logistic.newton(X, m.cells, K, r, u)[0])

    errs = [abs((J(t) - J(-t)) / (2 * t) - dJ) / abs(dJ) for t in (1e-2, 1e-3, 1e-4, 1e-5)]
    assert errs[1] < errs[0] / 50 or errs[1] < 1e-8, errs
    assert min(errs) < 1e-7, errs
    # the volume term: lam S1^C gives lam d|Omega|/V exactly
    lam, V = 0.7, 0.5
    bl = logistic.rhs(m.coords, m.cells, K, r, u, p, lam, chi.astype(np.float64), V) - b
    vol_t = lambda t: shape.volume(fem.geometry(m.coords + t * theta.reshape(-1, dim), m.cells)[0], chi)
    fd = (vol_t(1e-6) - vol_t(-1e-6)) / 2e-6
    assert abs(bl @ theta - lam * fd / V) < 1e-8 * max(1.0, abs(lam * fd / V))
