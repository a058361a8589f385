"""Pins of the oracle's operators and state solves: textbook stencils, closed forms,
kernels, patch tests and manufactured-solution convergence rates."""
import math

import numpy as np
import pytest

from oracle import fem, shape, solvers
from oracle.algorithm import ELASTIC, HEAT, Problem
from oracle.mesh import BoxMesh


def _scalar_K(m, A=None):
    vol, g = fem.geometry(m.coords, m.cells)
    A = np.ones(m.num_elems) if A is None else A
    return fem.assemble(fem.scalar_stiffness(vol, g, A), m.cells.astype(np.int64), m.num_nodes)


def test_scalar_stiffness_is_five_point_stencil():
    # right isosceles Kuhn triangles: the diagonal couplings vanish and K is the 5-point Laplacian
    n = 8
    m = BoxMesh(2, (n, n), (0, 0), (1, 1))
    K = _scalar_K(m).toarray()
    idx = m.node_index
    for a in range(m.num_nodes):
        i, j = idx[a]
        if 0 < i < n and 0 < j < n:
            row = np.zeros(m.num_nodes)
            row[a] = 4.0
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                row[m.node_id(np.array([i + di, j + dj]))] = -1.0
            assert np.allclose(K[a], row, atol=1e-13)


def test_scalar_stiffness_rowsum_symmetry():
    m = BoxMesh(3, (3, 4, 2), (0, 0, 0), (1, 2, 1))
    rng = np.random.default_rng(0)
    A = np.where(rng.random(m.num_elems) < 0.5, 1.0, 1e-3)
    K = _scalar_K(m, A)
    assert np.max(np.abs(K @ np.ones(m.num_nodes))) < 1e-13
    assert abs(K - K.T).max() < 1e-15


def test_scalar_patch_test():
    # any linear u gives a zero residual at interior nodes (any mesh, any A constant)
    m = BoxMesh(3, (4, 3, 3), (0, 0, 0), (1, 1, 1))
    K = _scalar_K(m)
    u = 0.3 + 1.1 * m.coords[:, 0] - 0.7 * m.coords[:, 1] + 2.0 * m.coords[:, 2]
    r = K @ u
    inner = np.ones(m.num_nodes, dtype=bool)
    for a in range(3):
        inner &= ~(m.face_nodes(a, 0) | m.face_nodes(a, 1))
    assert np.max(np.abs(r[inner])) < 1e-12


def test_heat_1d_reduction_rates():
    # A = 1 everywhere, f = 1, u = 0 on x = 0, Neumann elsewhere: the continuous solution is
    # u = x - x^2/2 with J = int |grad u|^2 = 1/3.  On the Kuhn mesh the consistent load at the
    # two corners of x = 1 differs (h^2/3 vs h^2/6), so u_h is not y-independent and only
    # O(h^2) agreement holds at the nodes, while J_h keeps the 1D value 1/3 - h^2/12 (the
    # midpoint-rule error of int (1-x)^2) up to a higher-order corner term.
    errs, jerr = [], []
    for n in (16, 32, 64):
        m = BoxMesh(2, (n, n), (0, 0), (1, 1))
        prob = Problem(mesh=m, kind=HEAT, a_in=1.0, a_out=1e-3, dirichlet_faces=[(0, 0)],
                       f_nodal=np.ones(m.num_nodes))
        u, A, chi = prob.state(-np.ones(m.num_nodes))
        x = m.coords[:, 0]
        errs.append(np.max(np.abs(u - (x - 0.5 * x * x))))
        J = prob.cost(u, A)
        jerr.append(abs(J - (1.0 / 3.0 - 1.0 / (12.0 * n * n))))
        assert abs(J - prob.load() @ u) < 1e-13           # Galerkin identity J = F^T u
        assert np.all(chi == 1) and np.all(A == 1.0)
    for k in range(2):
        assert 3.2 < errs[k] / errs[k + 1] < 4.4
        assert jerr[k] / jerr[k + 1] > 8.0
    assert jerr[-1] < 5e-9


def _mms_errors(n):
    m = BoxMesh(2, (n, n), (0, 0), (1, 1))
    x, y = m.coords[:, 0], m.coords[:, 1]
    f = 2 * np.pi**2 * np.sin(np.pi * x) * np.sin(np.pi * y)
    faces = [(0, 0), (0, 1), (1, 0), (1, 1)]
    prob = Problem(mesh=m, kind=HEAT, a_in=1.0, dirichlet_faces=faces, f_nodal=f)
    u, _, _ = prob.state(-np.ones(m.num_nodes))
    vol, g = fem.geometry(m.coords, m.cells)
    from oracle.levelset import quadrature
    pts, wts = quadrature(2)
    X = m.coords[m.cells]
    gu = np.einsum("ea,eak->ek", u[m.cells], g)
    e_l2 = e_h1 = 0.0
    for lam, w in zip(pts, wts):
        xq = np.einsum("a,eak->ek", lam, X)
        ex = np.sin(np.pi * xq[:, 0]) * np.sin(np.pi * xq[:, 1])
        gx = np.stack([np.pi * np.cos(np.pi * xq[:, 0]) * np.sin(np.pi * xq[:, 1]),
                       np.pi * np.sin(np.pi * xq[:, 0]) * np.cos(np.pi * xq[:, 1])], axis=1)
        uq = u[m.cells] @ lam
        e_l2 += np.sum(w * vol * (uq - ex) ** 2)
        e_h1 += np.sum(w * vol * np.sum((gu - gx) ** 2, axis=1))
    return math.sqrt(e_l2), math.sqrt(e_h1)


def test_mms_convergence_rates():
    errs = [_mms_errors(n) for n in (8, 16, 32, 64)]
    l2 = [math.log2(errs[i][0] / errs[i + 1][0]) for i in range(3)]
    h1 = [math.log2(errs[i][1] / errs[i + 1][1]) for i in range(3)]
    assert abs(l2[-1] - 2.0) < 0.1 and abs(l2[-2] - 2.0) < 0.15
    assert abs(h1[-1] - 1.0) < 0.1


def _elastic_K(m, A=None, E=1.0, nu=0.3):
    vol, g = fem.geometry(m.coords, m.cells)
    A = np.ones(m.num_elems) if A is None else A
    lam, mu = fem.lame(E, nu)
    Ke = fem.elastic_stiffness(vol, g, A, lam, mu)
    return fem.assemble(Ke, fem.element_dofs(m.cells, m.dim), m.dim * m.num_nodes)


@pytest.mark.parametrize("dim", [2, 3])
def test_elastic_rigid_modes_and_symmetry(dim):
    n = (3, 2) if dim == 2 else (2, 2, 2)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    rng = np.random.default_rng(1)
    A = np.where(rng.random(m.num_elems) < 0.5, 1.0, 1e-3)
    K = _elastic_K(m, A)
    X = m.coords
    modes = []
    for c in range(dim):
        t = np.zeros((m.num_nodes, dim))
        t[:, c] = 1.0
        modes.append(t)
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (0, 2)]
    for a, b in pairs:
        r = np.zeros((m.num_nodes, dim))
        r[:, a], r[:, b] = -X[:, b], X[:, a]
        modes.append(r)
    for r in modes:
        assert np.max(np.abs(K @ r.reshape(-1))) < 1e-12
    assert abs(K - K.T).max() < 1e-14
    # the Neumann kernel has exactly 3 (2D) / 6 (3D) rigid modes
    ev = np.linalg.eigvalsh(K.toarray())
    assert np.sum(ev < 1e-10) == len(modes)


def test_elastic_patch_and_galerkin_identity():
    m = BoxMesh(2, (8, 4), (0, 0), (2, 1))
    K = _elastic_K(m)
    Xc = m.coords
    u = np.stack([0.1 + 0.3 * Xc[:, 0] - 0.2 * Xc[:, 1], -0.4 + 0.5 * Xc[:, 0] + 0.7 * Xc[:, 1]], axis=1)
    r = (K @ u.reshape(-1)).reshape(-1, 2)
    inner = ~(m.face_nodes(0, 0) | m.face_nodes(0, 1) | m.face_nodes(1, 0) | m.face_nodes(1, 1))
    assert np.max(np.abs(r[inner])) < 1e-12
    # Galerkin identity J = int A sigma(u):eps(u) = F^T u for the compliance problem
    prob = Problem(mesh=m, kind=ELASTIC, dirichlet_faces=[(0, 0)], point_loads=[(m.node_id(np.array([8, 2])), (0.0, -1.0))])
    phi = np.cos(3 * m.coords[:, 0]) * np.cos(5 * m.coords[:, 1]) + 0.2
    u, A, _ = prob.state(phi)
    assert abs(prob.cost(u, A) - prob.load() @ u) < 1e-10 * abs(prob.load() @ u)


def test_elastic_mms_rate():
    # manufactured body force for u = (sin(pi x) sin(pi y), 0) with all-Dirichlet data, plane strain
    lam, mu = fem.lame(1.0, 0.3)

    def err(n):
        m = BoxMesh(2, (n, n), (0, 0), (1, 1))
        x, y = m.coords[:, 0], m.coords[:, 1]
        s, c, pi = np.sin, np.cos, np.pi
        # f = -div sigma(u): for u1 = sin sin, u2 = 0
        f1 = (lam + 2 * mu) * pi**2 * s(pi * x) * s(pi * y) + mu * pi**2 * s(pi * x) * s(pi * y)
        f2 = -(lam + mu) * pi**2 * c(pi * x) * c(pi * y)
        K = _elastic_K(m)
        vol, _ = fem.geometry(m.coords, m.cells)
        Me = fem.mass(vol, 2)
        F = np.zeros(2 * m.num_nodes)
        for comp, f in ((0, f1), (1, f2)):
            Fe = np.einsum("eab,eb->ea", Me, f[m.cells])
            np.add.at(F, 2 * m.cells.astype(np.int64).ravel() + comp, Fe.ravel())
        mask = m.dirichlet_mask([(0, 0), (0, 1), (1, 0), (1, 1)], 2)
        F[mask == 1] = 0.0
        uh = solvers.solve_free(K, F, mask == 0).reshape(-1, 2)
        ex = np.stack([s(pi * x) * s(pi * y), 0 * x], axis=1)
        e = (uh - ex).reshape(-1)
        M = fem.assemble(np.einsum("eab,ij->eaibj", Me, np.eye(2)).reshape(-1, 6, 6),
                         fem.element_dofs(m.cells, 2), 2 * m.num_nodes)
        return math.sqrt(e @ (M @ e))

    e1, e2, e3 = err(8), err(16), err(32)
    assert abs(math.log2(e2 / e3) - 2.0) < 0.15


def test_pcg_matches_direct():
    m = BoxMesh(2, (16, 16), (0, 0), (1, 1))
    phi = np.cos(4 * np.pi * m.coords[:, 0]) * np.cos(4 * np.pi * m.coords[:, 1]) + 0.3
    prob = Problem(mesh=m, kind=HEAT, dirichlet_faces=[(0, 0)], f_nodal=np.ones(m.num_nodes))
    A, _ = shape.coefficient(phi, m.cells, 1.0, 1e-3)
    K = prob.stiffness(A)
    F = prob.load()
    free = prob.dirichlet() == 0
    u = solvers.solve_free(K, F, free)
    idx = np.flatnonzero(free)
    x, it, rel = solvers.jacobi_pcg(K[idx][:, idx], F[idx], rtol=1e-13)
    assert rel <= 1e-13 and it > 10
    assert np.linalg.norm(x - u[idx]) <= 1e-9 * np.linalg.norm(u)
    y, it2, rel2 = solvers.jacobi_bicgstab(K[idx][:, idx], F[idx], rtol=1e-13)
    assert np.linalg.norm(y - u[idx]) <= 1e-9 * np.linalg.norm(u)


def test_coefficient_rule_and_tie():
    cells = np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int32)
    phi = np.array([-1.0, 0.5, 0.5, 0.0])
    A, chi = shape.coefficient(phi, cells, 1.0, 1e-3)
    assert list(chi) == [0, 0]          # (-1 + 0.5) + 0.5 == 0 -> outside (strict)
    phi[0] = -1.0 - 2**-40
    A, chi = shape.coefficient(phi, cells, 1.0, 1e-3)
    assert list(chi) == [1, 0] and A[0] == 1.0 and A[1] == 1e-3
