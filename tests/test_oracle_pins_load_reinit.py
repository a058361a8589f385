"""Pins of the traction load (eq. compli_weak, the boundary term int_{Gamma_1} g . v) and of
one step of the reinitialisation scheme (Sec. 5.7, eqs Eikonal, HJ, grad_H, weak_HJ).

Traction: for P1 functions int_f psi_a = |f| / d on a facet with d vertices (barycentric
moment), so a constant traction t gives t |f| / d at each vertex of each facet; over a whole
face the load sums to t |Gamma| and its first moments are t int_Gamma x (a P1 interpolant of
a linear function is exact).  The checks below use hand-computed facets, quadrature by
subdivision and the face's own area / centroid, never the oracle's formula.

Reinitialisation: (1) from a constant level set the step is the L2 projection of
phi + dt S(phi0), i.e. exactly c + dt c / sqrt(c^2 + h^2) (and c + 2 dt S(c) after the
AB2 step); (2) with phi(t - dt) = phi(t) the AB2 step equals the explicit Euler step
(G(u, u, w) = -H(grad u) w - h^2 grad u . grad w); (3) brute force: one Euler step and
one AB2 step on a 3 x 3 mesh assembled densely from a pointwise evaluation of the paper's
definitions, with grad psi^ taken by central finite differences of psi^ itself (so the
derivative of tau S along grad phi0 is included without writing it out).
"""
import math

import numpy as np
import pytest

from oracle import fem, levelset
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads


# --------------------------------------------------------------------- traction load
def test_facet_load_single_facets_hand_values():
    # 2D: one segment of length 5 ((0,0)-(3,4)); t = (2, -1): each end gets t * 5 / 2
    coords = np.array([[0.0, 0.0], [3.0, 4.0], [9.0, 9.0]])
    F = fem.facet_load(coords, np.array([[0, 1]]), (2.0, -1.0), 2)
    assert np.allclose(F.reshape(-1, 2), [[5.0, -2.5], [5.0, -2.5], [0.0, 0.0]], rtol=0, atol=1e-15)
    # 3D: right triangle with legs 2 and 3 in the plane z = 0 (area 3); t = (0, 0, -1):
    # each vertex gets -1 (= -3 / 3), not -1.5 (a /2 in 3D) or -3
    coords = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 3.0, 0.0], [5.0, 5.0, 5.0]])
    F = fem.facet_load(coords, np.array([[0, 1, 2]]), (0.0, 0.0, -1.0), 3).reshape(-1, 3)
    assert np.allclose(F[:3], [[0, 0, -1.0]] * 3, rtol=0, atol=1e-15) and np.all(F[3] == 0)
    # scalar field (ncomp = 1) on the same triangle, t = 5: 5 * 3 / 3 = 5 per vertex
    F1 = fem.facet_load(coords, np.array([[0, 1, 2]]), (5.0,), 1)
    assert np.allclose(F1, [5.0, 5.0, 5.0, 0.0], rtol=0, atol=1e-15)


def _subdivided_moment(X, a, levels=6):
    """int_f psi_a over a triangle by midpoint subdivision (exact for the linear psi_a)."""
    # barycentric coordinates of the sub-triangle centroids of a uniform 4^levels split
    n = 2 ** levels
    tot = 0.0
    area = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
    for i in range(n):
        for j in range(n - i):
            for up in (0, 1):
                if up and i + j == n - 1:
                    continue
                if not up:
                    pts = np.array([[i, j], [i + 1, j], [i, j + 1]], dtype=float)
                else:
                    pts = np.array([[i + 1, j], [i, j + 1], [i + 1, j + 1]], dtype=float)
                c = pts.mean(axis=0) / n                    # (l1, l2) of the centroid
                lam = np.array([1.0 - c.sum(), c[0], c[1]])
                tot += lam[a] * area / n**2
    return tot


def test_facet_load_matches_subdivision_quadrature():
    rng = np.random.default_rng(5)
    X = rng.random((3, 3))
    t = np.array([0.3, -1.2, 0.7])
    F = fem.facet_load(X, np.array([[0, 1, 2]]), t, 3).reshape(3, 3)
    for a in range(3):
        assert np.allclose(F[a], t * _subdivided_moment(X, a), rtol=1e-12, atol=0)


@pytest.mark.parametrize("dim,n,hi", [(2, (6, 5), (2.0, 1.0)), (3, (4, 3, 5), (2.0, 1.0, 1.5))])
def test_facet_load_face_sums_and_moments(dim, n, hi):
    m = BoxMesh(dim, n, (0.0,) * dim, hi)
    t = np.array([0.4, -1.0, 0.25][:dim])
    for axis in range(dim):
        for side in (0, 1):
            F = fem.facet_load(m.coords, m.boundary_facets(axis, side), t, dim).reshape(-1, dim)
            others = [hi[b] for b in range(dim) if b != axis]
            area = float(np.prod(others))                            # |Gamma|
            assert np.allclose(F.sum(axis=0), t * area, rtol=1e-13, atol=0)
            # first moments: sum_a F_a x_a = t int_Gamma x = t |Gamma| (face centroid)
            centroid = np.array([hi[b] / 2 if b != axis else (hi[b] if side else 0.0) for b in range(dim)])
            mom = F.T @ m.coords                                     # [comp, coord]
            assert np.allclose(mom, np.outer(t, centroid * area), rtol=1e-12, atol=1e-14)
            on = m.face_nodes(axis, side)
            assert np.all(F[~on] == 0.0)


# ------------------------------------------------------------------- reinitialisation
def _dense(Pe, re, cells, n):
    P = np.zeros((n, n))
    r = np.zeros(n)
    for e in range(cells.shape[0]):
        for a in range(cells.shape[1]):
            r[cells[e, a]] += re[e, a]
            for b in range(cells.shape[1]):
                P[cells[e, a], cells[e, b]] += Pe[e, a, b]
    return P, r


@pytest.mark.parametrize("dim", [2, 3])
def test_reinit_constant_level_set_closed_form(dim):
    n = (4, 3) if dim == 2 else (2, 2, 2)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    h = m.diameter()
    c, T = -0.37, 0.02
    phi = np.full(m.num_nodes, c)
    S = c / math.sqrt(c * c + h * h)
    one = levelset.reinit(m, phi, 1, T, h)                       # one Euler step of size T
    assert np.allclose(one, c + T * S, rtol=0, atol=1e-14)
    two = levelset.reinit(m, phi, 2, T, h)                       # Euler then AB2, dt = T / 2
    assert np.allclose(two, c + T * S, rtol=0, atol=1e-14)       # c + 2 (T/2) S(c)


@pytest.mark.parametrize("dim", [2, 3])
def test_reinit_ab2_with_equal_history_is_euler(dim):
    n = (5, 4) if dim == 2 else (3, 2, 2)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    h = m.diameter()
    phi0 = levelset.initial_level(m.coords, [(0.4,) * dim], [0.3])
    cur = phi0 + 0.05 * workloads.smooth_field(m.coords, 1, 3)
    P1, r1 = levelset.reinit_step_system(m.coords, m.cells, phi0, cur, None, 0.01, h)
    P2, r2 = levelset.reinit_step_system(m.coords, m.cells, phi0, cur, cur.copy(), 0.01, h)
    assert np.allclose(P1, P2, rtol=0, atol=1e-16)
    assert np.allclose(r1, r2, rtol=1e-13, atol=1e-16)
    # and a different history changes the right-hand side (the history term is present)
    _, r3 = levelset.reinit_step_system(m.coords, m.cells, phi0, cur, phi0, 0.01, h)
    assert np.max(np.abs(r3 - r1)) > 1e-6


def _brute_step(coords, cells, phi0, cur, prev, dt, h):
    """One step of eq. weak_HJ, evaluated point by point (2D), assembled densely and solved."""
    nn = coords.shape[0]
    P = np.zeros((nn, nn))
    rhs = np.zeros(nn)
    pts, wts = levelset.quadrature(2)
    for e in range(cells.shape[0]):
        X = coords[cells[e]]
        E = np.column_stack([X[1] - X[0], X[2] - X[0]])
        Einv = np.linalg.inv(E)
        area = abs(np.linalg.det(E)) / 2.0

        def bary(x):
            l12 = Einv @ (x - X[0])
            return np.array([1.0 - l12.sum(), l12[0], l12[1]])

        def interp(vals, x):
            return float(bary(x) @ vals[cells[e]])

        def fd_grad(f, x, eps=1e-6):
            return np.array([(f(x + eps * np.eye(2)[k]) - f(x - eps * np.eye(2)[k])) / (2 * eps) for k in range(2)])

        gcur = fd_grad(lambda x: interp(cur, x), X.mean(axis=0))
        ncur = np.linalg.norm(gcur)
        ghat = gcur / ncur if ncur > 0 else np.zeros(2)
        gprev = None if prev is None else fd_grad(lambda x: interp(prev, x), X.mean(axis=0))
        glam = [fd_grad(lambda x, a=a: bary(x)[a], X.mean(axis=0)) for a in range(3)]

        def S(x):
            p = interp(phi0, x)
            return p / math.sqrt(p * p + h * h)

        def psihat(a, x):
            s = S(x)
            grad_H = s * ghat                                     # eq. grad_H at p = grad cur
            tau = 0.5 / math.sqrt(1.0 / dt**2 + (grad_H @ grad_H) / h**2)
            return bary(x)[a] + tau * (grad_H @ glam[a])

        for lam, w in zip(pts, wts):
            xq = lam @ X
            s = S(xq)
            Hc = s * ncur
            if prev is None:                                      # explicit Euler
                src = interp(cur, xq) + dt * s - dt * Hc
                flux = -h * h * gcur
            else:                                                 # G(u, v, w) with u = cur, v = prev
                Hv = s * np.linalg.norm(gprev)
                src = interp(cur, xq) + dt * s + dt * (Hv - 3.0 * Hc) / 2.0
                flux = h * h * (gprev - 3.0 * gcur) / 2.0
            for a in range(3):
                ph = psihat(a, xq)
                gph = fd_grad(lambda x, a=a: psihat(a, x), xq)
                A = cells[e, a]
                rhs[A] += w * area * (src * ph + dt * (flux @ gph))
                for b in range(3):
                    P[A, cells[e, b]] += w * area * ph * lam[b]
    return np.linalg.solve(P, rhs)


def test_reinit_two_steps_brute_force():
    m = BoxMesh(2, (3, 3), (0, 0), (1, 1))
    h = m.diameter()
    phi0 = 1.7 * levelset.initial_level(m.coords, [(0.45, 0.4)], [0.3]) + 0.02 * workloads.smooth_field(m.coords, 1, 8)
    T = 0.04
    dt = T / 2
    s1 = _brute_step(m.coords, m.cells, phi0, phi0, None, dt, h)
    s2 = _brute_step(m.coords, m.cells, phi0, s1, phi0, dt, h)
    got1 = levelset.reinit(m, phi0, 1, dt, h)
    got2 = levelset.reinit(m, phi0, 2, T, h)
    scale = np.max(np.abs(phi0))
    assert np.max(np.abs(got1 - s1)) <= 1e-7 * scale, np.max(np.abs(got1 - s1))
    assert np.max(np.abs(got2 - s2)) <= 1e-7 * scale, np.max(np.abs(got2 - s2))
    # the step did something beyond rounding
    assert np.max(np.abs(got2 - phi0)) > 1e-3
