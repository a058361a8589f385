"""Pins of the oracle's exact cut-cell fraction |e cap {phi < 0}| / |e| (the variant of the
ersatz coefficient that replaces the one-point rule): planar cuts of the reference triangle
and tetrahedron with closed-form areas / volumes, the complement rule, invariance under the
vertex order, and sampling on random simplices."""
import math

import numpy as np
import pytest

from oracle import shape


def test_triangle_planar_cut_closed_form():
    cells = np.array([[0, 1, 2]])
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    for t in (0.1, 0.37, 0.5, 0.9):
        phi = X[:, 0] - t                               # {x < t}: area t - t^2/2 of 1/2
        assert abs(shape.cut_fraction(phi, cells)[0] - (2 * t - t * t)) < 1e-14
        phi2 = X[:, 0] + X[:, 1] - t                    # {x + y < t}: area t^2/2
        assert abs(shape.cut_fraction(phi2, cells)[0] - t * t) < 1e-14


def test_tetrahedron_planar_cuts_closed_form():
    cells = np.array([[0, 1, 2, 3]])
    X = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    for t in (0.2, 0.5, 0.77):
        # one vertex on the negative side: {x + y + z < t} has volume t^3 / 6
        assert abs(shape.cut_fraction(X.sum(axis=1) - t, cells)[0] - t ** 3) < 1e-14
        # three on the negative side: {x < t} is the tet minus (1 - t)^3 of it
        assert abs(shape.cut_fraction(X[:, 0] - t, cells)[0] - (1 - (1 - t) ** 3)) < 1e-14
        # two and two: {x + y < t} has fraction 3 t^2 - 2 t^3
        assert abs(shape.cut_fraction(X[:, 0] + X[:, 1] - t, cells)[0] - (3 * t * t - 2 * t ** 3)) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_complement_order_and_sampling(d):
    rng = np.random.default_rng(d)
    n = 60
    cells = np.arange(n * (d + 1)).reshape(n, d + 1)
    phi = rng.standard_normal(n * (d + 1))
    f = shape.cut_fraction(phi, cells)
    assert np.all((f >= 0) & (f <= 1))
    assert np.allclose(f + shape.cut_fraction(-phi, cells), 1.0, atol=1e-14)
    perm = cells[:, rng.permutation(d + 1)]
    assert np.allclose(shape.cut_fraction(phi, perm), f, atol=1e-14)
    # sampling: uniform barycentric points (Dirichlet(1,...,1)); phi linear in them
    lam = rng.dirichlet(np.ones(d + 1), size=200000)
    for e in range(6):
        est = np.mean(lam @ phi[cells[e]] < 0.0)
        assert abs(est - f[e]) < 6e-3, (e, est, f[e])


def test_vertex_on_zero_counts_outside_and_whole_elements():
    cells = np.array([[0, 1, 2]])
    assert shape.cut_fraction(np.array([0.0, 1.0, 2.0]), cells)[0] == 0.0
    assert shape.cut_fraction(np.array([0.0, -1.0, -2.0]), cells)[0] == pytest.approx(1.0, abs=1e-15)
    assert shape.cut_fraction(np.array([-1.0, -1.0, -2.0]), cells)[0] == 1.0
    A, frac = shape.coefficient_cut(np.array([-1.0, 1.0, 1.0]), cells, 1.0, 1e-3)
    assert frac[0] == pytest.approx(0.25, abs=1e-15)          # (1/2)^2
    assert A[0] == pytest.approx(1e-3 + (1 - 1e-3) * 0.25, rel=1e-15)
