"""Pins of the oracle's transport, reinitialisation and initial level set."""
import math

import numpy as np
import pytest

from oracle import fem, levelset
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads


def test_quadrature_degree_two():
    for d in (2, 3):
        pts, w = levelset.quadrature(d)
        assert abs(w.sum() - 1.0) < 1e-15
        assert np.allclose(pts.sum(axis=1), 1.0)
        # exact moments on the reference simplex: int l_a = 1/(d+1), int l_a l_b = (1+delta)/((d+1)(d+2))
        for a in range(d + 1):
            assert abs(np.sum(w * pts[:, a]) - 1 / (d + 1)) < 1e-15
            for b in range(d + 1):
                ref = (1 + (a == b)) / ((d + 1) * (d + 2))
                assert abs(np.sum(w * pts[:, a] * pts[:, b]) - ref) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_velocity_no_smoothing_is_identity(dim):
    n = (6, 5) if dim == 2 else (3, 3, 2)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    phi = workloads.phi_cos(m.coords)
    out = levelset.transport(m, phi, np.zeros(dim * m.num_nodes), 0.05, 8, m.diameter(), smooth=False)
    assert np.max(np.abs(out - phi)) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_velocity_smoothing_conserves_mass(dim):
    n = (8, 6) if dim == 2 else (3, 3, 3)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    phi = workloads.phi_cos(m.coords)
    out = levelset.transport(m, phi, np.zeros(dim * m.num_nodes), 0.05, 10, m.diameter(), smooth=True)
    vol, _ = fem.geometry(m.coords, m.cells)
    M = fem.assemble(fem.mass(vol, dim), m.cells.astype(np.int64), m.num_nodes)
    one = np.ones(m.num_nodes)
    assert abs(one @ (M @ out) - one @ (M @ phi)) < 1e-13
    assert np.max(np.abs(out - phi)) > 1e-6           # diffusion acted


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_velocity_linear_phi_exact(dim):
    # phi(t) = phi0 - t theta . grad phi0 is linear, lies in V_h and satisfies the SUPG/CN weak form
    # exactly, so n steps reproduce it to rounding
    n = (7, 5) if dim == 2 else (3, 4, 3)
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    gphi = np.array([0.8, -0.5, 0.3][:dim])
    th = np.array([0.3, 0.7, -0.2][:dim])
    phi0 = 0.1 + m.coords @ gphi
    theta = np.tile(th, m.num_nodes)
    t_end, ns = 0.04, 9
    out = levelset.transport(m, phi0, theta, t_end, ns, m.diameter(), smooth=False)
    exact = phi0 - t_end * (th @ gphi)
    assert np.max(np.abs(out - exact)) < 1e-13


def test_transport_moves_interface_downstream():
    # a round hole advected by theta = (1, 0): the zero set moves right by ~ t_end
    m = BoxMesh(2, (64, 32), (0, 0), (2, 1))
    phi0 = levelset.initial_level(m.coords, [(0.8, 0.5)], [0.2], factor=-1.0)   # Omega = disk
    theta = np.tile([1.0, 0.0], m.num_nodes)
    out = levelset.transport(m, phi0, theta, 0.1, 16, m.diameter(), smooth=False)
    row = m.node_index[:, 1] == 16
    x = m.coords[row, 0]
    inside = x[out[row] < 0]
    assert abs(inside.min() - 0.7) < 0.04 and abs(inside.max() - 1.1) < 0.04


def _fd_grad_test(coords, cells, theta, dt, h, e, a, lam):
    """Finite-difference gradient of psi^_a = psi_a + tau theta . grad psi_a at a point of element e."""
    vol, g = fem.geometry(coords, cells)
    X = coords[cells[e]]
    th = theta.reshape(-1, coords.shape[1])[cells[e]]
    x0 = lam @ X
    E = (X[1:] - X[0]).T
    Einv = np.linalg.inv(E)

    def bary(x):
        l = Einv @ (x - X[0])
        return np.concatenate([[1 - l.sum()], l])

    def test(x):
        l = bary(x)
        thx = l @ th
        tau = 0.5 / math.sqrt(1 / dt**2 + thx @ thx / h**2)
        return l[a] + tau * (thx @ g[e, a])

    eps = 1e-6
    return np.array([(test(x0 + eps * np.eye(len(x0))[k]) - test(x0 - eps * np.eye(len(x0))[k])) / (2 * eps)
                     for k in range(len(x0))])


def test_transport_diffusion_term_uses_full_test_gradient():
    # reconstruct the diffusion part of L - R with finite-difference gradients of psi^
    m = BoxMesh(2, (3, 3), (0, 0), (1, 1))
    theta = workloads.smooth_field(m.coords, 2, 21)
    dt, h = 0.05, m.diameter()
    L0, R0 = levelset.transport_element_matrices(m.coords, m.cells, theta, dt, h, smooth=False)
    L1, R1 = levelset.transport_element_matrices(m.coords, m.cells, theta, dt, h, smooth=True)
    diff = (L1 - L0) / (0.5 * dt)                         # = int h^2 grad psi_b . grad psi^_a
    vol, g = fem.geometry(m.coords, m.cells)
    pts, wts = levelset.quadrature(2)
    for e in (0, 5, 11):
        for a in range(3):
            ref = np.zeros(3)
            for lam, w in zip(pts, wts):
                gt = _fd_grad_test(m.coords, m.cells, theta, dt, h, e, a, lam)
                ref += w * vol[e] * h * h * (g[e] @ gt)
            assert np.allclose(diff[e, a], ref, rtol=1e-7, atol=1e-12)
    assert np.allclose(L1 + R1, L0 + R0, atol=1e-15)     # L + R = 2 M^ whatever the smoothing


def test_initial_level_closed_form():
    X = np.array([[0.5, 0.5], [0.0, 0.0], [1.0, 0.5]])
    phi = levelset.initial_level(X, [(0.5, 0.5), (1.0, 0.5)], [0.1, 0.2], factor=1.0)
    assert phi[0] == pytest.approx(0.1)
    assert phi[1] == pytest.approx(max(0.1 - math.sqrt(0.5), 0.2 - math.sqrt(1.25)))
    assert phi[2] == pytest.approx(0.2)
    phi_inf = levelset.initial_level(X, [(0.5, 0.5)], [0.3], factor=-2.0, ord=np.inf)
    assert phi_inf[1] == pytest.approx(-2.0 * (0.3 - 0.5))


def test_reinit_properties():
    # parity unpinned: the scheme has no closed-form answer.  Properties: the sign of phi is kept
    # away from the interface, and |grad phi| near the interface moves towards 1.
    m = BoxMesh(2, (64, 64), (0, 0), (1, 1))
    phi = 3.0 * levelset.initial_level(m.coords, [(0.5, 0.5)], [0.25])      # |grad phi| = 3
    h = m.diameter()
    out = levelset.reinit(m, phi, 20, 0.1, h)
    far = np.abs(phi) > 6 * h
    assert np.all(np.sign(out[far]) == np.sign(phi[far]))
    vol, g = fem.geometry(m.coords, m.cells)
    c = m.centroids()
    band = np.abs(np.linalg.norm(c - 0.5, axis=1) - 0.25) < 3 * h
    gn0 = np.linalg.norm(np.einsum("ea,eak->ek", phi[m.cells], g), axis=1)[band].mean()
    gn1 = np.linalg.norm(np.einsum("ea,eak->ek", out[m.cells], g), axis=1)[band].mean()
    assert abs(gn1 - 1.0) < 0.5 * abs(gn0 - 1.0)
