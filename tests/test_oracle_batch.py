"""Pins of the oracle's task-parallel batch (summed cost, summed shape derivative).

A plausible mistake in the batch layer (a dropped instance, an instance's k or omega
paired with another's f, the volume term added once per instance) fails one of:
the Taylor test of the summed cost, invariance under a permutation of the instances,
linearity in the sources, and the omega = 0, k = 1 reduction to the heat problem.
"""
import numpy as np

from oracle import fem, shape
from oracle.algorithm import HEAT, Problem
from oracle.batch import Batch
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads
from tests.test_oracle_shape import _bubble_theta, _helm_J, _taylor


def _batch(m, n_inst=3, seed=1):
    k, om, amp = workloads.batch_parameters(n_inst, seed)
    f = workloads.fourier_loads(m.coords, amp)
    return Batch(m, k, om, f, dirichlet_faces=[(0, 0)], a_in=1.0, a_out=1e-2), amp


def test_batch_taylor_summed_cost():
    """d/dt sum_i J_i(moved mesh) = b . theta with b the summed tensors.  The sources are
    linear, f_i = c_i + g_i . x, so that their P1 interpolants are exact and the moved-mesh
    cost sees the same grad f_i as the distributed formula."""
    m = BoxMesh(2, (10, 10), (0, 0), (1, 1))
    rng = np.random.default_rng(4)
    k, om, _ = workloads.batch_parameters(3, seed=4)
    c = rng.standard_normal(3)
    gv = rng.standard_normal((3, 2))

    def f_fun(i):
        return lambda Y: c[i] + Y @ gv[i]

    bt = Batch(m, k, om, np.stack([f_fun(i)(m.coords) for i in range(3)]), dirichlet_faces=[(0, 0)],
               a_in=1.0, a_out=1e-2)
    phi = workloads.phi_cos(m.coords)
    U, A, chi = bt.state(phi)
    b = bt.rhs(U, A, chi)
    theta = _bubble_theta(m, 21)
    dJ = b @ theta
    dir_mask = m.face_nodes(0, 0)

    def Jsum(t):
        X = m.coords + t * theta.reshape(-1, 2)
        return sum(_helm_J(X, m.cells, A, bt.k[i], bt.omega[i], f_fun(i), dir_mask)[0] for i in range(3))

    errs = _taylor(Jsum, theta, dJ, 2)
    assert errs[1] < errs[0] / 50
    assert min(errs) < 1e-7


def test_batch_permutation_invariance():
    m = BoxMesh(2, (8, 6), (0, 0), (1, 1))
    bt, _ = _batch(m, 4, seed=2)
    phi = workloads.phi_cos(m.coords)
    U, A, chi = bt.state(phi)
    perm = np.array([2, 0, 3, 1])
    bp = Batch(m, bt.k[perm], bt.omega[perm], bt.f_nodal[perm], bt.dirichlet_faces, bt.a_in, bt.a_out)
    Up, _, _ = bp.state(phi)
    assert np.array_equal(Up, U[:, perm])
    assert np.allclose(bp.costs(Up, A), bt.costs(U, A)[perm], rtol=0, atol=0)
    assert np.allclose(bp.rhs(Up, A, chi), bt.rhs(U, A, chi), rtol=1e-13, atol=1e-15)


def test_batch_linear_in_sources():
    """Instance with f = f_0 + f_1 (same k, omega) has u = u_0 + u_1."""
    m = BoxMesh(2, (8, 8), (0, 0), (1, 1))
    rng = np.random.default_rng(3)
    f0, f1 = rng.standard_normal(m.num_nodes), rng.standard_normal(m.num_nodes)
    k = np.array([1.7, 1.7, 1.7])
    om = np.array([2.0, 2.0, 2.0])
    bt = Batch(m, k, om, np.stack([f0, f1, f0 + f1]), dirichlet_faces=[(0, 0)])
    U, _, _ = bt.state(workloads.phi_cos(m.coords))
    assert np.allclose(U[:, 2], U[:, 0] + U[:, 1], rtol=0, atol=1e-12 * np.abs(U).max())


def test_batch_reduces_to_heat():
    """omega = 0 and k = 1: each instance is the heat state problem with source f_i, and
    its J_i = int f u equals the heat compliance int A |grad u|^2 (Galerkin identity)."""
    m = BoxMesh(2, (8, 8), (0, 0), (1, 1))
    f = workloads.fourier_loads(m.coords, np.random.default_rng(5).standard_normal((2, 8)))
    bt = Batch(m, np.ones(2), np.zeros(2), f, dirichlet_faces=[(0, 0)])
    phi = workloads.phi_cos(m.coords)
    U, A, chi = bt.state(phi)
    vol, g = fem.geometry(m.coords, m.cells)
    for i in range(2):
        heat = Problem(m, HEAT, dirichlet_faces=[(0, 0)], f_nodal=f[i])
        u_h, A_h, _ = heat.state(phi)
        assert np.allclose(U[:, i], u_h, rtol=0, atol=1e-13 * np.abs(u_h).max())
        J_heat = shape.heat_cost(vol, g, A_h, u_h, m.cells)
        assert abs(bt.costs(U, A)[i] - J_heat) <= 1e-10 * abs(J_heat)
        # the tensors coincide too: S of J = int f u with omega = 0 is the heat S (Sec. 6.3)
        b_heat = shape.heat_rhs(m.coords, m.cells, A_h, u_h, f[i])
        b_i = bt.problem(i).rhs(U[:, i], A, chi, 0.0)
        assert np.allclose(b_i, b_heat, rtol=0, atol=1e-12 * np.abs(b_heat).max())


def test_batch_volume_term_added_once():
    m = BoxMesh(2, (6, 6), (0, 0), (1, 1))
    bt, _ = _batch(m, 3, seed=6)
    bt.volume_target = 0.4
    phi = workloads.phi_cos(m.coords)
    U, A, chi = bt.state(phi)
    lam = 0.37
    diff = bt.rhs(U, A, chi, lam) - bt.rhs(U, A, chi, 0.0)
    ref = lam * shape.volume_rhs(m.coords, m.cells, chi, 0.4)
    assert np.allclose(diff, ref, rtol=1e-12, atol=1e-14)
