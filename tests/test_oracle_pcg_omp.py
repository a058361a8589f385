"""The OpenMP Jacobi-PCG of the oracle (the benchmark's all-cores CPU figure) against the
oracle's direct solve of a state system, and its iteration count against the textbook
bound on a matrix with a known spectrum."""
import math

import numpy as np
import scipy.sparse as sp

from oracle import pcg_omp, solvers
from tests.helpers import cantilever2d, oracle_problem
from paper_2601_05709_gb300 import workloads
from oracle import levelset


def test_pcg_omp_matches_direct_solve_on_cantilever():
    c = cantilever2d((32, 16))
    op = oracle_problem(c)
    cen, rad = workloads.hole_lattice()
    phi = levelset.initial_level(op.mesh.coords, cen, rad)
    u_ref, A, _ = op.state(phi)
    free = np.flatnonzero(op.dirichlet() == 0)
    K = op.stiffness(A)[free][:, free]
    x, it, rr, nt = pcg_omp.pcg(K, op.load()[free], rtol=1e-13, maxit=100000)
    assert rr <= 1e-13 and nt >= 1 and it > 10
    assert np.max(np.abs(x - u_ref[free])) <= 1e-8 * np.max(np.abs(u_ref))


def test_pcg_omp_iterations_within_cg_bound():
    # D^{-1} K = I + E with a known spectrum in [1, kappa]: CG needs at most
    # ceil(sqrt(kappa)/2 * ln(2/eps)) iterations for a relative A-norm reduction eps
    n, kappa = 400, 100.0
    lam = np.linspace(1.0, kappa, n)
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((n, n)))
    M = (Q * lam) @ Q.T
    Dh = np.sqrt(np.diag(M))
    K = sp.csr_matrix(M)
    b = np.random.default_rng(4).standard_normal(n)
    x, it, rr, _ = pcg_omp.pcg(K, b, rtol=1e-10)
    assert np.linalg.norm(K @ x - b) <= 1e-9 * np.linalg.norm(b)
    assert np.allclose(x, solvers.solve(K, b), rtol=0, atol=1e-8 * np.max(np.abs(x)))
    # Jacobi scaling changes the spectrum; bound with the scaled matrix's condition number
    S = M / np.outer(Dh, Dh)
    ev = np.linalg.eigvalsh(S)
    k2 = ev[-1] / ev[0]
    bound = math.ceil(0.5 * math.sqrt(k2) * math.log(2.0 / 1e-10 * math.sqrt(k2))) + 5
    assert it <= bound, (it, bound)
