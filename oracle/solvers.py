"""Linear solvers of the oracle: sparse direct, Jacobi-PCG, Jacobi-BiCGStab.

The paper never states its PETSc solvers; the oracle answers with the exact
solution of each discrete system (sparse LU), so GPU Krylov results are
compared with the system's solution, not with another iterative method.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve_free(A, b, free):
    """Solve A u = b on the free DOFs with u = 0 on the others (homogeneous Dirichlet)."""
    idx = np.flatnonzero(free)
    u = np.zeros(A.shape[0])
    if idx.size:
        Aff = A[idx][:, idx].tocsc()
        u[idx] = spla.spsolve(Aff, b[idx])
    return u


def solve(A, b):
    """Sparse direct solve of a square system."""
    return spla.spsolve(sp.csc_matrix(A), b)


def jacobi_pcg(A, b, rtol=1e-12, maxit=100000, x0=None):
    """Textbook preconditioned conjugate gradients with the Jacobi preconditioner.

    Stops when ||r||_2 <= rtol ||b||_2.  Returns (x, iterations, ||r||/||b||).
    """
    n = b.shape[0]
    dinv = 1.0 / A.diagonal()
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    r = b - A @ x
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros(n), 0, 0.0
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    while np.linalg.norm(r) > rtol * bn and it < maxit:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it, np.linalg.norm(r) / bn


def jacobi_bicgstab(A, b, rtol=1e-12, maxit=100000, x0=None):
    """Textbook right-preconditioned BiCGStab (van der Vorst) with a Jacobi preconditioner."""
    n = b.shape[0]
    dinv = 1.0 / A.diagonal()
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    r = b - A @ x
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros(n), 0, 0.0
    rhat = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros(n)
    p = np.zeros(n)
    it = 0
    while np.linalg.norm(r) > rtol * bn and it < maxit:
        rho_new = rhat @ r
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        y = dinv * p
        v = A @ y
        alpha = rho_new / (rhat @ v)
        s = r - alpha * v
        zs = dinv * s
        t = A @ zs
        omega = (t @ s) / (t @ t) if (t @ t) > 0 else 0.0
        x += alpha * y + omega * zs
        r = s - omega * t
        rho = rho_new
        it += 1
    return x, it, np.linalg.norm(r) / bn
