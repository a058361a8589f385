"""Logistic population model with a Newton state solve (oracle; Sec. 6.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

State (eq. log_weak): find u in H^1(D) with
    F(u)(v) = int grad u . grad v - int r u (1 - u / K) v = 0   for all v,
no Dirichlet condition, K = K_Omega the carrying capacity of eq. log_KOmega:
K = k_in on Omega = {phi < 0} and k_out elsewhere (k_in = 1, k_out = 1e-2 in the paper),
evaluated per element with the same one-point (vertex-sum) rule as the ersatz coefficient.
Newton (the method the paper names for this model) with the Jacobian
    DF(u)(du, v) = int grad du . grad v + int r (2u / K - 1) du v,
from the initial guess u_0 (the paper's 1 + 0.2 sin(6 pi x) sin(6 pi y) in its example).
Every integral is exact for P1 data: the cubic terms use
    int_e lambda_a lambda_b lambda_c = |e| d! m(a, b, c) / (d + 3)!,
m = 1, 2 or 6 when a, b, c take three, two or one distinct values.

Adjoint (linear, Sec. 6.4): int grad p . grad q + int r (2u / K - 1) p q = int q.
Cost J = -int u (eq. log_cost); constraint C = int chi / V (eq. log_const).
Shape derivative (Sec. 6.4): S0^J = 0,
    S1^J = (grad u . grad p - u - r u (1 - u / K) p) I - (grad u (x) grad p + grad p (x) grad u),
S1^C = chi / V I.  The velocity right-hand side is b[a, k] = sum_e int_e (S1 grad psi_a)_k.

Newton stopping rule (the paper does not state one): stop at the first iterate with
||F(u_k)||_2 <= rtol ||F(u_0)||_2 + atol, or when the update ||du||_inf <= 1e-14 ||u||_inf.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, shape


def carrying_capacity(phi, cells, k_in=1.0, k_out=1e-2):
    """K_e and chi_e: k_in on inside elements (vertex sum of phi < 0), k_out elsewhere."""
    return shape.coefficient(phi, cells, k_in, k_out)


def cubic_tensor(d):
    """T[a, b, c] = int_e lambda_a lambda_b lambda_c / |e| on a d-simplex."""
    n = d + 1
    T = np.zeros((n, n, n))
    for a in range(n):
        for b in range(n):
            for c in range(n):
                distinct = len({a, b, c})
                mult = {3: 1, 2: 2, 1: 6}[distinct]
                T[a, b, c] = math.factorial(d) * mult / math.factorial(d + 3)
    return T


def _elements(coords, cells):
    vol, g = fem.geometry(coords, cells)
    return vol, g, cells.astype(np.int64)


def residual(coords, cells, K, r, u, extra=None):
    """F(u)_a = int grad u . grad psi_a - r int u psi_a + r int (u^2 / K) psi_a  (- extra_a)."""
    vol, g, c = _elements(coords, cells)
    d = coords.shape[1]
    ue = u[c]
    Ke = fem.scalar_stiffness(vol, g, np.ones_like(vol))
    Me = fem.mass(vol, d)
    T = cubic_tensor(d)
    Fe = np.einsum("eab,eb->ea", Ke, ue) - r * np.einsum("eab,eb->ea", Me, ue)
    Fe += (r / K * vol)[:, None] * np.einsum("abc,eb,ec->ea", T, ue, ue)
    F = fem.assemble_vector(Fe, c, coords.shape[0])
    if extra is not None:
        F = F - extra
    return F


def jacobian(coords, cells, K, r, u):
    """DF(u): stiffness + the mass weighted by the P1 function w = r (2u / K_e - 1)."""
    vol, g, c = _elements(coords, cells)
    d = coords.shape[1]
    Ke = fem.scalar_stiffness(vol, g, np.ones_like(vol))
    we = r * (2.0 * u[c] / K[:, None] - 1.0)                     # vertex values of w per element
    Mw = vol[:, None, None] * np.einsum("abc,ec->eab", cubic_tensor(d), we)
    return fem.assemble(Ke + Mw, c, coords.shape[0])


def newton(coords, cells, K, r, u0, rtol=1e-13, atol=0.0, maxit=50, extra=None):
    """Newton's method with sparse direct solves; returns (u, [||F(u_k)||_2 for k = 0, 1, ...])."""
    u = np.array(u0, dtype=np.float64)
    F = residual(coords, cells, K, r, u, extra)
    hist = [float(np.linalg.norm(F))]
    for _ in range(maxit):
        if hist[-1] <= rtol * hist[0] + atol:
            break
        du = spla.spsolve(sp.csc_matrix(jacobian(coords, cells, K, r, u)), -F)
        u = u + du
        F = residual(coords, cells, K, r, u, extra)
        hist.append(float(np.linalg.norm(F)))
        if np.max(np.abs(du)) <= 1e-14 * np.max(np.abs(u)):
            break
    return u, hist


def adjoint(coords, cells, K, r, u):
    """p with DF(u)^T p = (int psi_a)_a (DF is symmetric)."""
    one = fem.body_load(coords, cells, np.ones(coords.shape[0]))
    return spla.spsolve(sp.csc_matrix(jacobian(coords, cells, K, r, u)), one)


def cost(coords, cells, u):
    """J = -int_D u, exact for P1 u."""
    vol, _, c = _elements(coords, cells)
    return float(-np.sum(vol * u[c].mean(axis=1)))


def rhs(coords, cells, K, r, u, p, lam=0.0, chi=None, V=1.0):
    """b[d*a + k] = sum_e int_e (S1 grad psi_a)_k with S1 = S1^J + lam S1^C (Sec. 6.4)."""
    vol, g, c = _elements(coords, cells)
    d = coords.shape[1]
    ue, pe = u[c], p[c]
    gu = np.einsum("ea,eak->ek", ue, g)
    gp = np.einsum("ea,eak->ek", pe, g)
    Me = fem.mass(vol, d)
    T = cubic_tensor(d)
    int_u = vol * ue.mean(axis=1)                                  # int_e u
    int_up = np.einsum("ea,eab,eb->e", ue, Me, pe)                 # int_e u p
    int_uup = vol * np.einsum("abc,ea,eb,ec->e", T, ue, ue, pe)    # int_e u^2 p
    scal = vol * np.einsum("ek,ek->e", gu, gp) - int_u - r * int_up + (r / K) * int_uup
    S1 = scal[:, None, None] * np.eye(d)[None] - vol[:, None, None] * (
        np.einsum("ei,ej->eij", gu, gp) + np.einsum("ei,ej->eij", gp, gu))
    if chi is not None and lam != 0.0:
        S1 = S1 + (lam * chi * vol / V)[:, None, None] * np.eye(d)[None]
    be = np.einsum("eij,eaj->eai", S1, g)
    out = np.zeros((coords.shape[0], d))
    for a in range(cells.shape[1]):
        np.add.at(out, c[:, a], be[:, a, :])
    return out.reshape(-1)

