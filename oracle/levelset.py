"""Level-set transport, reinitialisation and initial level set (oracle).

Quadrature: the transport and reinitialisation forms contain tau, S(phi) and
grad H, which are not polynomial; they are integrated with a fixed degree-2
rule (2D: the three points with barycentrics (2/3, 1/6, 1/6) and permutations,
weights |e|/3; 3D: the four points (a, b, b, b), a = (5 + 3 sqrt 5)/20,
b = (5 - sqrt 5)/20, weights |e|/4).  The rule is exact on the polynomial
(quadratic) parts of the forms.
"""
import math

import numpy as np

from . import fem, solvers


def quadrature(d):
    """Barycentric points [Q, d+1] and weights (fractions of |e|) of the degree-2 rule."""
    if d == 2:
        pts = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
        return pts, np.full(3, 1 / 3)
    a = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
    b = (5.0 - math.sqrt(5.0)) / 20.0
    pts = np.full((4, 4), b)
    np.fill_diagonal(pts, a)
    return pts, np.full(4, 1 / 4)


# ------------------------------------------------------------------ transport
def transport_element_matrices(coords, cells, theta, dt, h, smooth):
    """Element matrices of the SUPG / Crank-Nicolson transport step (Sec. 5.6).

    eq. weak_transport: int phi^{n+1} psi^ + dt F(phi^{n+1}, psi^)
                        = int phi^n psi^ - dt F(phi^n, psi^),
    F(u, v) = (theta . grad u) v / 2 + s h^2 grad u . grad v / 2 (s = 1 with
    ``smooth``, else 0: the diffusion of eq. transport is optional),
    psi^ = psi + tau theta . grad psi, tau from eq. tau_lv evaluated pointwise.
    The diffusion term is tested with grad psi^ in full:
    grad psi^ = grad psi + (theta . grad psi) grad tau + tau (D theta)^T grad psi,
    grad tau = -(1/2) s^{-3/2} (D theta)^T theta / h^2, s = 1/dt^2 + |theta|^2/h^2.
    Returns (L_e, R_e) with rows = test psi_a, columns = trial psi_b.
    """
    vol, g = fem.geometry(coords, cells)
    d = coords.shape[1]
    th = theta.reshape(-1, d)[cells]                          # [NT, d+1, d]
    Dth = np.einsum("ebi,ebj->eij", th, g)                    # (D theta)_ij = d_j theta_i
    pts, wts = quadrature(d)
    mass_hat = np.zeros((cells.shape[0], d + 1, d + 1))
    adv = np.zeros_like(mass_hat)
    diff = np.zeros_like(mass_hat)
    for lam, w in zip(pts, wts):
        thq = np.einsum("b,ebi->ei", lam, th)
        s = 1.0 / dt**2 + np.einsum("ei,ei->e", thq, thq) / h**2
        tau = 0.5 / np.sqrt(s)
        gtau = -0.5 * s**-1.5 / h**2
        gtau = gtau[:, None] * np.einsum("eji,ej->ei", Dth, thq)
        thg = np.einsum("ei,eai->ea", thq, g)                # theta . grad psi_a
        test = lam[None, :] + tau[:, None] * thg             # psi^_a(q)
        gtest = (g + thg[:, :, None] * gtau[:, None, :]
                 + tau[:, None, None] * np.einsum("eji,eaj->eai", Dth, g))
        wv = w * vol
        mass_hat += wv[:, None, None] * test[:, :, None] * lam[None, None, :]
        adv += wv[:, None, None] * test[:, :, None] * thg[:, None, :]
        diff += (wv * h * h)[:, None, None] * np.einsum("eai,ebi->eab", gtest, g)
    F = adv + (diff if smooth else 0.0)
    return mass_hat + 0.5 * dt * F, mass_hat - 0.5 * dt * F


def transport_matrices(mesh, theta, dt, h, smooth):
    Le, Re = transport_element_matrices(mesh.coords, mesh.cells, theta, dt, h, smooth)
    cells = mesh.cells.astype(np.int64)
    return fem.assemble(Le, cells, mesh.num_nodes), fem.assemble(Re, cells, mesh.num_nodes)


def transport(mesh, phi, theta, t_end, nsteps, h, smooth):
    """nsteps Crank-Nicolson steps of size t_end / nsteps: L phi^{n+1} = R phi^n."""
    dt = t_end / nsteps
    L, R = transport_matrices(mesh, theta, dt, h, smooth)
    for _ in range(nsteps):
        phi = solvers.solve(L, R @ phi)
    return phi


# ------------------------------------------------------------- reinitialisation
def reinit_step_system(coords, cells, phi0, cur, prev, dt, h):
    """Matrix and RHS of one step of the reinitialisation scheme (Sec. 5.7).

    Diffusive eikonal equation (eq. Eikonal) with S(phi0) = phi0 / sqrt(phi0^2 + h^2)
    evaluated at quadrature points, H(p) = S |p| (eq. HJ), grad H(p) = S p / |p|
    (eq. grad_H; taken as 0 where p = 0).  Test function
    psi^ = psi + tau grad H(grad cur) . grad psi, tau = (1/2)(1/dt^2 + |grad H|^2/h^2)^{-1/2},
    with grad psi^ taken in full (the derivative of tau S along grad phi0).
    eq. weak_HJ (two-step Adams-Bashforth, prev = phi(t - dt)):
      int phi^{n+1} psi^ = int (cur + dt S) psi^ + dt int G(cur, prev, psi^),
      G(u, v, w) = (H(grad v) - 3 H(grad u))/2 w + h^2 (grad v - 3 grad u)/2 . grad w.
    With prev = None the first step is explicit Euler:
      G -> -H(grad u) w - h^2 grad u . grad w.
    Returns element matrices P_e [NT, d+1, d+1] and element RHS [NT, d+1].
    """
    vol, g = fem.geometry(coords, cells)
    d = coords.shape[1]
    pts, wts = quadrature(d)
    p0e, ce = phi0[cells], cur[cells]
    gc = np.einsum("ea,eak->ek", ce, g)                      # grad cur
    gp0 = np.einsum("ea,eak->ek", p0e, g)                    # grad phi0
    nc = np.linalg.norm(gc, axis=1)
    has = nc > 0.0
    ghat = np.where(has[:, None], gc / np.where(has, nc, 1.0)[:, None], 0.0)
    gv = None if prev is None else np.einsum("ea,eak->ek", prev[cells], g)
    P = np.zeros((cells.shape[0], d + 1, d + 1))
    rhs = np.zeros((cells.shape[0], d + 1))
    ghg = np.einsum("ei,eai->ea", ghat, g)                   # ghat . grad psi_a
    for lam, w in zip(pts, wts):
        p0q = p0e @ lam
        cq = ce @ lam
        r2 = p0q * p0q + h * h
        S = p0q / np.sqrt(r2)
        dS = h * h / (r2 * np.sqrt(r2))                      # S'(phi0)
        gH = np.where(has, np.abs(S), 0.0)                   # |grad H|
        sq = 1.0 / dt**2 + gH * gH / h**2
        tau = 0.5 / np.sqrt(sq)
        dtau = -0.5 * sq**-1.5 * S / h**2                    # d tau / d S
        beta = np.where(has, tau * S, 0.0)                   # psi^ = psi + beta ghat.grad psi
        dbeta = np.where(has, (tau + S * dtau) * dS, 0.0)    # d beta / d phi0
        gbeta = dbeta[:, None] * gp0
        test = lam[None, :] + beta[:, None] * ghg
        gtest = g + ghg[:, :, None] * gbeta[:, None, :]
        wv = w * vol
        P += wv[:, None, None] * test[:, :, None] * lam[None, None, :]
        Hc = S * nc
        if gv is None:
            src = cq + dt * S - dt * Hc
            flux = -(h * h) * gc
        else:
            Hv = S * np.linalg.norm(gv, axis=1)
            src = cq + dt * S + dt * 0.5 * (Hv - 3.0 * Hc)
            flux = (h * h) * 0.5 * (gv - 3.0 * gc)
        rhs += wv[:, None] * (src[:, None] * test + dt * np.einsum("ek,eak->ea", flux, gtest))
    return P, rhs


def reinit(mesh, phi, nsteps, t_final, h):
    """nsteps steps of size t_final / nsteps; the first by explicit Euler, then AB2."""
    dt = t_final / nsteps
    cells = mesh.cells.astype(np.int64)
    prev, cur = None, phi.copy()
    for _ in range(nsteps):
        Pe, re = reinit_step_system(mesh.coords, mesh.cells, phi, cur, prev, dt, h)
        P = fem.assemble(Pe, cells, mesh.num_nodes)
        rhs = fem.assemble_vector(re, cells, mesh.num_nodes)
        prev, cur = cur, solvers.solve(P, rhs)
    return cur


# -------------------------------------------------------------- initial guess
def initial_level(coords, centers, radii, factor=1.0, ord=2):
    """phi0(x) = factor * max_k (radii_k - |x - centers_k|_ord)  (eq. phi0)."""
    centers = np.asarray(centers, dtype=np.float64)
    radii = np.asarray(radii, dtype=np.float64)
    diff = coords[:, None, :] - centers[None, :, :]
    dist = np.linalg.norm(diff, ord=ord, axis=2)
    return factor * np.max(radii[None, :] - dist, axis=1)
