"""Ersatz coefficient, functionals and the distributed shape derivative (oracle).

Omega = {phi < 0} (eq. subdomain).  The material coefficient
A_Omega = a_in chi_Omega + a_out chi_{D \\ Omega} (eqs heat_AOmega,
compli_AOmega; UFL conditional(lt(phi, 0), a_in, a_out)) is evaluated with a
one-point rule: element e is inside when the vertex values of phi, summed in
vertex order, are < 0 (a zero sum counts as outside, matching the strict lt).

The shape derivative has the tensor representation of Def. 2,
dJ(Omega; theta) = int_D S1 : D theta + S0 . theta, with S = S^J + lambda S^C
(eq. S0andS1).  Tested with the vector hat function theta = psi_a e_k, whose
Jacobian is e_k (x) grad psi_a, it gives the velocity right-hand side
    b[a, k] = sum_e int_e S0_k psi_a + (S1 grad psi_a)_k,
stored interleaved at index d*a + k.
"""
import numpy as np

from . import fem


def element_inside(phi, cells):
    """chi_e in {0, 1}: 1 when (phi_0 + phi_1) + phi_2 (+ phi_3) < 0."""
    s = phi[cells[:, 0]].copy()
    for m in range(1, cells.shape[1]):
        s = s + phi[cells[:, m]]
    return (s < 0.0).astype(np.uint8)


def coefficient(phi, cells, a_in, a_out):
    """A_e = a_in on inside elements, a_out elsewhere."""
    chi = element_inside(phi, cells)
    return np.where(chi == 1, a_in, a_out), chi


def cut_fraction(phi, cells):
    """|e cap {phi < 0}| / |e| for the P1 interpolant of phi on every simplex (exact).

    phi is linear on the simplex, so in barycentric coordinates the set {phi < 0} is the
    convex polytope spanned by the vertices with phi < 0 and the points where phi vanishes on
    the edges joining them to the other vertices (the vertex with phi = 0 belongs to the
    other side, matching the strict inequality).  Its measure in the reference simplex is that
    polytope's convex-hull measure (qhull), divided by the reference simplex's 1/d!.
    """
    from scipy.spatial import ConvexHull, QhullError
    import math
    d = cells.shape[1] - 1
    ref = np.vstack([np.zeros(d), np.eye(d)])            # reference vertices (barycentrics 1..d)
    out = np.zeros(cells.shape[0])
    for e in range(cells.shape[0]):
        v = phi[cells[e]]
        neg = v < 0.0
        if not neg.any():
            continue
        if neg.all():
            out[e] = 1.0
            continue
        pts = [ref[i] for i in range(d + 1) if neg[i]]
        for i in range(d + 1):
            for j in range(d + 1):
                if neg[i] and not neg[j]:
                    t = v[i] / (v[i] - v[j])             # phi = 0 at ref[i] + t (ref[j] - ref[i])
                    pts.append(ref[i] + t * (ref[j] - ref[i]))
        try:
            out[e] = ConvexHull(np.array(pts)).volume * math.factorial(d)
        except QhullError:                               # a flat set: measure zero
            out[e] = 0.0
    return out


def coefficient_cut(phi, cells, a_in, a_out):
    """Exact cut-cell coefficient: A_e = a_out + (a_in - a_out) |e cap Omega| / |e|, with the
    material fraction itself as chi_e (the element-wise constant of int_e chi_Omega / |e|)."""
    frac = cut_fraction(phi, cells)
    return a_out + (a_in - a_out) * frac, frac


def volume(vol, chi):
    """|Omega| = int_D chi_Omega, exact for the element-wise constant chi."""
    return float(np.sum(chi * vol))


# ---------------------------------------------------------------- heat model
def heat_cost(vol, grads, A, u, cells):
    """J = int_D A |grad u|^2 (eq. heat_cost), exact for P1 u."""
    gu = np.einsum("ea,eak->ek", u[cells], grads)
    return float(np.sum(A * vol * np.einsum("ek,ek->e", gu, gu)))


def heat_rhs(coords, cells, A, u, f, lam=0.0, chi=None, V=1.0):
    """Velocity RHS of the heat model (Sec. 6.3) plus lambda times the volume term.

    S0^J = 2 u grad f,   S1^J = (2 u f - A |grad u|^2) I + 2 A grad u (x) grad u,
    S1^C = chi / V I.  u f is integrated exactly with the consistent mass.
    """
    vol, g = fem.geometry(coords, cells)
    d = coords.shape[1]
    ue, fe = u[cells], f[cells]
    gu = np.einsum("ea,eak->ek", ue, g)
    gf = np.einsum("ea,eak->ek", fe, g)
    Me = fem.mass(vol, d)
    uf = np.einsum("ea,eab,eb->e", ue, Me, fe)                   # int_e u f
    S1c = (A * vol)[:, None, None] * (
        -np.einsum("ek,ek->e", gu, gu)[:, None, None] * np.eye(d)[None]
        + 2.0 * np.einsum("ei,ej->eij", gu, gu))
    if chi is not None and lam != 0.0:
        S1c = S1c + (lam * chi * vol / V)[:, None, None] * np.eye(d)[None]
    be = np.einsum("eij,eaj->eai", S1c, g)                        # int_e S1 grad psi_a
    be += 2.0 * uf[:, None, None] * g                             # int_e 2uf I grad psi_a
    Mu = np.einsum("eab,eb->ea", Me, ue)                          # int_e u psi_a
    be += 2.0 * Mu[:, :, None] * gf[:, None, :]                   # int_e 2 u grad f psi_a
    return _scatter(be, cells, coords.shape[0], d)


# ---------------------------------------------------------- elastic model
def strain_stress(grads, ue, lam, mu):
    """Du, eps(u), sigma(u) per element for P1 vector u (Sec. 3)."""
    Du = np.einsum("eai,eaj->eij", ue, grads)                    # (Du)_ij = d_j u_i
    eps = 0.5 * (Du + np.swapaxes(Du, 1, 2))
    d = grads.shape[2]
    tr = np.trace(eps, axis1=1, axis2=2)
    sig = lam * tr[:, None, None] * np.eye(d)[None] + 2.0 * mu * eps
    return Du, eps, sig


def elastic_cost(vol, grads, A, u, cells, lam, mu):
    """J = int_D A sigma(u) : eps(u) (eq. compli_cost)."""
    d = grads.shape[2]
    ue = u.reshape(-1, d)[cells]
    _, eps, sig = strain_stress(grads, ue, lam, mu)
    return float(np.sum(A * vol * np.einsum("eij,eij->e", sig, eps)))


def elastic_rhs(coords, cells, A, u, lam_e, mu_e, lam=0.0, chi=None, V=1.0):
    """Velocity RHS of compliance (Sec. 6.2) plus lambda times the volume term.

    S0^J = 0,  S1^J = A (2 Du^T sigma(u) - sigma(u) : eps(u) I),  S1^C = chi / V I.
    """
    vol, g = fem.geometry(coords, cells)
    d = coords.shape[1]
    ue = u.reshape(-1, d)[cells]
    Du, eps, sig = strain_stress(g, ue, lam_e, mu_e)
    se = np.einsum("eij,eij->e", sig, eps)
    S1 = A[:, None, None] * (2.0 * np.einsum("eki,ekj->eij", Du, sig)
                             - se[:, None, None] * np.eye(d)[None])
    if chi is not None and lam != 0.0:
        S1 = S1 + (lam * chi / V)[:, None, None] * np.eye(d)[None]
    be = vol[:, None, None] * np.einsum("eij,eaj->eai", S1, g)
    return _scatter(be, cells, coords.shape[0], d)


# ------------------------------------------------ screened Helmholtz family
def helmholtz_rhs(coords, cells, A, k, omega, u, f):
    """Velocity RHS of J = int f u for -div(A k grad u) + omega^2 u = f, adjoint p = -u.

    Re-derived from the shape-Lagrangian steps of Sec. 3 (the heat case of
    Sec. 6.3 with the extra zero-order term):
    S0 = 2 u grad f,
    S1 = (2 u f - A k |grad u|^2 - omega^2 u^2) I + 2 A k grad u (x) grad u.
    u f and u^2 are integrated exactly with the consistent mass.
    """
    vol, g = fem.geometry(coords, cells)
    d = coords.shape[1]
    ue, fe = u[cells], f[cells]
    gu = np.einsum("ea,eak->ek", ue, g)
    gf = np.einsum("ea,eak->ek", fe, g)
    Me = fem.mass(vol, d)
    uf = np.einsum("ea,eab,eb->e", ue, Me, fe)
    uu = np.einsum("ea,eab,eb->e", ue, Me, ue)
    Ak = A * k
    S1c = (Ak * vol)[:, None, None] * (
        -np.einsum("ek,ek->e", gu, gu)[:, None, None] * np.eye(d)[None]
        + 2.0 * np.einsum("ei,ej->eij", gu, gu))
    be = np.einsum("eij,eaj->eai", S1c, g)
    be += (2.0 * uf - omega * omega * uu)[:, None, None] * g
    Mu = np.einsum("eab,eb->ea", Me, ue)
    be += 2.0 * Mu[:, :, None] * gf[:, None, :]
    return _scatter(be, cells, coords.shape[0], d)


def volume_rhs(coords, cells, chi, V):
    """Velocity RHS of the volume constraint alone: S1^C = chi / V I."""
    vol, g = fem.geometry(coords, cells)
    d = coords.shape[1]
    be = (chi * vol / V)[:, None, None] * g
    return _scatter(be, cells, coords.shape[0], d)


def _scatter(be, cells, num_nodes, d):
    out = np.zeros((num_nodes, d))
    for a in range(cells.shape[1]):
        np.add.at(out, cells[:, a], be[:, a, :])
    return out.reshape(-1)
