"""P1 finite-element building blocks on general simplices (oracle).

Everything is computed from the vertex coordinates of each element (no use of
the structured-grid layout), so the same code serves moved meshes in the
Taylor test of the shape derivative.
"""
import math

import numpy as np
import scipy.sparse as sp


def geometry(coords, cells):
    """Measure |e| and barycentric gradients of every simplex.

    With edge matrix E = [x_1 - x_0, ..., x_d - x_0] (columns), the barycentric
    coordinates lambda_1..lambda_d are the rows of E^{-1} applied to x - x_0, so
    grad lambda_m is row m of E^{-1} and grad lambda_0 = -sum_m grad lambda_m.
    Returns vol [NT] and grads [NT, d+1, d] (grads[e, a, k] = d psi_a / d x_k).
    """
    X = coords[cells]                                   # [NT, d+1, d]
    d = X.shape[2]
    E = np.swapaxes(X[:, 1:, :] - X[:, :1, :], 1, 2)    # [NT, d, d], columns = edges
    vol = np.abs(np.linalg.det(E)) / math.factorial(d)
    Einv = np.linalg.inv(E)
    grads = np.concatenate([-Einv.sum(axis=1, keepdims=True), Einv], axis=1)
    return vol, grads


def lame(E, nu):
    """Lame parameters of an isotropic material, plane strain in 2D.

    sigma(w) = lambda tr(eps(w)) I + 2 mu eps(w) (Sec. 3, stress/strain) written
    with d = 2 is the plane-strain law.
    """
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def scalar_stiffness(vol, grads, coef):
    """K_e[a, b] = coef_e |e| grad psi_a . grad psi_b  (eq. heat_weak)."""
    return (coef * vol)[:, None, None] * np.einsum("eak,ebk->eab", grads, grads)


def elastic_stiffness(vol, grads, coef, lam, mu):
    """K_e[(a,i),(b,j)] = coef_e int_e sigma(psi_b e_j) : eps(psi_a e_i)  (eq. compli_weak).

    With eps(psi_b e_j) = sym(e_j (x) grad psi_b):
    sigma(psi_b e_j) : eps(psi_a e_i) =
        lam d_i psi_a d_j psi_b + mu d_j psi_a d_i psi_b + mu delta_ij grad psi_a . grad psi_b.
    Returned with DOF order (a, i) -> a*d + i, shape [NT, (d+1)d, (d+1)d].
    """
    NT, n1, d = grads.shape
    g = grads
    dot = np.einsum("eak,ebk->eab", g, g)
    K = (lam * np.einsum("eai,ebj->eaibj", g, g)
         + mu * np.einsum("eaj,ebi->eaibj", g, g)
         + mu * np.einsum("eab,ij->eaibj", dot, np.eye(d)))
    K *= (coef * vol)[:, None, None, None, None]
    return K.reshape(NT, n1 * d, n1 * d)


def mass(vol, d, coef=None):
    """Consistent P1 mass: M_e[a, b] = |e| (1 + delta_ab) / ((d+1)(d+2))."""
    n1 = d + 1
    ref = (np.ones((n1, n1)) + np.eye(n1)) / (n1 * (n1 + 1))
    w = vol if coef is None else vol * coef
    return w[:, None, None] * ref[None, :, :]


def facet_measure(coords, facets):
    """Length (2D segments) or area (3D triangles) of boundary facets."""
    X = coords[facets]
    if X.shape[2] == 2:
        return np.linalg.norm(X[:, 1] - X[:, 0], axis=1)
    return 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1)


def facet_mass(coords, facets):
    """Consistent P1 mass on (d-1)-simplices: |f| (1 + delta_ab) / (d (d+1))."""
    k = facets.shape[1]                                 # = d vertices
    ref = (np.ones((k, k)) + np.eye(k)) / (k * (k + 1))
    return facet_measure(coords, facets)[:, None, None] * ref[None, :, :]


def element_dofs(cells, ncomp):
    """Global DOF numbers of each element: node*ncomp + comp, order (a, comp)."""
    if ncomp == 1:
        return cells.astype(np.int64)
    base = cells.astype(np.int64)[:, :, None] * ncomp + np.arange(ncomp)[None, None, :]
    return base.reshape(cells.shape[0], -1)


def assemble(Ke, dofs, n):
    """Sum element matrices Ke [NE, k, k] with DOF lists [NE, k] into an n x n CSR."""
    k = dofs.shape[1]
    rows = np.repeat(dofs, k, axis=1).ravel()
    cols = np.tile(dofs, (1, k)).ravel()
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def assemble_vector(Fe, dofs, n):
    """Sum element vectors Fe [NE, k] into a length-n vector."""
    out = np.zeros(n)
    np.add.at(out, dofs.ravel(), Fe.ravel())
    return out


def facet_load(coords, facets, traction, ncomp):
    """int_{Gamma_1} t . psi_a for a constant traction t: t |f| / d at each facet vertex."""
    d = facets.shape[1]
    n = coords.shape[0] * ncomp
    w = facet_measure(coords, facets) / d
    Fe = w[:, None, None] * np.asarray(traction, dtype=np.float64)[None, None, :]
    Fe = np.broadcast_to(Fe, (facets.shape[0], d, ncomp)).reshape(facets.shape[0], -1)
    return assemble_vector(Fe, element_dofs(facets, ncomp), n)


def body_load(coords, cells, f_nodal):
    """int_D f psi_a with f the P1 interpolant of nodal values: F = M f."""
    vol, _ = geometry(coords, cells)
    Me = mass(vol, coords.shape[1])
    Fe = np.einsum("eab,eb->ea", Me, f_nodal[cells])
    return assemble_vector(Fe, cells.astype(np.int64), coords.shape[0])
