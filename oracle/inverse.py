"""Inverse elasticity by a Kohn-Vogelius-type cost (oracle; Sec. 3 model problem, Sec. 6.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For each force-displacement pair (f_k, g_k) (Sec. 6.1 sums the cost over the pairs):
  u: find u in H^1_{Gamma0}(D)^d with  int A sigma(u):eps(w) = int_{Gamma1} f . w   (eq. w-f),
  v: find v in H^1_0(D)^d with         int A sigma(v + g):eps(w) = 0              (eq. w-g),
     g the extension of the measured displacement into D, y = v + g;
  J = alpha/2 int_D |u - v - g|^2 + beta/2 int_{Gamma1} |u - g|^2                  (eq. cost),
  p in H^1_{Gamma0}: int A sigma(p):eps(r) = -alpha int (u - v - g).r - beta int_{Gamma1} (u - g).r,
  q in H^1_0:        int A sigma(q):eps(r) =  alpha int (u - v - g).r,
  S0 = -alpha Dg^T (u - v - g) + A sum_ij sigma(q)_ij grad(eps(g)_ij)   (the second term is zero
       for a P1 g: eps(g) is constant on each element),
  S1 = (alpha/2 |u - v - g|^2 + A sigma(u):eps(p) + A sigma(v + g):eps(q)) I
       - A (Du^T sigma(p) + Dp^T sigma(u)) - A (Dv^T sigma(q) + Dq^T sigma(v + g))   (eq. SDelast_inv).
A = kappa chi_Omega + chi_{D \\ Omega} (eq. AOmega) per element by the one-point rule; Gamma1 is
the union of the listed faces of the box, Gamma0 the Dirichlet faces.  Every integral is exact
for P1 data (consistent volume and facet mass matrices).

Dirichlet extension (Sec. 5.7): eta with int D eta : D zeta = 0 for zeta vanishing on Gamma_sub
and eta = the given values on Gamma_sub (natural condition elsewhere).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, shape, solvers


def _vec(cells, d):
    return fem.element_dofs(cells, d)


def elastic_matrix(coords, cells, A, lam, mu):
    vol, g = fem.geometry(coords, cells)
    d = coords.shape[1]
    return fem.assemble(fem.elastic_stiffness(vol, g, A, lam, mu), _vec(cells, d), coords.size)


def vector_mass(coords, cells):
    """Consistent P1 mass acting on every component (interleaved DOFs)."""
    vol, _ = fem.geometry(coords, cells)
    d = coords.shape[1]
    Me = fem.mass(vol, d)
    Mv = np.einsum("eab,ij->eaibj", Me, np.eye(d)).reshape(cells.shape[0], (d + 1) * d, (d + 1) * d)
    return fem.assemble(Mv, _vec(cells, d), coords.size)


def facet_vector_mass(coords, facets):
    d = coords.shape[1]
    Mf = fem.facet_mass(coords, facets)
    k = facets.shape[1]
    Mv = np.einsum("eab,ij->eaibj", Mf, np.eye(d)).reshape(facets.shape[0], k * d, k * d)
    return fem.assemble(Mv, _vec(facets, d), coords.size)


def gamma_facets(mesh, faces):
    return np.concatenate([mesh.boundary_facets(a, s) for a, s in faces], axis=0)


def boundary_dofs(mesh):
    on = np.zeros(mesh.num_nodes, dtype=bool)
    for a in range(mesh.dim):
        on |= mesh.face_nodes(a, 0) | mesh.face_nodes(a, 1)
    return np.repeat(on, mesh.dim)


def states(mesh, K, F, g, dir0):
    """u (Gamma0 clamped, load F) and v (zero on the boundary, K (v + g) = 0 inside)."""
    u = solvers.solve_free(K, F, dir0 == 0)
    inner = ~boundary_dofs(mesh)
    v = solvers.solve_free(K, -(K @ g), inner)
    return u, v


def cost(M, Mg, u, v, g, alpha, beta):
    w = u - v - g
    e = u - g
    return float(0.5 * alpha * (w @ (M @ w)) + 0.5 * beta * (e @ (Mg @ e)))


def adjoints(mesh, K, M, Mg, u, v, g, alpha, beta, dir0):
    w = u - v - g
    p = solvers.solve_free(K, -alpha * (M @ w) - beta * (Mg @ (u - g)), dir0 == 0)
    q = solvers.solve_free(K, alpha * (M @ w), ~boundary_dofs(mesh))
    return p, q


def rhs(coords, cells, A, lam, mu, u, v, p, q, g, alpha):
    """b[d a + k] = sum_e int_e S0_k psi_a + (S1 grad psi_a)_k."""
    vol, gr = fem.geometry(coords, cells)
    d = coords.shape[1]
    c = cells.astype(np.int64)

    def fields(x):
        return shape.strain_stress(gr, x.reshape(-1, d)[c], lam, mu)

    Du, eu, su = fields(u)
    Dv, ev, sv = fields(v)
    Dp, ep, sp_ = fields(p)
    Dq, eq, sq = fields(q)
    Dvg, evg, svg = fields(v + g)
    Dg = np.einsum("eai,eaj->eij", g.reshape(-1, d)[c], gr)          # (Dg)_ij = d_j g_i
    we = (u - v - g).reshape(-1, d)[c]                                # [NT, d+1, d]
    Me = fem.mass(vol, d)
    ww = np.einsum("eai,eab,ebi->e", we, Me, we)                      # int_e |w|^2
    scal = 0.5 * alpha * ww + A * vol * (np.einsum("eij,eij->e", su, ep) + np.einsum("eij,eij->e", svg, eq))
    tens = (np.einsum("eki,ekj->eij", Du, sp_) + np.einsum("eki,ekj->eij", Dp, su)
            + np.einsum("eki,ekj->eij", Dv, sq) + np.einsum("eki,ekj->eij", Dq, svg))
    S1 = scal[:, None, None] * np.eye(d)[None] - (A * vol)[:, None, None] * tens
    be = np.einsum("eij,eaj->eai", S1, gr)
    Mw = np.einsum("eab,ebj->eaj", Me, we)                            # int_e w_j psi_a
    be += -alpha * np.einsum("ejk,eaj->eak", Dg, Mw)                  # int_e S0_k psi_a
    out = np.zeros((coords.shape[0], d))
    for a in range(cells.shape[1]):
        np.add.at(out, c[:, a], be[:, a, :])
    return out.reshape(-1)


def dirichlet_extension(mesh, values, faces):
    """eta = values on the nodes of the listed faces, int D eta : D zeta = 0 otherwise."""
    vol, gr = fem.geometry(mesh.coords, mesh.cells)
    L = fem.assemble(fem.scalar_stiffness(vol, gr, np.ones_like(vol)), mesh.cells.astype(np.int64), mesh.num_nodes)
    fixed = np.zeros(mesh.num_nodes, dtype=bool)
    for a, s in faces:
        fixed |= mesh.face_nodes(a, s)
    free = ~fixed
    d = mesh.dim
    V = values.reshape(-1, d)
    eta = np.zeros_like(V)
    Lff = sp.csc_matrix(L[free][:, free])
    Lfx = L[free][:, fixed]
    for k in range(d):
        eta[fixed, k] = V[fixed, k]
        eta[free, k] = spla.spsolve(Lff, -(Lfx @ V[fixed, k]))
    return eta.reshape(-1)
