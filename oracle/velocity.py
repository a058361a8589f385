"""Velocity (descent-direction) equation of the oracle (Sec. 5.5).

Find theta in H with B(theta, xi) = -int_D S0 . xi + S1 : D xi  (eq. velocity), with
    B(theta, xi) = alpha_m int_D theta . xi + int_D D theta : D xi
                 + gamma_b int_{dD} (theta . n)(xi . n)          (eq. bd_plt)
                 + gamma_0 int_D chi_{Omega_0} theta . xi       (eq. sub_dom)
and H = H^1(D)^d, or H^1_0(D)^d when ``dirichlet`` is set (eq. compli1_bili is
the instance alpha_m = 0.1, gamma_b = gamma_0 = 1e4).  On the faces of an
axis-aligned box n = +-e_a, so the boundary term couples only component a of
theta on the two faces normal to e_a, and B splits into d scalar forms.
"""
from dataclasses import dataclass, field

import numpy as np

from . import fem, solvers


@dataclass
class VelocityForm:
    alpha_mass: float = 0.1
    normal_penalty: float = 0.0           # gamma_b
    omega0_weight: float = 0.0            # gamma_0
    omega0_boxes: list = field(default_factory=list)
    dirichlet: bool = False               # H^1_0(D)^d


def component_matrix(mesh, form, comp):
    """Assembled scalar form B_comp (N_n x N_n CSR) acting on theta_comp."""
    vol, g = fem.geometry(mesh.coords, mesh.cells)
    d = mesh.dim
    cells = mesh.cells.astype(np.int64)
    Ke = fem.scalar_stiffness(vol, g, np.ones_like(vol))
    Ke = Ke + form.alpha_mass * fem.mass(vol, d)
    if form.omega0_weight != 0.0 and form.omega0_boxes:
        chi0 = mesh.subdomain_mask(form.omega0_boxes).astype(np.float64)
        Ke = Ke + form.omega0_weight * fem.mass(vol, d, chi0)
    B = fem.assemble(Ke, cells, mesh.num_nodes)
    if form.normal_penalty != 0.0:
        for side in (0, 1):
            facets = mesh.boundary_facets(comp, side)
            Mf = fem.facet_mass(mesh.coords, facets)
            B = B + form.normal_penalty * fem.assemble(Mf, facets.astype(np.int64), mesh.num_nodes)
    return B.tocsr()


def free_nodes(mesh, form):
    if not form.dirichlet:
        return np.ones(mesh.num_nodes, dtype=bool)
    on = np.zeros(mesh.num_nodes, dtype=bool)
    for a in range(mesh.dim):
        on |= mesh.face_nodes(a, 0) | mesh.face_nodes(a, 1)
    return ~on


def solve(mesh, form, b):
    """theta = B^{-1}(-b) per component; returns (theta interleaved, B(theta, theta) = -b . theta)."""
    d = mesh.dim
    b2 = b.reshape(-1, d)
    theta = np.zeros_like(b2)
    free = free_nodes(mesh, form)
    for a in range(d):
        Ba = component_matrix(mesh, form, a)
        theta[:, a] = solvers.solve_free(Ba, -b2[:, a], free)
    theta = theta.reshape(-1)
    return theta, float(-(b @ theta))


def bilinear(mesh, form, theta):
    """B(theta, theta) evaluated with the assembled form (for tests)."""
    d = mesh.dim
    t2 = theta.reshape(-1, d)
    return float(sum(t2[:, a] @ (component_matrix(mesh, form, a) @ t2[:, a]) for a in range(d)))
