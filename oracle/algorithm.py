"""One iteration of Algorithm 1 ("Level set algorithm", Sec. 4) in the oracle.

Order within iteration i (0-based): coefficients from phi^i; state solve (Newton for
the logistic model, Sec. 6.4); adjoint (closed form for the compliance costs: p = -u
for heat, Sec. 6.3, and p = -2u for elasticity, Sec. 6.2, already folded into the S
tensors; a linear solve for the logistic model); cost and
constraint; one PPL update giving lambda (Sec. 5.4); S-assembly; velocity solve
and B(theta, theta); adaptive time; transport to phi^{i+1}; reinitialisation
when reinit_step > 0, i > 0 and i mod reinit_step == 0 (Sec. 5.7).
"""
from dataclasses import dataclass, field

import numpy as np

from . import fem, levelset, logistic, ppl as ppl_mod, shape, solvers, velocity
from .mesh import BoxMesh

HEAT, ELASTIC, HELMHOLTZ, LOGISTIC = 0, 1, 2, 3


@dataclass
class Problem:
    mesh: BoxMesh
    kind: int = HEAT
    a_in: float = 1.0
    a_out: float = 1e-3
    E: float = 1.0
    nu: float = 0.3
    dirichlet_faces: list = field(default_factory=list)     # [(axis, side)]
    f_nodal: np.ndarray = None                               # heat / Helmholtz body source
    point_loads: list = field(default_factory=list)          # [(node, vector)]
    tractions: list = field(default_factory=list)            # [(axis, side, vector)]
    volume_target: float = 0.0                               # V; 0 = unconstrained
    k: float = 1.0                                           # Helmholtz conductivity factor
    omega: float = 0.0                                       # Helmholtz zero-order coefficient
    vform: velocity.VelocityForm = field(default_factory=velocity.VelocityForm)
    coef_rule: str = "centroid"                              # or "cut": exact cut-cell fraction
    # Several load cases (eq. compli_plus: J = sum_k J(u_k), u_k the state of load case k):
    # a list of (point_loads, tractions) per case; None = the single case above.  f_nodal
    # belongs to case 0.
    load_cases: list = None
    # Several volume constraints C_j = |Omega cap R_j| / V_j (Sec. 5.4 with N_c = len), R_j a
    # box (lo, hi) with strict inequalities on the element centroid; None = |Omega| / V.
    volume_regions: list = None
    # Logistic population model (Sec. 6.4): growth rate r, initial Newton guess u_init (None:
    # u = a_in); the carrying capacity is the element coefficient (a_in inside, a_out outside).
    growth_rate: float = 0.0
    u_init: np.ndarray = None

    @property
    def ncomp(self):
        return self.mesh.dim if self.kind == ELASTIC else 1

    def dirichlet(self):
        return self.mesh.dirichlet_mask(self.dirichlet_faces, self.ncomp)

    def load(self):
        m = self.mesh
        n = m.num_nodes * self.ncomp
        F = np.zeros(n)
        if self.kind in (HEAT, HELMHOLTZ) and self.f_nodal is not None:
            F += fem.body_load(m.coords, m.cells, self.f_nodal)
        for node, vec in self.point_loads:
            for c in range(self.ncomp):
                F[node * self.ncomp + c] += vec[c]
        for axis, side, vec in self.tractions:
            F += fem.facet_load(m.coords, m.boundary_facets(axis, side), vec, self.ncomp)
        F[self.dirichlet() == 1] = 0.0
        return F

    # ---- several load cases and constraints (Sec. 5.4, eq. compli_plus) --------------
    def cases(self):
        if self.load_cases is None:
            return [(self.point_loads, self.tractions)]
        return self.load_cases

    def case_load(self, k):
        """F_k: f (case 0 only), case k's point loads and tractions; zero on Dirichlet DOFs."""
        m = self.mesh
        F = np.zeros(m.num_nodes * self.ncomp)
        if k == 0 and self.kind in (HEAT, HELMHOLTZ) and self.f_nodal is not None:
            F += fem.body_load(m.coords, m.cells, self.f_nodal)
        pts, trs = self.cases()[k]
        for node, vec in pts:
            for c in range(self.ncomp):
                F[node * self.ncomp + c] += vec[c]
        for axis, side, vec in trs:
            F += fem.facet_load(m.coords, m.boundary_facets(axis, side), vec, self.ncomp)
        F[self.dirichlet() == 1] = 0.0
        return F

    def coefficients(self, phi):
        if self.coef_rule == "cut":
            return shape.coefficient_cut(phi, self.mesh.cells, self.a_in, self.a_out)
        return shape.coefficient(phi, self.mesh.cells, self.a_in, self.a_out)

    def states(self, phi):
        """U [n_cases, N_dof]: the state of every load case, with A_e and chi_e."""
        A, chi = self.coefficients(phi)
        K = self.stiffness(A)
        free = self.dirichlet() == 0
        U = np.stack([solvers.solve_free(K, self.case_load(k), free) for k in range(len(self.cases()))])
        return U, A, chi

    def total_cost(self, U, A):
        """J = sum over the load cases (eq. compli_plus)."""
        return float(sum(self.cost_of(U[k], A, k) for k in range(U.shape[0])))

    def cost_of(self, u, A, k):
        m = self.mesh
        vol, g = fem.geometry(m.coords, m.cells)
        if self.kind == ELASTIC:
            lam, mu = fem.lame(self.E, self.nu)
            return shape.elastic_cost(vol, g, A, u, m.cells, lam, mu)
        if self.kind == HEAT:
            return shape.heat_cost(vol, g, A, u, m.cells)
        return float(self.case_load(k) @ u)

    def regions(self):
        """[(region mask per element, V_j)] of the constraints."""
        if self.volume_regions is None:
            return [(np.ones(self.mesh.num_elems), self.volume_target)] if self.volume_target > 0 else []
        return [(self.mesh.subdomain_mask([(lo, hi)]).astype(np.float64), V) for lo, hi, V in self.volume_regions]

    def constraints(self, chi):
        """C_j = int_{R_j} chi / V_j for every constraint j."""
        vol, _ = fem.geometry(self.mesh.coords, self.mesh.cells)
        return np.array([shape.volume(vol, chi * r) / V for r, V in self.regions()])

    def total_rhs(self, U, A, chi, lams):
        """b = sum_k b^J(u_k) + sum_j lambda_j b^C_j, b^C_j the term of S1^C_j = chi chi_Rj / V_j I."""
        m = self.mesh
        b = np.zeros(m.dim * m.num_nodes)
        for k in range(U.shape[0]):
            if self.kind == HEAT and k > 0:      # f belongs to case 0: S0 = 2u grad f, 2uf vanish
                saved, self.f_nodal = self.f_nodal, None
                b += self.rhs(U[k], A, chi, 0.0)
                self.f_nodal = saved
            else:
                b += self.rhs(U[k], A, chi, 0.0)
        for (r, V), lam in zip(self.regions(), lams):
            if lam != 0.0:
                b += lam * shape.volume_rhs(m.coords, m.cells, chi * r, V)
        return b

    def stiffness(self, A):
        m = self.mesh
        vol, g = fem.geometry(m.coords, m.cells)
        if self.kind == ELASTIC:
            lam, mu = fem.lame(self.E, self.nu)
            Ke = fem.elastic_stiffness(vol, g, A, lam, mu)
        else:
            Ke = fem.scalar_stiffness(vol, g, A * self.k)
            if self.kind == HELMHOLTZ and self.omega != 0.0:
                Ke = Ke + self.omega**2 * fem.mass(vol, m.dim)
        return fem.assemble(Ke, fem.element_dofs(m.cells, self.ncomp), m.num_nodes * self.ncomp)

    def logistic_state(self, phi):
        """Newton solution u, carrying capacity K_e and chi_e (Sec. 6.4)."""
        m = self.mesh
        K, chi = shape.coefficient(phi, m.cells, self.a_in, self.a_out)
        u0 = self.u_init if self.u_init is not None else np.full(m.num_nodes, self.a_in)
        u, _ = logistic.newton(m.coords, m.cells, K, self.growth_rate, u0)
        return u, K, chi

    def state(self, phi):
        if self.kind == LOGISTIC:
            return self.logistic_state(phi)
        if self.coef_rule == "cut":
            A, chi = shape.coefficient_cut(phi, self.mesh.cells, self.a_in, self.a_out)
        else:
            A, chi = shape.coefficient(phi, self.mesh.cells, self.a_in, self.a_out)
        K = self.stiffness(A)
        u = solvers.solve_free(K, self.load(), self.dirichlet() == 0)
        return u, A, chi

    def cost(self, u, A):
        m = self.mesh
        if self.kind == LOGISTIC:
            return logistic.cost(m.coords, m.cells, u)
        vol, g = fem.geometry(m.coords, m.cells)
        if self.kind == ELASTIC:
            lam, mu = fem.lame(self.E, self.nu)
            return shape.elastic_cost(vol, g, A, u, m.cells, lam, mu)
        if self.kind == HEAT:
            return shape.heat_cost(vol, g, A, u, m.cells)
        return float(self.load() @ u)                      # J = int f u

    def constraint(self, chi):
        vol, _ = fem.geometry(self.mesh.coords, self.mesh.cells)
        return shape.volume(vol, chi) / self.volume_target

    def rhs(self, u, A, chi, lam):
        m = self.mesh
        V = self.volume_target if self.volume_target > 0 else 1.0
        if self.kind == LOGISTIC:      # the adjoint is a linear solve of its own (Sec. 6.4)
            p = logistic.adjoint(m.coords, m.cells, A, self.growth_rate, u)
            return logistic.rhs(m.coords, m.cells, A, self.growth_rate, u, p, lam, chi, V)
        if self.kind == ELASTIC:
            le, me = fem.lame(self.E, self.nu)
            return shape.elastic_rhs(m.coords, m.cells, A, u, le, me, lam, chi, V)
        if self.kind == HEAT:
            f = self.f_nodal if self.f_nodal is not None else np.zeros(m.num_nodes)
            return shape.heat_rhs(m.coords, m.cells, A, u, f, lam, chi, V)
        b = shape.helmholtz_rhs(m.coords, m.cells, A, self.k, self.omega, u, self.f_nodal)
        if lam != 0.0:
            b = b + lam * shape.volume_rhs(m.coords, m.cells, chi, V)
        return b


@dataclass
class RunOptions:
    """Run parameters of runDP / runTP / runMP (Sec. 5.1) used by one iteration."""
    dfactor: float = 1e-2
    lv_time: tuple = (1e-3, 1e-1)
    lv_iter: tuple = (8, 16)
    smooth: bool = False
    reinit_step: int = 0
    reinit_pars: tuple = (8, 1e-1)
    h: float = None


def opt_step_multi(prob, phi, i, ppl_state, opts):
    """One iteration of Algorithm 1 with several load cases and / or constraints: the states of
    every case, J = sum of their costs, C_j per constraint, one PPL update of the vector C, and
    b = sum_k b^J(u_k) + sum_j lambda_j b^C_j (eq. S0andS1 with N_c constraints)."""
    h = opts.h if opts.h is not None else prob.mesh.diameter()
    U, A, chi = prob.states(phi)
    J = prob.total_cost(U, A)
    C = prob.constraints(chi)
    lams, L = np.zeros(len(C)), J
    if len(C):
        lams, L = ppl_state.update(C, J)
    b = prob.total_rhs(U, A, chi, lams)
    theta, Btt = velocity.solve(prob.mesh, prob.vform, b)
    t_end, ns = ppl_mod.adaptime(Btt, opts.dfactor, opts.lv_time, opts.lv_iter)
    phi_new = levelset.transport(prob.mesh, phi, theta, t_end, ns, h, opts.smooth)
    reinit_done = False
    if opts.reinit_step and i > 0 and i % opts.reinit_step == 0:
        phi_new = levelset.reinit(prob.mesh, phi_new, opts.reinit_pars[0], opts.reinit_pars[1], h)
        reinit_done = True
    return phi_new, dict(J=J, C=C, L=L, lam=lams, Btt=Btt, t_end=t_end, nsteps=ns, reinit=reinit_done, U=U,
                         theta=theta, rhs=b)


def opt_step(prob, phi, i, ppl_state, opts):
    """One iteration of Algorithm 1; returns (phi^{i+1}, log dict)."""
    if prob.load_cases is not None or prob.volume_regions is not None:
        return opt_step_multi(prob, phi, i, ppl_state, opts)
    h = opts.h if opts.h is not None else prob.mesh.diameter()
    u, A, chi = prob.state(phi)
    J = prob.cost(u, A)
    lam, L, C = 0.0, J, None
    if prob.volume_target > 0:
        C = prob.constraint(chi)
        lam_v, L = ppl_state.update([C], J)
        lam = float(lam_v[0])
    b = prob.rhs(u, A, chi, lam)
    theta, Btt = velocity.solve(prob.mesh, prob.vform, b)
    t_end, ns = ppl_mod.adaptime(Btt, opts.dfactor, opts.lv_time, opts.lv_iter)
    phi_new = levelset.transport(prob.mesh, phi, theta, t_end, ns, h, opts.smooth)
    reinit_done = False
    if opts.reinit_step and i > 0 and i % opts.reinit_step == 0:
        phi_new = levelset.reinit(prob.mesh, phi_new, opts.reinit_pars[0], opts.reinit_pars[1], h)
        reinit_done = True
    log = dict(J=J, C=C, L=L, lam=lam, Btt=Btt, t_end=t_end, nsteps=ns, reinit=reinit_done,
               u=u, theta=theta, rhs=b)
    return phi_new, log
