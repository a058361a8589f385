"""Task-parallel family of state problems on one mesh (oracle; test infrastructure only).

Sec. 5.3 (task parallelism) solves a set of state equations that differ only in their
parameters, each on its own copy of the mesh, and forms the velocity and the level-set
update once from all of them.  The family here is the screened Helmholtz problem of
each instance i < n,

    -div(A k_i grad u_i) + omega_i^2 u_i = f_i  in D,   u_i = 0 on the Dirichlet faces,

sharing the mesh, phi and hence the ersatz coefficient A_e.  The cost is the sum
J = sum_i J_i with J_i = int f_i u_i; each J_i is self-adjoint (p_i = -u_i), so the
distributed shape derivative of J is the sum of the per-instance tensors S0, S1 and the
velocity right-hand side is b = sum_i b_i (plus lambda times the volume term once, when
a volume constraint is present).  Every per-instance quantity is the single-problem
oracle of algorithm.Problem with kind HELMHOLTZ; this module only adds the sums.
"""
from dataclasses import dataclass, field

import numpy as np

from . import shape
from .algorithm import HELMHOLTZ, Problem
from .mesh import BoxMesh
from . import velocity


@dataclass
class Batch:
    mesh: BoxMesh
    k: np.ndarray                 # [n] conductivity factors k_i
    omega: np.ndarray             # [n] zero-order coefficients omega_i
    f_nodal: np.ndarray           # [n, N_n] nodal sources f_i
    dirichlet_faces: list = field(default_factory=list)
    a_in: float = 1.0
    a_out: float = 1e-3
    volume_target: float = 0.0
    vform: velocity.VelocityForm = field(default_factory=velocity.VelocityForm)

    @property
    def n_inst(self):
        return len(self.k)

    def problem(self, i):
        """The single-instance problem i."""
        return Problem(self.mesh, HELMHOLTZ, a_in=self.a_in, a_out=self.a_out,
                       dirichlet_faces=list(self.dirichlet_faces), f_nodal=np.asarray(self.f_nodal[i], float),
                       k=float(self.k[i]), omega=float(self.omega[i]), volume_target=self.volume_target,
                       vform=self.vform)

    def state(self, phi):
        """U[:, i] = u_i (instance-minor, [N_n, n]), with A_e and chi_e."""
        cols = []
        A = chi = None
        for i in range(self.n_inst):
            u, A, chi = self.problem(i).state(phi)
            cols.append(u)
        return np.stack(cols, axis=1), A, chi

    def loads(self):
        """F[:, i] = int f_i psi_a with the Dirichlet rows zeroed ([N_n, n])."""
        return np.stack([self.problem(i).load() for i in range(self.n_inst)], axis=1)

    def costs(self, U, A):
        """J_i = int f_i u_i for every instance."""
        return np.array([self.problem(i).cost(U[:, i], A) for i in range(self.n_inst)])

    def cost(self, U, A):
        return float(np.sum(self.costs(U, A)))

    def rhs(self, U, A, chi, lam=0.0):
        """b = sum_i b_i (+ lambda * volume term), interleaved [d * N_n]."""
        b = np.zeros(self.mesh.dim * self.mesh.num_nodes)
        for i in range(self.n_inst):
            b += self.problem(i).rhs(U[:, i], A, chi, 0.0)
        if lam != 0.0:
            V = self.volume_target if self.volume_target > 0 else 1.0
            b += lam * shape.volume_rhs(self.mesh.coords, self.mesh.cells, chi, V)
        return b
