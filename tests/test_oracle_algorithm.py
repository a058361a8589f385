"""One Algorithm-1 iteration of the oracle end to end on small versions of the workloads."""
import numpy as np

from oracle import levelset
from oracle.algorithm import ELASTIC, HEAT, Problem, RunOptions, opt_step
from oracle.mesh import BoxMesh
from oracle.ppl import PPL
from oracle.velocity import VelocityForm
from paper_2601_05709_gb300 import workloads


def test_heat_iteration_decreases_cost():
    m = BoxMesh(2, (32, 32), (0, 0), (1, 1))
    prob = Problem(mesh=m, kind=HEAT, dirichlet_faces=[(0, 0)], f_nodal=np.ones(m.num_nodes),
                   vform=VelocityForm(alpha_mass=0.01, dirichlet=True))
    phi = workloads.phi_cos(m.coords)
    phi1, log = opt_step(prob, phi, 0, PPL(0), RunOptions())
    assert log["Btt"] > 0 and 8 <= log["nsteps"] <= 16
    assert abs(log["Btt"] + log["rhs"] @ log["theta"]) < 1e-12 * log["Btt"]
    u1, A1, _ = prob.state(phi1)
    assert prob.cost(u1, A1) < log["J"]          # a descent step on the thermal compliance


def test_cantilever_iterations_with_ppl_and_reinit():
    m = BoxMesh(2, (32, 16), (0, 0), (2, 1))
    c, r = workloads.hole_lattice()
    phi = levelset.initial_level(m.coords, c, r)
    prob = Problem(mesh=m, kind=ELASTIC, dirichlet_faces=[(0, 0)],
                   point_loads=[(int(m.node_id(np.array([32, 8]))), (0.0, -1.0))], volume_target=1.0,
                   vform=VelocityForm(alpha_mass=0.1, normal_penalty=1e4, omega0_weight=1e4,
                                      omega0_boxes=[((1.95, 0.42), (np.inf, 0.58))]))
    opts = RunOptions(dfactor=1e-1, smooth=True, reinit_step=1, reinit_pars=(4, 0.05))
    ppl = PPL(1)
    logs = []
    for i in range(3):
        phi, log = opt_step(prob, phi, i, ppl, opts)
        logs.append(log)
    assert logs[0]["reinit"] is False and logs[1]["reinit"] is True
    assert all(np.isfinite(l["J"]) and l["Btt"] > 0 for l in logs)
    assert logs[0]["C"] > 0.5
