"""Plain FP64 CPU oracle for the level-set shape-optimisation hot path of
arXiv 2601.05709 ("FormOpt": distributed shape derivative + level-set method).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA library never calls it; the two share no code, headers, tables or
constants.  Inputs reach both sides from the seeded generators in
``paper_2601_05709_gb300.workloads`` (which hold none of the method's
arithmetic).

The oracle is written for readability, not speed: numpy arrays over elements,
scipy.sparse assembly of the global matrices, and a sparse direct solve
(SuperLU) wherever the method solves a linear system, so that its answers are
the exact solutions of the discrete systems the paper defines.  A textbook
Jacobi-PCG is kept beside the direct solve for timing and iteration counts.

Module map (paper section / equation each follows):

* ``mesh``      structured Kuhn simplicial mesh of the box D, DOF maps, Dirichlet
                masks, boundary facets, penalised subdomain mask, mesh diameter
                h (Sec. 5.2, 5.6 "mesh diameter", 5.7 "Penalized subdomains").
* ``fem``       P1 element geometry and element matrices: scalar stiffness,
                linear-elastic stiffness (Sec. 3 strain/stress, eq. compli_weak),
                consistent mass, facet mass, load vectors (eqs heat_weak,
                compli_weak).
* ``shape``     ersatz coefficient A_Omega (eqs heat_AOmega, compli_AOmega),
                cost / constraint functionals (eqs heat_cost, compli_cost,
                compli_constr), and the distributed shape-derivative right-hand
                side (Def. 2, eqs dJ1, dC1, S0andS1 and the S-tensors of
                Sec. 6.2 / 6.3).
* ``velocity``  the H1-type velocity equation (eqs velocity, bd_plt, sub_dom,
                compli1_bili).
* ``levelset``  SUPG/Crank-Nicolson transport (eqs transport, weak_transport,
                tau_lv), reinitialisation (eqs Eikonal, HJ, grad_H, weak_HJ) and
                the initial level set (eq. phi0).
* ``ppl``       Proximal-Perturbed Lagrangian update (eqs lagrangian,
                lag_method) and adaptive time stepping (eqs tend, steps).
* ``logistic``  the population model of Sec. 6.4 (eqs log_cost, log_prob, log_KOmega,
                log_weak): Newton state solve, linear adjoint, cost and the S1 tensor.
* ``inverse``   the inverse-elasticity model of Sec. 3 / Sec. 6.1 (eqs cost, w-f, w-g, the two
                adjoints and eq. SDelast_inv) and the Dirichlet extension (Sec. 5.7, eq. dir).
* ``algorithm`` one iteration of Algorithm 1.
* ``solvers``   sparse direct solve, Jacobi-PCG, Jacobi-BiCGStab.

Pins: every function is checked in ``tests/test_oracle_*.py`` against closed
forms, textbook special cases, invariants, brute force and a Taylor test.  The
reinitialisation step (``levelset.reinit_step_system`` / ``reinit``) is pinned
by the closed form of a step from a constant level set, the identity "AB2 with
an equal history = explicit Euler", and a pointwise brute-force evaluation of
one Euler and one AB2 step with finite-difference test-function gradients
(``tests/test_oracle_pins_load_reinit.py``); the traction load
(``fem.facet_load``) by hand-computed facets, subdivision quadrature and the
face sums and first moments.  The logistic model (``logistic``) by the cubic integrals
against a collapsed Gauss product rule, the residual against per-element quadrature, the
Jacobian against central differences of the residual, constant equilibria, quadratic Newton
convergence, the adjoint against a finite-difference source derivative and a Taylor test of
the shape derivative (``tests/test_oracle_logistic.py``).  The inverse-elasticity model
(``inverse``) by Taylor tests of its shape derivative with a linear measurement field, the zero
of the cost, states, adjoints and derivative at the true inclusion, finite-difference checks
of both adjoints through the traction and the measurement, and the Dirichlet extension's patch
test (``tests/test_oracle_inverse.py``).
"""
