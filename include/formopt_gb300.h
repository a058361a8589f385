/*
 * formopt_gb300.h -- C ABI of the GB300 (sm_103a) level-set shape-optimisation hot path.
 *
 * The library computes one iteration of the level-set algorithm of arXiv 2601.05709
 * (Algorithm 1, Sec. 4) on a fixed simplicial mesh -- a structured Kuhn mesh of a box D
 * (fo_mesh_box) or a general mesh given as arrays (fo_mesh_from_arrays) -- with P1 finite
 * elements:
 *   state solve with the ersatz coefficient A_Omega(phi)     (Sec. 6.2 eq. compli_weak,
 *                                                             Sec. 6.3 eq. heat_weak)
 *   cost and volume constraint                               (eqs compli_cost, heat_cost,
 *                                                             compli_constr)
 *   distributed shape derivative (S0, S1) assembled into the velocity right-hand side
 *                                                            (Def. 2, eqs dJ1, dC1, S0andS1)
 *   H1-type velocity solve for the descent direction theta   (Sec. 5.5, eq. velocity)
 *   SUPG / Crank-Nicolson level-set transport                (Sec. 5.6, eq. weak_transport)
 *   reinitialisation                                         (Sec. 5.7, eq. weak_HJ)
 *   Proximal-Perturbed Lagrangian constraint update, on the host (Sec. 5.4, eq. lag_method)
 *
 * Conventions
 *   - Every call returns fo_status (0 = FO_OK, negative = error).  No C++ exception crosses
 *     the ABI.  fo_last_error(ctx) gives a message for the last failing call on that
 *     context; the string is owned by the context and valid until its next call.
 *   - A context owns every device allocation made for it (meshes, problems, scratch); the
 *     matching _destroy call, or fo_ctx_destroy, frees them.  Handles die with the context.
 *   - Device work is enqueued on the context's stream (the one given to fo_ctx_create, or a
 *     stream the context creates).  Calls that return host values (fo_functionals,
 *     fo_descent's B(theta, theta), fo_get, stats) synchronise that stream.
 *   - Host arrays passed in are copied before the call returns.  Where a call takes
 *     `on_device`, a nonzero value means the pointer is device memory on the context's
 *     device (for example a torch tensor's data_ptr()); the caller keeps ownership.
 *   - A context is not thread-safe: use one context per host thread.
 *   - Mesh layout.  Node (i, j, k) has id i + (nx+1)(j + (ny+1)k) and coordinate
 *     lo_a + (hi_a - lo_a) * i_a / n_a.  Cell (i, j, k) has id c = i + nx(j + ny k) and holds
 *     d! simplices d!*c + p, one per permutation pi of the axes in lexicographic order, with
 *     vertices v_0 = cell corner, v_{m+1} = v_m + e_{pi_m}.  Scalar DOF = node; vector DOF =
 *     d*node + component.  Faces are numbered 2*axis + side (side 0: x_axis = lo, 1: = hi).
 */
#ifndef FORMOPT_GB300_H
#define FORMOPT_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FO_API __attribute__((visibility("default")))
#else
#define FO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int fo_status;
#define FO_OK              0
#define FO_EINVAL         -1   /* bad argument (null pointer, size, enum)                    */
#define FO_ENOMEM         -2   /* cudaMalloc failed                                         */
#define FO_ENOMEM_BUDGET  -3   /* the allocation would exceed the context's memory budget   */
#define FO_ECUDA          -4   /* a CUDA runtime call failed; see fo_last_error             */
#define FO_ENOCONV        -5   /* a Krylov solve hit maxit; the result is written, stats say why */
#define FO_ENAN           -6   /* NaN or Inf found in an input or a residual                */
#define FO_ETIMEOUT       -7   /* a bounded device wait gave up (grid barrier) or fo_wait timed out */
#define FO_EBUSY          -8   /* queue full (serving)                                      */
#define FO_ESTATE         -9   /* call out of order (e.g. descent before shape derivative)  */

typedef struct fo_ctx fo_ctx;
typedef struct fo_mesh fo_mesh;
typedef struct fo_problem fo_problem;

/* model kinds (fo_model_desc.kind) */
#define FO_HEAT       0   /* -div(A grad u) = f, J = int A |grad u|^2          (Sec. 6.3) */
#define FO_ELASTIC    1   /* -div(A sigma(u)) = 0 + loads, J = int A sigma:eps   (Sec. 6.2) */
#define FO_HELMHOLTZ  2   /* -div(A k grad u) + omega^2 u = f, J = int f u (screened family) */
#define FO_LOGISTIC   3   /* -Delta u = r u (1 - u / K), K = a_in on {phi < 0}, a_out     */
                          /* elsewhere, natural boundary; J = -int u; Newton state,      */
                          /* linear adjoint (Sec. 6.4, eqs log_cost, log_prob, log_KOmega) */

/* precisions (fo_solve_opts.precision) */
#define FO_FP64   0       /* FP64 operator, vectors and reductions                        */
#define FO_MIXED  1       /* FP32 inner PCG (FP64 dots) wrapped in FP64 iterative refinement */

/* fields (fo_get / fo_set) */
#define FO_FIELD_PHI    0 /* level set, N_n                                                */
#define FO_FIELD_U      1 /* state, N_dof                                                 */
#define FO_FIELD_P      2 /* adjoint, N_dof                                               */
#define FO_FIELD_THETA  3 /* velocity, d*N_n interleaved                                  */
#define FO_FIELD_RHS    4 /* shape-derivative RHS b, d*N_n interleaved                    */
#define FO_FIELD_COEF   5 /* A_e per element (double)                                     */
#define FO_FIELD_CHI    6 /* chi_e per element as double (0 / 1; the fraction for FO_COEF_CUT) */
#define FO_FIELD_LOAD   7 /* state load F, N_dof (zero on Dirichlet DOFs)                 */
#define FO_FIELD_OMEGA0 8 /* penalised-subdomain mask per element as double (0 / 1)       */
#define FO_FIELD_V      9 /* inverse elasticity: second states v_k (y_k = v_k + g_k), n_cases x N_dof */
#define FO_FIELD_Q     10 /* inverse elasticity: their adjoints q_k, n_cases x N_dof        */
#define FO_FIELD_MEAS  11 /* inverse elasticity: measurement extensions g_k, n_cases x N_dof */

/* operators (fo_apply) */
#define FO_OP_STATE      0 /* y = K_A x, Dirichlet rows/columns replaced by identity      */
#define FO_OP_VELOCITY   1 /* y = B x on d*N_n interleaved vectors (component-blocked)    */
#define FO_OP_TRANSPORT_L 2 /* y = L x (after fo_transport_assemble)                      */
#define FO_OP_TRANSPORT_R 3 /* y = R x (after fo_transport_assemble)                      */
#define FO_OP_STATE_FP32 4 /* the FP32 state operator of the mixed path (x, y still double) */

typedef struct {
  int dim;                  /* 2 or 3                                                   */
  int n[3];                 /* cells per axis                                           */
  double lo[3], hi[3];      /* box                                                      */
  int64_t num_nodes, num_cells, num_elems;
  double volume;            /* |D|                                                      */
  double h;                 /* mesh diameter of Sec. 5.6: the edge of the equilateral   */
                            /* triangle / regular tet of measure |D|/N_T (square root   */
                            /* of the printed expression)                               */
} fo_mesh_info;

typedef struct {
  int kind;                 /* FO_HEAT / FO_ELASTIC / FO_HELMHOLTZ                      */
  double a_in, a_out;       /* ersatz coefficient: a_in on {phi < 0}, a_out elsewhere   */
  double E, nu;             /* elasticity (plane strain in 2D)                          */
  double k, omega;          /* Helmholtz: conductivity factor and zero-order coefficient */
  uint32_t dirichlet_faces; /* bit (2*axis + side): homogeneous Dirichlet on that face  */
  const double *f_nodal;    /* host, N_n nodal source values (heat / Helmholtz) or NULL */
  int n_point_loads;        /* <= 4                                                     */
  int64_t point_node[4];
  double point_vec[4][3];
  int n_tractions;          /* <= 4, constant traction on a whole face                  */
  int traction_face[4];
  double traction_vec[4][3];
  double volume_target;     /* V of C = |Omega| / V; 0 = unconstrained                  */
  /* velocity form B (Sec. 5.5, eqs bd_plt, sub_dom, compli1_bili)                      */
  double alpha_mass;        /* alpha_m int theta . xi                                   */
  double normal_penalty;    /* gamma_b int_{dD} (theta.n)(xi.n)                         */
  double omega0_weight;     /* gamma_0 int chi_{Omega_0} theta . xi                     */
  int n_omega0;             /* <= 4 boxes; element in Omega_0 when its centroid is      */
  double omega0_lo[4][3];   /* strictly inside one box (use +-inf for open sides)       */
  double omega0_hi[4][3];
  int velocity_dirichlet;   /* 1: H = H^1_0(D)^d                                        */
  /* Task-parallel batch (Sec. 5.3: one PDE family with varying parameters), FO_HELMHOLTZ
   * only.  n_inst >= 1 makes the problem a batch of n_inst <= FO_MAX_INSTANCES instances
   * sharing the mesh, phi and A_e; instance i solves
   *   -div(A k_i grad u_i) + omega_i^2 u_i = f_i   (same Dirichlet faces),
   * its cost is J_i = int f_i u_i (adjoint p_i = -u_i), and the batch cost is sum_i J_i.
   * inst_k[i], inst_omega[i] and inst_f[i * N_n + a] are host arrays, copied at creation;
   * the single-problem fields k, omega and f_nodal are ignored.  0 = a single problem.
   * Batched fields (FO_FIELD_U, FO_FIELD_P, FO_FIELD_LOAD) are instance-minor:
   * value of instance i at node a at index a * n_inst + i.                              */
  int n_inst;
  const double *inst_k;
  const double *inst_omega;
  const double *inst_f;
  /* Element coefficient rule (single problems; batches take the one-point rule):
   * FO_COEF_CENTROID -- A_e = a_in when the vertex values of phi, summed in vertex order, are
   *   < 0, else a_out (one-point reading of conditional(lt(phi, 0), ...), eqs heat_AOmega,
   *   compli_AOmega); chi_e in {0, 1};
   * FO_COEF_CUT -- the exact cut-cell fraction of the P1 phi, f_e = |e cap {phi < 0}| / |e|
   *   (closed form per simplex), A_e = a_out + (a_in - a_out) f_e and chi_e = f_e in the volume
   *   constraint and its shape derivative. */
  int coef_rule;
  /* Several load cases (CompliancePlus / HeatPlus, eq. compli_plus: J = sum_k J(u_k), u_k the
   * state of load case k; single problems only).  n_cases in [0, 4] (0 or 1: one case);
   * point load i and traction t belong to case point_case[i] and traction_case[t]; f_nodal
   * belongs to case 0.  State-sized fields (FO_FIELD_U, FO_FIELD_P, FO_FIELD_LOAD) then hold
   * n_cases blocks of N_dof, case-major.  The shape derivative sums the cases' tensors. */
  int n_cases;
  int point_case[4];
  int traction_case[4];
  /* Several volume constraints (Sec. 5.4 with N_c = n_volume <= 4; single problems only):
   * C_j = |Omega cap R_j| / volume_V[j], R_j the elements whose centroid lies strictly inside
   * the box (volume_lo[j], volume_hi[j]) (use +-inf for open sides); S^C_j = chi chi_Rj / V_j I.
   * n_volume = 0: the single constraint |Omega| / volume_target when volume_target > 0. */
  int n_volume;
  double volume_lo[4][3], volume_hi[4][3], volume_V[4];
  /* Logistic population model (FO_LOGISTIC, Sec. 6.4; box meshes, one load case, the
   * one-point coefficient rule, at most the single constraint |Omega| / volume_target).
   * growth_rate: r > 0.  The carrying capacity K_e is the element coefficient (a_in inside,
   * a_out outside; the paper's example takes 1 and 1e-2).  u_init: host array of N_n initial
   * Newton values, copied at creation (NULL: u = a_in everywhere); a state solve with
   * warm_start = 1 starts from the current state instead.  Newton stops at the first iterate
   * with ||F(u_k)||_2 <= newton_rtol ||F(u_0)||_2 + newton_atol, or when the update has
   * ||du||_inf <= 1e-14 ||u||_inf, and fails (FO_ENOCONV, result kept) after newton_maxit
   * steps; zeros select 1e-13, 0 and 50.  Each Newton step solves DF(u) du = -F(u) with the
   * Jacobi-preconditioned CG of the state options (multigrid is not used for this model). */
  double growth_rate;
  const double *u_init;
  double newton_rtol, newton_atol;
  int newton_maxit;
  /* Inverse elasticity by a Kohn-Vogelius cost (Sec. 3, Sec. 6.1; kind FO_ELASTIC, box meshes,
   * the one-point coefficient rule, no constraint).  inverse = 1 makes every load case k a
   * force-displacement pair: its tractions (traction_case) are the applied force f_k on
   * Gamma1 and meas[k * N_dof ..] (host, interleaved, copied at creation) the measured
   * displacement extended into D (g_k; see fo_dirichlet_extension).  Gamma0 = dirichlet_faces
   * (clamped), Gamma1 = gamma1_faces (same bitmask form).  States: u_k (Gamma0 clamped, force
   * f_k) and v_k (zero on the whole boundary, int A sigma(v_k + g_k):eps(w) = 0); cost
   * J = sum_k alpha/2 int |u_k - v_k - g_k|^2 + beta/2 int_Gamma1 |u_k - g_k|^2 with
   * alpha = kv_alpha, beta = kv_beta; fo_adjoint_solve solves both adjoints p_k, q_k and the
   * shape derivative is the paper's S0, S1 summed over the pairs.  A = a_in (kappa) inside,
   * a_out outside. */
  int inverse;
  uint32_t gamma1_faces;
  const double *meas;
  double kv_alpha, kv_beta;
} fo_model_desc;

#define FO_COEF_CENTROID 0
#define FO_COEF_CUT      1

#define FO_MAX_INSTANCES 128

typedef struct {
  int precision;            /* FO_FP64 or FO_MIXED                                      */
  double rtol;              /* stop when ||r||_2 <= rtol ||b||_2                        */
  int maxit;                /* iteration cap (FO_ENOCONV when reached)                  */
  int warm_start;           /* 1: start from the field's current value                  */
  double inner_rtol;        /* FO_MIXED: relative reduction asked of each FP32 solve    */
  int inner_maxit;          /* FO_MIXED: cap per FP32 solve                             */
  int grid_blocks;          /* 0 = autotuned; else blocks of the persistent kernel      */
  int precond;              /* FO_PC_JACOBI, or FO_PC_MG: an FP32 geometric-multigrid   */
                            /* V-cycle as preconditioner.  Single problems coarsen any  */
                            /* grid of >= 3 cells per axis (ceil(n/2) per axis where an */
                            /* axis does not halve) down to a coarsest level of <= 8192 */
                            /* unknowns (else the Jacobi solver runs); batches need     */
                            /* grids that halve.  Single problems: FO_FP64 ->           */
                            /* FP64 CG; FO_MIXED (state, adjoint) -> FP64 refinement     */
                            /* around an FP32 CG (FP32 rows and vectors, FP64 dots;      */
                            /* inner_rtol, inner_maxit per step); the velocity solve is */
                            /* FP64 CG whatever the precision.                          */
                            /* Batches (state, adjoint): FO_FP64 -> FP64 CG; FO_MIXED -> */
                            /* FP64 refinement around an FP32 CG (inner_rtol,           */
                            /* inner_maxit per refinement step), stopping an instance   */
                            /* also when a step fails to halve its true residual.       */
  int mg_bf16;              /* FO_PC_MG, single problems: 1 = the V-cycle levels run by  */
                            /* the whole grid read their rows rounded to BF16 (FP32      */
                            /* arithmetic); the CG operator, its vectors and dots keep   */
                            /* their precision, so only the preconditioner changes and   */
                            /* the stopping test and accuracy are those of `precision`.  */
                            /* The rows are difference-form weights, so the rounded      */
                            /* operator keeps its symmetry and constant kernel.  Costs   */
                            /* half the FP32 rows' bytes more memory.  0 = FP32 rows.    */
} fo_solve_opts;

#define FO_PC_JACOBI 0
#define FO_PC_MG     1

typedef struct {
  int iterations;           /* Krylov iterations (FP64, or total inner FP32)            */
  int outer_iterations;     /* FO_MIXED refinement steps                                */
  int operator_applies;     /* operator applications in total                          */
  double rel_residual;      /* final ||r||/||b|| (FP64)                                 */
} fo_solve_stats;

typedef struct {
  double dfactor;           /* t_end = dfactor / B(theta, theta)        (eq. tend)      */
  double t_min, t_max;      /* lv_time                                                  */
  int s_min, s_max;         /* lv_iter                                  (eq. steps)     */
  int smooth;               /* diffusion in the transport (eq. transport)               */
  int reinit_step;          /* 0 = never; else reinitialise when i > 0, i % step == 0   */
  int reinit_steps;         /* reinit_pars[0]                                           */
  double reinit_time;       /* reinit_pars[1]                                           */
  double h;                 /* mesh diameter used by transport / reinit (0 = mesh's)    */
  fo_solve_opts state, velocity, transport;
} fo_run_options;

typedef struct {
  int nc;                   /* number of constraints (<= 4)                             */
  double r, delta, alpha, beta;
  double z[4], lambda[4], mu[4];
} fo_ppl;

typedef struct {
  double J, C, L, lambda, Btt, t_end;
  int nsteps, reinit;
  fo_solve_stats state, velocity, transport, reinit_stats;
  /* device time of each phase in ms (CUDA events on the context stream; filled when
   * fo_ctx_set_timing(ctx, 1) is on, else 0): coefficients + state solve, functionals,
   * shape derivative, velocity, transport (assembly + steps), reinitialisation */
  double ms_state, ms_functionals, ms_shape, ms_velocity, ms_transport, ms_reinit;
  /* with timing on: device time of the persistent state-solve CG launch(es) alone (no
   * operator or hierarchy rebuild; summed over refinement steps and restarts) */
  double ms_state_kernel;
  int nc;                   /* constraints of this iteration (0 = none)                 */
  double Cv[4], lambdav[4]; /* C_j and lambda_j of every constraint (C, lambda = [0])    */
  fo_solve_stats adjoint;   /* explicit adjoint solve of the iteration (FO_LOGISTIC)     */
  int newton_steps;         /* Newton steps of the state solve (FO_LOGISTIC)             */
} fo_iter_log;

/* ---------------------------------------------------------------- context ----- */
/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to enqueue on
 * (NULL: the context creates its own).  mem_budget_bytes: 0 = unlimited; otherwise device
 * allocations beyond it fail with FO_ENOMEM_BUDGET. */
FO_API fo_status fo_ctx_create(int device, void *cuda_stream, size_t mem_budget_bytes, fo_ctx **out);
FO_API fo_status fo_ctx_destroy(fo_ctx *ctx);
FO_API const char *fo_last_error(const fo_ctx *ctx);
/* bytes of device memory currently held by the context */
FO_API fo_status fo_ctx_memory(const fo_ctx *ctx, size_t *bytes_in_use);
/* Turn per-phase device timing of fo_opt_step on (1) or off (0). */
FO_API fo_status fo_ctx_set_timing(fo_ctx *ctx, int on);
/* Size this context's persistent solver launches (the grid-synchronised CG, multigrid CG and
 * Krylov kernels) for at most 1/share of the blocks the device can hold co-resident (1, the
 * default: all of them), so that launches of other contexts running at the same time find
 * room beside them on every SM.  A latency-bound solve loses little from the smaller grid and
 * two of them overlap almost perfectly (measured: two 3D cantilever state solves in 61 ms at
 * share 2 against 100 ms one after the other at share 1).  Results depend on the grid (the
 * order of the block sums), so a problem solved at two settings agrees to rounding only.
 * share in [1, 16]. */
FO_API fo_status fo_ctx_set_grid_share(fo_ctx *ctx, int share);
/* Number of kernels this library has launched in the process so far (all contexts). */
FO_API fo_status fo_launch_count(unsigned long long *out);
/* With timing on (fo_ctx_set_timing): device time in ms of the persistent CG launch(es) of
 * the last single-problem state or adjoint solve alone (summed over refinement steps and
 * restarts), measured with CUDA events on the context's stream. */
FO_API fo_status fo_ctx_solve_kernel_ms(const fo_ctx *ctx, double *ms);
/* wait for all work enqueued on the context's stream */
FO_API fo_status fo_ctx_sync(fo_ctx *ctx);

/* ------------------------------------------------------------------- mesh ----- */
/* Structured Kuhn mesh of prod [lo_a, hi_a] with n[a] cells per axis (Sec. 5.2 domain,
 * replacing the paper's Gmsh meshes).  Connectivity and coordinates are built on the GPU. */
FO_API fo_status fo_mesh_box(fo_ctx *ctx, int dim, const int n[3], const double lo[3], const double hi[3],
                      fo_mesh **out);
/* A general simplicial mesh given as arrays (the role of the paper's Gmsh / DOLFINx meshes,
 * Sec. 5.1 helpers and Sec. 6 examples): coords [nn][dim] FP64 and cells [nt][dim+1] int32
 * vertex ids (any numbering, vertex order and orientation), host arrays copied before the call
 * returns.  Box faces (face = 2*axis + side, as for fo_mesh_box) are those of the nodes'
 * bounding box: a node lies on a face when its coordinate equals the box's bound exactly, and
 * a boundary facet (a facet of one element only) belongs to a face when all its vertices do.
 * Dirichlet faces, tractions, the H^1_0 velocity space and the normal penalty refer to these
 * (the penalty uses every boundary facet with its outward normal).  Operators are assembled
 * per coefficient update into the node graph (node-block CSR); solves are Jacobi-PCG (state,
 * velocity; FO_MIXED: FP32 inner solves in FP64 refinement) and BiCGStab (transport,
 * reinitialisation).  fo_mesh_query reports n = 0, the bounding box, and |D| = the sum of the
 * element measures (which also defines h).  Task-parallel batches and serving need box meshes.
 * FO_EINVAL on a vertex id out of range, a facet shared by more than two elements or a
 * degenerate element; FO_ENAN on a non-finite coordinate. */
FO_API fo_status fo_mesh_from_arrays(fo_ctx *ctx, int dim, int64_t nn, const double *coords, int64_t nt,
                                     const int32_t *cells, fo_mesh **out);
FO_API fo_status fo_mesh_destroy(fo_mesh *mesh);
FO_API fo_status fo_mesh_query(const fo_mesh *mesh, fo_mesh_info *out);
/* Copy connectivity (int32 [N_T][d+1]) and coordinates (f64 [N_n][d]) to host arrays;
 * either pointer may be NULL. */
FO_API fo_status fo_mesh_copy_out(const fo_mesh *mesh, int32_t *cells, double *coords);

/* ---------------------------------------------------------------- problem ----- */
FO_API fo_status fo_problem_create(fo_mesh *mesh, const fo_model_desc *desc, fo_problem **out);
FO_API fo_status fo_problem_destroy(fo_problem *prob);
/* Set the level set phi (N_n values). */
FO_API fo_status fo_set_levelset(fo_problem *prob, const double *phi, int on_device);
/* InitialLevel (Sec. 5.7, eq. phi0): phi = factor * max_k (radii_k - |x - centers_k|_ord),
 * ord = 2 or 0 (0 means the infinity norm); centers [count][d] and radii on the host. */
FO_API fo_status fo_initial_level(fo_problem *prob, int count, const double *centers, const double *radii,
                           double factor, int ord);
/* Random-bump level set: phi(x) = sum_k exp(-|x - c_k|^2 / (2 width^2)) - offset, terms
 * added in k order; centers [count][d] on the host (the bumps are the holes of Omega). */
FO_API fo_status fo_levelset_bumps(fo_problem *prob, int count, const double *centers, double width, double offset);
/* Element coefficient A_e and chi_e from phi (one-point rule: the vertex values of phi
 * summed in vertex order; < 0 is inside, eqs heat_AOmega / compli_AOmega). */
FO_API fo_status fo_coefficients(fo_problem *prob);
/* State solve K_A u = F (Algorithm 1 step "state"). */
FO_API fo_status fo_state_solve(fo_problem *prob, const fo_solve_opts *opts, fo_solve_stats *stats);
/* Explicit adjoint solve K_A p = -c F with c = 2 for FO_ELASTIC (p = -2u, Sec. 6.2) and
 * c = 1 otherwise (p = -u, Sec. 6.3); the shape derivative uses these closed forms. */
FO_API fo_status fo_adjoint_solve(fo_problem *prob, const fo_solve_opts *opts, fo_solve_stats *stats);
/* Cost J and constraint C = |Omega| / V (C = |Omega| when V = 0); synchronises. */
FO_API fo_status fo_functionals(fo_problem *prob, double *J, double *C);
/* Velocity RHS b[d*a + k] = sum_e int_e S0_k psi_a + (S1 grad psi_a)_k with
 * S = S^J + lambda S^C (eq. S0andS1).  rhs_out (host, d*N_n) may be NULL. */
FO_API fo_status fo_shape_derivative(fo_problem *prob, double lambda, double *rhs_out);
/* Cost and every constraint: J (summed over the load cases) and C[0..nc) with nc the
 * problem's number of constraints (n_volume, or 1 when volume_target > 0, or 0); C may be NULL
 * when nc = 0; FO_EINVAL when nc differs from the problem's.  Synchronises. */
FO_API fo_status fo_functionals_v(fo_problem *prob, double *J, double *C, int nc);
/* Velocity RHS with one multiplier per constraint: S = sum_k S^J(u_k) + sum_j lambda_j S^C_j
 * (eq. S0andS1, Sec. 5.4); nc as for fo_functionals_v; rhs_out (host) may be NULL. */
FO_API fo_status fo_shape_derivative_v(fo_problem *prob, const double *lambda, int nc, double *rhs_out);
/* Velocity solve B theta = -b (eq. velocity); Btt = B(theta, theta) = -b . theta. */
FO_API fo_status fo_descent(fo_problem *prob, const fo_solve_opts *opts, double *Btt, fo_solve_stats *stats);
/* Build the transport matrices L, R for time step dt (eq. weak_transport, tau of
 * eq. tau_lv at degree-2 quadrature points, diffusion tested with the full grad psi^). */
FO_API fo_status fo_transport_assemble(fo_problem *prob, double dt, double h, int smooth);
/* nsteps Crank-Nicolson steps of size t_end/nsteps moving phi along theta. */
FO_API fo_status fo_levelset_step(fo_problem *prob, double t_end, int nsteps, double h, int smooth,
                           const fo_solve_opts *opts, fo_solve_stats *stats);
/* Reinitialisation: nsteps steps of size t_final/nsteps, explicit Euler then AB2 (eq. weak_HJ). */
FO_API fo_status fo_reinit(fo_problem *prob, int nsteps, double t_final, double h,
                    const fo_solve_opts *opts, fo_solve_stats *stats);
/* One Algorithm-1 iteration number `iter` (0-based): coefficients, state, functionals,
 * PPL update (when V > 0), shape derivative, velocity, adaptive time, transport, reinit. */
FO_API fo_status fo_opt_step(fo_problem *prob, int iter, const fo_run_options *opts, fo_ppl *ppl,
                      fo_iter_log *log);
/* Copy a field out to the host (synchronises) / in from host or device memory. */
FO_API fo_status fo_get(fo_problem *prob, int field, double *host_out);
FO_API fo_status fo_set(fo_problem *prob, int field, const double *values, int on_device);
/* y = Op x for parity tests; x and y are host arrays (or device if on_device). */
FO_API fo_status fo_apply(fo_problem *prob, int op, const double *x, double *y, int on_device);

/* State solve that allocates no device memory.  The paper has no counterpart: this is for
 * callers that cannot let a library call cudaMalloc / cudaFree while they run -- those calls
 * may synchronise the whole device (a stall a latency-bound loop cannot take), and another
 * framework's caching allocator or a fixed memory budget may already own the device memory.
 * Solves K_A x = b with fo_state_solve's FP64 Jacobi-PCG (FO_PC_JACOBI: the same recurrence,
 * then at most two restarts from the true residual b - A x while it is above rtol), but its working
 * memory (Krylov vectors, reduction partials, grid-barrier counter, status words) is one
 * fixed array of FO_NOALLOC_SCRATCH_BYTES that the library declares in device memory; every
 * GPU that loads the library holds it until the process exits.
 *   b: device array, N_dof values (zero on Dirichlet DOFs, like FO_FIELD_LOAD); read only.
 *   x: device array, N_dof values; the solution (also the start value when o->warm_start).
 *   o: NULL for defaults; o->precision must be FO_FP64 (FO_MIXED -> FO_EINVAL).
 * Returns FO_EINVAL when N_dof > FO_NOALLOC_MAX_DOFS; FO_ENOCONV / FO_ENAN / FO_ETIMEOUT as
 * fo_state_solve.  The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  Every call uses the same array and finds it as the
 * previous call left it (the call clears what must start at zero): two calls that overlap on
 * the GPU -- other streams, other contexts, other threads -- race; serialise them. */
#define FO_NOALLOC_SCRATCH_BYTES (16 << 20)
#define FO_NOALLOC_MAX_DOFS 258048      /* (16 MiB / 8 - 32768 header doubles) / 8 vectors */
FO_API fo_status fo_state_solve_noalloc(fo_problem *prob, const double *b, double *x, const fo_solve_opts *o,
                                        fo_solve_stats *stats);

/* Self-test of the bounded grid barrier that every persistent solver uses (no counterpart in
 * the paper).  Launches `blocks` co-resident blocks (clamped to [2, number of SMs]) that meet
 * at one grid barrier with a wait limit of limit_ms; block `skip` (or none when skip < 0)
 * never arrives.  With skip < 0 the barrier is released: FO_OK, *gave_up = 0.  Otherwise
 * every other block gives up after limit_ms: FO_ETIMEOUT, *gave_up = blocks - 1.  No block
 * faults or hangs; the context stays usable.  limit_ms must be in (0, 10000]. */
FO_API fo_status fo_selftest_barrier(fo_ctx *ctx, int blocks, int skip, double limit_ms, int *gave_up);

/* ------------------------------------------------------------ batch (TP) ----- */
/* A batch problem (fo_model_desc.n_inst >= 1) goes through the same calls as a single
 * problem: fo_coefficients, fo_state_solve / fo_adjoint_solve (all instances in one
 * persistent cooperative launch), fo_functionals (J = sum_i J_i), fo_shape_derivative
 * (b = sum_i b_i + lambda * volume term), fo_descent, fo_levelset_step and fo_opt_step.
 * The calls below are batch-only (FO_EINVAL on a single problem). */

/* Per-instance costs J_i = F_i . u_i of the current state (n_inst values, host). */
FO_API fo_status fo_batch_costs(fo_problem *prob, double *J_inst);
/* Per-instance results of the last batched state or adjoint solve (host arrays of n_inst,
 * either may be NULL): inner Krylov iterations in which the instance was active, summed over
 * refinement steps, and the final FP64 relative residual ||b_i - K_i x_i|| / ||b_i||. */
FO_API fo_status fo_batch_solve_info(fo_problem *prob, int *inst_iters, double *inst_res);

/* Launch shape of the batched Jacobi solver (FO_PC_JACOBI; the batched multigrid uses two
 * blocks of 256 threads per SM). */
typedef struct {
  int block;                /* threads per block (a warp owns a node)                   */
  int blocks_per_sm;        /* co-resident blocks per SM; grid = blocks_per_sm * SMs   */
  double us_per_iteration;  /* tuning run time / its Krylov iterations                  */
  int candidates;           /* launch shapes timed                                     */
  int tile[3];              /* nodes per shared-memory tile along x, y, z              */
} fo_tune_result;
/* Time the batched solver's candidate launch shapes (node tile x threads per block x blocks
 * per SM, within the device's shared-memory and co-residency limits) on this problem for `precision` (FO_FP64 or
 * FO_MIXED): each runs a fixed number of Krylov iterations on the current coefficients and
 * loads, writing a scratch solution only.  The fastest shape is kept on the problem and used
 * by later solves whose opts->grid_blocks is 0; the first such solve tunes by itself. */
FO_API fo_status fo_batch_autotune(fo_problem *prob, int precision, fo_tune_result *out);

/* Schedule of the batched multigrid (FO_PC_MG). */
typedef struct {
  int blocks_per_sm;        /* co-resident blocks per SM; grid = blocks_per_sm * SMs   */
  int nu0;                  /* smoothing sweeps before and after the coarse correction */
                            /* on the finest level                                      */
  int inst_levels;          /* coarse levels run one instance per block in shared memory */
  double ms;                /* the chosen schedule's solve time (CUDA events)           */
  int iterations;           /* its Krylov iterations (inner ones for FO_MIXED)          */
  int candidates;           /* schedules timed                                          */
  int tile[3];              /* nodes per FP32-pass tile along x, y, z (fixed per        */
                            /* dimension and batch width; a 16x16 2D tile at one block  */
                            /* per SM measured 22-28 % slower than 16x8 at two)         */
} fo_mg_tune_result;
/* Time the batched multigrid's schedules on this problem for `precision` (FO_FP64 or FO_MIXED):
 * blocks per SM from one to the kernel's co-residency limit, one or two finest-level sweeps,
 * and the per-instance levels from the size limit or one level later.  Each candidate solves
 * the current system from zero to rtol into a scratch solution (the problem's fields are not
 * touched); the fastest one that converges is kept and used by later multigrid solves whose
 * opts->grid_blocks is 0 (a schedule changes the iteration count, not the stopping test).
 * Untuned problems use two blocks per SM, one finest-level sweep and the size limit.  The
 * schedule changes the order of the block sums, so results of a tuned and an untuned problem
 * agree to rounding only. */
FO_API fo_status fo_batch_mg_autotune(fo_problem *prob, int precision, double rtol, fo_mg_tune_result *out);

/* Dirichlet extension (Sec. 5.7, eq. dir), the helper that extends boundary measurements into D:
 * per component, eta = values at the nodes of the listed faces (bitmask (2 axis + side), as
 * dirichlet_faces) and int D eta : D zeta = 0 for every P1 zeta vanishing there (natural
 * condition elsewhere).  values and out are host arrays of d * N_n (interleaved; only the
 * values at the face nodes are read).  Box meshes; solved by Jacobi-preconditioned CG to
 * opts->rtol (NULL: the defaults), with temporary device memory freed before returning. */
FO_API fo_status fo_dirichlet_extension(fo_mesh *mesh, uint32_t faces, const double *values, double *out,
                                        const fo_solve_opts *opts);

/* --------------------------------------------------------------- serving ----- */
/* A request is one Algorithm-1 step without the transport (state solve, explicit adjoint
 * solve, cost and constraint, shape derivative, velocity) on its own box mesh.  A server
 * runs `executors` requests at once, each on its own context and CUDA stream, so that the
 * device work of different requests overlaps; requests wait in a FIFO queue and are admitted
 * in order when an executor is free and the in-flight requests' device memory plus theirs
 * fits in mem_budget.  A request's memory estimate is exact for the library's allocations
 * (fo_request_device_bytes).  The device work of a request is the same whether it runs
 * alone or in a mix (same kernels, launch shapes and reduction order), so its results are
 * the same bits. */
typedef struct {
  int dim;                  /* 2 or 3                                                   */
  int n[3];                 /* cells per axis                                           */
  double lo[3], hi[3];      /* box                                                      */
  fo_model_desc model;      /* FO_HEAT or FO_ELASTIC (batches are not served); f_nodal  */
                            /* (N_n values) is copied at submit                         */
  int n_bumps;              /* > 0: phi = sum of Gaussian bumps - offset (fo_levelset_bumps) */
  const double *bump_centers; /* [n_bumps][dim], copied at submit                       */
  double bump_width, bump_offset;
  const double *phi;        /* n_bumps == 0: N_n nodal level set, copied at submit      */
  double lambda;            /* multiplier of the volume term in S                       */
  fo_solve_opts state;      /* state and adjoint solves                                 */
  fo_solve_opts velocity;
  double *theta_out;        /* optional host array of d*N_n, written before completion; */
                            /* it must stay valid until the request completes           */
} fo_request;

typedef struct {
  fo_status status;         /* FO_OK, FO_ENOCONV (results written), or the failing call's */
  char message[128];        /* fo_last_error text of a failing call                     */
  double J, C, Btt;         /* cost, constraint, B(theta, theta)                        */
  fo_solve_stats state, adjoint, velocity;
  int64_t dofs;             /* N_dof of the state                                       */
  size_t device_bytes;      /* the admission estimate                                   */
  double submit_ms, start_ms, end_ms;   /* host steady clock, ms since server creation  */
} fo_result;

typedef struct {
  int executors;            /* requests in flight at once (default 8)                   */
  size_t mem_budget;        /* device bytes in-flight requests may hold (default 8 GiB) */
  int queue_capacity;       /* queued requests before fo_submit says FO_EBUSY (4096)    */
  double dry_run_ms;        /* > 0: executors sleep this long instead of any device    */
                            /* work (tests of queueing and admission without a GPU)     */
  int grid_share;           /* fo_ctx_set_grid_share of every executor's context        */
                            /* (default 4: up to four large solves share the SMs)       */
  int policy;               /* FO_SERVE_FIFO (default): the queue's head is admitted    */
                            /* next, once it fits; FO_SERVE_SMALLEST_FIRST: the queued  */
                            /* request with the smallest footprint (a proxy for its     */
                            /* work; ties in submission order), which lowers the median */
                            /* latency of a backlog and can hold large requests back    */
                            /* while smaller ones keep arriving                        */
} fo_server_opts;

#define FO_SERVE_FIFO           0
#define FO_SERVE_SMALLEST_FIRST 1

typedef struct {
  int64_t submitted, completed, failed, rejected;
  int64_t peak_in_flight;   /* most requests running at once                           */
  size_t peak_bytes;        /* most admitted device memory at once                     */
} fo_server_stats;

typedef struct fo_server fo_server;
FO_API void fo_server_opts_default(fo_server_opts *o);
/* Device memory the library allocates for a request (mesh, problem fields, solver scratch). */
FO_API size_t fo_request_device_bytes(const fo_request *rq);
/* The server's executors use ctx's device; ctx receives create-time errors only (it may be
 * NULL for a dry-run server).  Destroy the server only when no other thread waits on it. */
FO_API fo_status fo_server_create(fo_ctx *ctx, const fo_server_opts *opts, fo_server **out);
/* Stops admitting, cancels queued requests (FO_ESTATE), waits for the running ones. */
FO_API fo_status fo_server_destroy(fo_server *srv);
/* Queue a request; its host arrays are copied.  FO_EBUSY when the queue is full,
 * FO_ENOMEM_BUDGET when it alone needs more than mem_budget, FO_EINVAL on a bad request. */
FO_API fo_status fo_submit(fo_server *srv, const fo_request *rq, uint64_t *ticket);
/* Non-blocking: *done = 1 and *res filled once the request has completed. */
FO_API fo_status fo_poll(fo_server *srv, uint64_t ticket, fo_result *res, int *done);
/* Wait at most timeout_s seconds: FO_ETIMEOUT if the request has not completed by then. */
FO_API fo_status fo_wait(fo_server *srv, uint64_t ticket, double timeout_s, fo_result *res);
/* Forget a completed request (its result is no longer kept). */
FO_API fo_status fo_release(fo_server *srv, uint64_t ticket);
FO_API fo_status fo_server_get_stats(fo_server *srv, fo_server_stats *out);

/* ------------------------------------------------------------- host-only ----- */
/* PPL state with r = 0.999, delta0 = 0.5, alpha = 2000, beta = 0.5, z = lambda = mu = 0. */
FO_API void fo_ppl_init(fo_ppl *s, int nc);
/* One update of eq. lag_method from C; writes lambda (nc values) and L of eq. lagrangian. */
FO_API void fo_ppl_update(fo_ppl *s, const double *C, double J, double *lambda_out, double *L_out);
/* Adaptive time (eqs tend, steps): t_end clamped to [t_min, t_max] with B(theta, theta)
 * floored at 1e-12, steps clamped to [s_min, s_max] and rounded half away from zero. */
FO_API void fo_adaptime(double Btt, const fo_run_options *opts, double *t_end, int *nsteps);
/* Stopping criterion of Sec. 5.7 at iteration i = n - 1: values[0..n) are J (no constraints)
 * or L (with constraints) of iterations 0..i; C the constraint vector of iteration i (nc
 * values, nc = 0 without constraints).  *stop = 1 when i > start_to_check and
 * max_{i - prev <= j < i} |v_i - v_j| < tol |v_i|, and, with constraints, max_j |C_j - 1| <
 * ctrn_tol.  Defaults (fo_stop_opts_default): 30, 1e-2, 1e-2, 10 (cost_tol = lgrn_tol = tol). */
typedef struct {
  int start_to_check;
  double tol;
  double ctrn_tol;
  int prev;
} fo_stop_opts;
FO_API void fo_stop_opts_default(fo_stop_opts *o);
FO_API void fo_stop_check(const double *values, int n, const double *C, int nc, const fo_stop_opts *o, int *stop);
/* Default run options of runDP (Sec. 5.1) and default solver options. */
FO_API void fo_run_options_default(fo_run_options *opts);
FO_API void fo_solve_opts_default(fo_solve_opts *opts);

#ifdef __cplusplus
}
#endif
#endif /* FORMOPT_GB300_H */
