"""Builders that set up the same problem on the GPU (through the C ABI) and in the oracle."""
import numpy as np

from oracle import algorithm as oalg
from oracle import velocity as ovel
from oracle.mesh import BoxMesh


def case(dim=2, n=(8, 8), lo=None, hi=None, kind=0, a_in=1.0, a_out=1e-3, E=1.0, nu=0.3, k=1.0, omega=0.0,
         dirichlet=((0, 0),), f=None, point_loads=(), tractions=(), volume=0.0, alpha_mass=0.1,
         normal_penalty=0.0, omega0_weight=0.0, omega0_boxes=(), velocity_dirichlet=False, coef_rule=0):
    lo = tuple(lo) if lo is not None else (0.0,) * dim
    hi = tuple(hi) if hi is not None else (1.0,) * dim
    return dict(dim=dim, n=tuple(n), lo=lo, hi=hi, kind=kind, a_in=a_in, a_out=a_out, E=E, nu=nu, k=k,
                omega=omega, dirichlet=list(dirichlet), f=f, point_loads=list(point_loads),
                tractions=list(tractions), volume=volume, alpha_mass=alpha_mass, normal_penalty=normal_penalty,
                omega0_weight=omega0_weight, omega0_boxes=list(omega0_boxes),
                velocity_dirichlet=velocity_dirichlet, coef_rule=coef_rule)


def oracle_problem(c):
    m = BoxMesh(c["dim"], c["n"], c["lo"], c["hi"])
    f = None
    if c["f"] is not None:
        f = c["f"](m.coords) if callable(c["f"]) else np.asarray(c["f"], dtype=np.float64)
    pl = [(int(m.node_id(np.array(ijk))), vec) for ijk, vec in c["point_loads"]]
    vform = ovel.VelocityForm(alpha_mass=c["alpha_mass"], normal_penalty=c["normal_penalty"],
                              omega0_weight=c["omega0_weight"], omega0_boxes=c["omega0_boxes"],
                              dirichlet=c["velocity_dirichlet"])
    return oalg.Problem(mesh=m, kind=c["kind"], a_in=c["a_in"], a_out=c["a_out"], E=c["E"], nu=c["nu"],
                        dirichlet_faces=c["dirichlet"], f_nodal=f, point_loads=pl, tractions=c["tractions"],
                        volume_target=c["volume"], k=c["k"], omega=c["omega"], vform=vform,
                        coef_rule="cut" if c.get("coef_rule", 0) == 1 else "centroid")


def gpu_problem(ctx, c):
    from paper_2601_05709_gb300 import api
    mesh = ctx.mesh_box(c["dim"], c["n"], c["lo"], c["hi"])
    _, coords = mesh.copy_out()
    f = None
    if c["f"] is not None:
        f = c["f"](coords) if callable(c["f"]) else np.asarray(c["f"], dtype=np.float64)
    pl = [(mesh.node_id(ijk), vec) for ijk, vec in c["point_loads"]]
    desc = api.model_desc(c["kind"], a_in=c["a_in"], a_out=c["a_out"], E=c["E"], nu=c["nu"], k=c["k"],
                          omega=c["omega"], dirichlet=c["dirichlet"], f_nodal=f, point_loads=pl,
                          tractions=c["tractions"], volume=c["volume"], alpha_mass=c["alpha_mass"],
                          normal_penalty=c["normal_penalty"], omega0_weight=c["omega0_weight"],
                          omega0_boxes=c["omega0_boxes"], velocity_dirichlet=c["velocity_dirichlet"],
                          coef_rule=c.get("coef_rule", 0))
    return mesh, mesh.problem(desc)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def close_scaled(a, b, tol):
    """max |a - b| <= tol * max |b| (elementwise agreement at the vector's own scale)."""
    return np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1e-300)


def solve_parity(K, F, free, u, u_ref):
    """How far a computed solution u of K u = F (free DOFs) is from the oracle's u_ref, and
    what the conditioning allows.

    Returns (forward, omega, omega_ref, skeel):
      forward    ||u - u_ref||_inf / ||u_ref||_inf;
      omega      Oettli-Prager componentwise backward error of u:
                 max_i |F - K u|_i / (|K| |u| + |F|)_i  -- u solves exactly a system whose every
                 entry is perturbed by at most omega relative;
      omega_ref  the same for the oracle's solution;
      skeel      Skeel condition number || |K^{-1}| |K| |u_ref| ||_inf / ||u_ref||_inf, estimated
                 with Higham's 1-norm estimator on the oracle's LU factors.
    First-order perturbation theory bounds the forward difference by about
    skeel * (omega + omega_ref).
    """
    import scipy.sparse.linalg as spla
    idx = np.flatnonzero(free)
    Kf = K[idx][:, idx].tocsc()
    Ff, uf, rf = F[idx], u[idx], u_ref[idx]
    absK = abs(Kf)

    def omega(x):
        return float(np.max(np.abs(Ff - Kf @ x) / (absK @ np.abs(x) + np.abs(Ff))))

    lu = spla.splu(Kf)
    g = absK @ np.abs(rf)
    op = spla.LinearOperator(Kf.shape, matvec=lambda v: g * lu.solve(v), rmatvec=lambda v: lu.solve(g * v),
                             dtype=np.float64)
    skeel = spla.onenormest(op.T) / np.max(np.abs(rf))
    fwd = float(np.max(np.abs(uf - rf)) / np.max(np.abs(rf)))
    return fwd, omega(uf), omega(rf), float(skeel)


def assert_solve_parity(K, F, free, u, u_ref, tol, omega_max=1e-13):
    """The stated tolerance where the conditioning allows it, else the perturbation bound.

    A solve is accepted when its componentwise backward error is at the FP64 rounding level
    (omega <= omega_max) and its forward difference from the oracle is within tol or, when
    the system is too ill-conditioned for tol to be reachable by any FP64 solver, within
    10 * skeel * (omega + omega_ref) (and never above 1e-8)."""
    fwd, om, om_ref, skeel = solve_parity(K, F, free, u, u_ref)
    bound = max(tol, min(1e-8, 10.0 * skeel * (om + om_ref)))
    assert om <= omega_max, ("backward error", om, fwd, skeel)
    assert fwd <= bound, ("forward error", fwd, bound, om, om_ref, skeel)
    return fwd, om, skeel


HEAT2D = dict(dim=2, n=(64, 64), kind=0, f=lambda X: np.ones(X.shape[0]), dirichlet=[(0, 0)],
              alpha_mass=0.01, velocity_dirichlet=True)


def cantilever2d(n=(256, 128)):
    nx, ny = n
    return case(dim=2, n=n, lo=(0, 0), hi=(2, 1), kind=1, dirichlet=[(0, 0)],
                point_loads=[((nx, ny // 2), (0.0, -1.0))], volume=1.0, alpha_mass=0.1, normal_penalty=1e4,
                omega0_weight=1e4, omega0_boxes=[((1.95, 0.42), (np.inf, 0.58))])


def cantilever3d(n=(12, 6, 6)):
    return case(dim=3, n=n, lo=(0, 0, 0), hi=(2, 1, 1), kind=1, dirichlet=[(0, 0)],
                tractions=[(0, 1, (0.0, 0.0, -1.0))], volume=1.0, alpha_mass=0.1, normal_penalty=1e4,
                omega0_weight=1e4, omega0_boxes=[((1.90, 0.35, 0.35), (np.inf, 0.65, 0.65))])


def batch_case(dim=2, n=(16, 16), n_inst=5, seed=1, a_in=1.0, a_out=1e-3, volume=0.0, alpha_mass=0.1,
               velocity_dirichlet=False):
    """A task-parallel batch: k_i ~ U[0.5, 2], omega_i ~ U[0, 5], Fourier sources (8 modes,
    N(0, 1) amplitudes, seeded), Dirichlet on x = 0, on the unit box."""
    from paper_2601_05709_gb300 import workloads
    k, om, amp = workloads.batch_parameters(n_inst, seed)
    return dict(dim=dim, n=tuple(n), n_inst=n_inst, k=k, omega=om, amp=amp, a_in=a_in, a_out=a_out,
                volume=volume, alpha_mass=alpha_mass, velocity_dirichlet=velocity_dirichlet)


def _batch_sources(coords, amp):
    from paper_2601_05709_gb300 import workloads
    return workloads.fourier_loads(coords[:, :2], amp)


def oracle_batch(c):
    from oracle.batch import Batch
    m = BoxMesh(c["dim"], c["n"], (0.0,) * c["dim"], (1.0,) * c["dim"])
    vform = ovel.VelocityForm(alpha_mass=c["alpha_mass"], dirichlet=c["velocity_dirichlet"])
    return Batch(m, c["k"], c["omega"], _batch_sources(m.coords, c["amp"]), dirichlet_faces=[(0, 0)],
                 a_in=c["a_in"], a_out=c["a_out"], volume_target=c["volume"], vform=vform)


def gpu_batch(ctx, c):
    from paper_2601_05709_gb300 import api
    mesh = ctx.mesh_box(c["dim"], c["n"], (0.0,) * c["dim"], (1.0,) * c["dim"])
    _, coords = mesh.copy_out()
    desc = api.model_desc(2, a_in=c["a_in"], a_out=c["a_out"], dirichlet=[(0, 0)], volume=c["volume"],
                          alpha_mass=c["alpha_mass"], velocity_dirichlet=c["velocity_dirichlet"],
                          inst_k=c["k"], inst_omega=c["omega"], inst_f=_batch_sources(coords, c["amp"]))
    return mesh, mesh.problem(desc)


# ------------------------------------------------------------------ meshes given as arrays
def umesh(dim=2, n=(8, 6), hi=None, jitter=0.3, seed=0, pattern="kuhn", shuffle=True):
    """A seeded general simplicial mesh (coords, cells) of the box (0, hi): jittered interior,
    shuffled numbering (workloads.simplex_mesh)."""
    from paper_2601_05709_gb300 import workloads
    hi = tuple(hi) if hi is not None else (1.0,) * dim
    return workloads.simplex_mesh(dim, n, (0.0,) * dim, hi, jitter=jitter, seed=seed, pattern=pattern, shuffle=shuffle)


def node_at(coords, x):
    """Index of the node at coordinates x (exact match)."""
    hit = np.flatnonzero(np.all(np.abs(coords - np.asarray(x, dtype=np.float64)[None, :]) < 1e-12, axis=1))
    assert hit.size == 1, x
    return int(hit[0])


def oracle_umesh_problem(coords, cells, c):
    """The oracle problem of case dict c (point loads given by coordinates) on an array mesh."""
    from oracle.mesh import ArrayMesh
    m = ArrayMesh(coords, cells)
    f = None
    if c["f"] is not None:
        f = c["f"](m.coords) if callable(c["f"]) else np.asarray(c["f"], dtype=np.float64)
    pl = [(node_at(m.coords, x), vec) for x, vec in c["point_loads"]]
    vform = ovel.VelocityForm(alpha_mass=c["alpha_mass"], normal_penalty=c["normal_penalty"],
                              omega0_weight=c["omega0_weight"], omega0_boxes=c["omega0_boxes"],
                              dirichlet=c["velocity_dirichlet"])
    return oalg.Problem(mesh=m, kind=c["kind"], a_in=c["a_in"], a_out=c["a_out"], E=c["E"], nu=c["nu"],
                        dirichlet_faces=c["dirichlet"], f_nodal=f, point_loads=pl, tractions=c["tractions"],
                        volume_target=c["volume"], k=c["k"], omega=c["omega"], vform=vform,
                        coef_rule="cut" if c.get("coef_rule", 0) == 1 else "centroid")


def gpu_umesh_problem(ctx, coords, cells, c):
    from paper_2601_05709_gb300 import api
    mesh = ctx.mesh_from_arrays(coords, cells)
    f = None
    if c["f"] is not None:
        f = c["f"](coords) if callable(c["f"]) else np.asarray(c["f"], dtype=np.float64)
    pl = [(node_at(coords, x), vec) for x, vec in c["point_loads"]]
    desc = api.model_desc(c["kind"], a_in=c["a_in"], a_out=c["a_out"], E=c["E"], nu=c["nu"], k=c["k"],
                          omega=c["omega"], dirichlet=c["dirichlet"], f_nodal=f, point_loads=pl,
                          tractions=c["tractions"], volume=c["volume"], alpha_mass=c["alpha_mass"],
                          normal_penalty=c["normal_penalty"], omega0_weight=c["omega0_weight"],
                          omega0_boxes=c["omega0_boxes"], velocity_dirichlet=c["velocity_dirichlet"],
                          coef_rule=c.get("coef_rule", 0))
    return mesh, mesh.problem(desc)
