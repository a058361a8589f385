"""Python binding of the C ABI: the same calls, with numpy / torch arrays marshalled.

Every computation runs in the CUDA library; this module only converts arguments, checks
status codes and owns handles.  Device arrays may be passed as torch CUDA tensors (their
data_ptr() is handed to the library with on_device = 1).
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import (FO_COEF_CENTROID, FO_COEF_CUT, FO_PC_JACOBI, FO_PC_MG, FO_ELASTIC, FO_FIELD_CHI, FO_FIELD_COEF, FO_FIELD_LOAD, FO_FIELD_OMEGA0, FO_FIELD_P,
                   FO_FIELD_PHI, FO_FIELD_RHS, FO_FIELD_THETA, FO_FIELD_U, FO_FP64, FO_HEAT, FO_HELMHOLTZ,
                   FO_LOGISTIC, FO_MIXED, FO_OP_STATE, FO_OP_STATE_FP32, FO_OP_TRANSPORT_L, FO_OP_TRANSPORT_R,
                   FO_OP_VELOCITY, FO_OK, FormoptError)

__all__ = ["Context", "Mesh", "Problem", "model_desc", "solve_opts", "run_options", "PPL", "adaptime",
           "FO_HEAT", "FO_ELASTIC", "FO_HELMHOLTZ", "FO_LOGISTIC", "FO_FP64", "FO_MIXED", "FormoptError"]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _is_device(x):
    return hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)


def solve_opts(precision=FO_FP64, rtol=1e-12, maxit=200000, warm_start=0, inner_rtol=1e-3, inner_maxit=20000,
               grid_blocks=0, precond=0, mg_bf16=0):
    o = _lib.SolveOpts()
    _lib.load().fo_solve_opts_default(C.byref(o))
    o.precision, o.rtol, o.maxit, o.warm_start = precision, rtol, maxit, int(warm_start)
    o.inner_rtol, o.inner_maxit, o.grid_blocks, o.precond = inner_rtol, inner_maxit, grid_blocks, precond
    o.mg_bf16 = int(bool(mg_bf16))
    return o


def run_options(dfactor=1e-2, lv_time=(1e-3, 1e-1), lv_iter=(8, 16), smooth=False, reinit_step=0,
                reinit_pars=(8, 1e-1), h=0.0, state=None, velocity=None, transport=None):
    o = _lib.RunOptions()
    _lib.load().fo_run_options_default(C.byref(o))
    o.dfactor = dfactor
    o.t_min, o.t_max = lv_time
    o.s_min, o.s_max = lv_iter
    o.smooth = int(bool(smooth))
    o.reinit_step = int(reinit_step or 0)
    o.reinit_steps, o.reinit_time = int(reinit_pars[0]), float(reinit_pars[1])
    o.h = h
    if state is not None:
        o.state = state
    if velocity is not None:
        o.velocity = velocity
    if transport is not None:
        o.transport = transport
    return o


def model_desc(kind, a_in=1.0, a_out=1e-3, E=1.0, nu=0.3, k=1.0, omega=0.0, dirichlet=(), f_nodal=None,
               point_loads=(), tractions=(), volume=0.0, alpha_mass=0.1, normal_penalty=0.0, omega0_weight=0.0,
               omega0_boxes=(), velocity_dirichlet=False, inst_k=None, inst_omega=None, inst_f=None, coef_rule=0,
               load_cases=None, volume_regions=None, growth_rate=0.0, u_init=None, newton_rtol=0.0,
               newton_atol=0.0, newton_maxit=0, inverse=False, gamma1=(), meas=None, kv_alpha=1.0, kv_beta=0.0):
    """Build a fo_model_desc.  dirichlet: [(axis, side)]; point_loads: [(node, vec)];
    tractions: [(axis, side, vec)]; omega0_boxes: [(lo, hi)] with strict inequalities.
    The logistic model (kind FO_LOGISTIC): growth_rate r, u_init [N_n] initial Newton values,
    carrying capacity a_in / a_out inside / outside.
    Inverse elasticity (kind FO_ELASTIC, inverse=True): every load case is a force-displacement
    pair; gamma1 [(axis, side)] the measured faces, meas [n_cases, d N_n] the measurement
    extensions g_k, kv_alpha / kv_beta the cost weights.
    A task-parallel batch (kind FO_HELMHOLTZ): inst_k, inst_omega [n_inst] and
    inst_f [n_inst, N_n]."""
    d = _lib.ModelDesc()
    d.kind, d.a_in, d.a_out, d.E, d.nu, d.k, d.omega = kind, a_in, a_out, E, nu, k, omega
    mask = 0
    for axis, side in dirichlet:
        mask |= 1 << (2 * axis + side)
    d.dirichlet_faces = mask
    keep = None
    if f_nodal is not None:
        keep = _f64(f_nodal)
        d.f_nodal = _dp(keep)
    if len(point_loads) > 4 or len(tractions) > 4 or len(omega0_boxes) > 4:
        raise ValueError("at most 4 point loads, tractions and subdomain boxes")
    d.n_point_loads = len(point_loads)
    for i, (node, vec) in enumerate(point_loads):
        d.point_node[i] = int(node)
        for c, v in enumerate(vec):
            d.point_vec[i][c] = v
    d.n_tractions = len(tractions)
    for i, (axis, side, vec) in enumerate(tractions):
        d.traction_face[i] = 2 * axis + side
        for c, v in enumerate(vec):
            d.traction_vec[i][c] = v
    d.volume_target = volume
    d.alpha_mass, d.normal_penalty, d.omega0_weight = alpha_mass, normal_penalty, omega0_weight
    d.n_omega0 = len(omega0_boxes)
    for i, (lo, hi) in enumerate(omega0_boxes):
        for c in range(3):
            d.omega0_lo[i][c] = lo[c] if c < len(lo) else -np.inf
            d.omega0_hi[i][c] = hi[c] if c < len(hi) else np.inf
    d.velocity_dirichlet = int(bool(velocity_dirichlet))
    d.coef_rule = int(coef_rule)
    if load_cases is not None:
        # several load cases: [(point_loads, tractions)] per case (f_nodal belongs to case 0)
        pts = [(k, pl) for k, (pls, _) in enumerate(load_cases) for pl in pls]
        trs = [(k, tr) for k, (_, trl) in enumerate(load_cases) for tr in trl]
        if len(load_cases) > 4 or len(pts) > 4 or len(trs) > 4:
            raise ValueError("at most 4 load cases, 4 point loads and 4 tractions")
        d.n_cases = len(load_cases)
        d.n_point_loads = len(pts)
        for i, (k, (node, vec)) in enumerate(pts):
            d.point_case[i] = k
            d.point_node[i] = int(node)
            for c, v in enumerate(vec):
                d.point_vec[i][c] = v
        d.n_tractions = len(trs)
        for i, (k, (axis, side, vec)) in enumerate(trs):
            d.traction_case[i] = k
            d.traction_face[i] = 2 * axis + side
            for c, v in enumerate(vec):
                d.traction_vec[i][c] = v
    if volume_regions is not None:
        # several volume constraints: [(lo, hi, V)] boxes on the element centroid
        if len(volume_regions) > 4:
            raise ValueError("at most 4 volume constraints")
        d.n_volume = len(volume_regions)
        for j, (lo, hi, V) in enumerate(volume_regions):
            d.volume_V[j] = V
            for c in range(3):
                d.volume_lo[j][c] = lo[c] if c < len(lo) else -np.inf
                d.volume_hi[j][c] = hi[c] if c < len(hi) else np.inf
    kept = [keep]
    if inst_k is not None:
        ik, io = _f64(inst_k), _f64(inst_omega)
        iF = _f64(inst_f).reshape(len(ik), -1)
        if len(io) != len(ik):
            raise ValueError("inst_k and inst_omega differ in length")
        d.n_inst = len(ik)
        d.inst_k, d.inst_omega, d.inst_f = _dp(ik), _dp(io), _dp(iF)
        kept += [ik, io, iF]
    d.growth_rate, d.newton_rtol, d.newton_atol, d.newton_maxit = growth_rate, newton_rtol, newton_atol, newton_maxit
    if inverse:
        d.inverse = 1
        gm = 0
        for axis, side in gamma1:
            gm |= 1 << (2 * axis + side)
        d.gamma1_faces = gm
        mv = _f64(meas).reshape(-1)
        d.meas = _dp(mv)
        d.kv_alpha, d.kv_beta = kv_alpha, kv_beta
        kept.append(mv)
    if u_init is not None:
        ui = _f64(u_init)
        d.u_init = _dp(ui)
        kept.append(ui)
    d._keep = kept                       # keep the arrays alive until fo_problem_create copied them
    return d


class Context:
    def __init__(self, device=0, stream=None, mem_budget=0):
        self.lib = _lib.load()
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(int(stream))
        st = self.lib.fo_ctx_create(device, s, mem_budget, C.byref(h))
        if st != FO_OK:
            raise FormoptError(st, "fo_ctx_create failed")
        self.handle = h
        self._children = []

    def check(self, st, what=""):
        if st != FO_OK:
            msg = self.lib.fo_last_error(self.handle)
            raise FormoptError(st, f"{what}: {msg.decode() if msg else ''}")
        return st

    def memory(self):
        v = C.c_size_t()
        self.check(self.lib.fo_ctx_memory(self.handle, C.byref(v)), "fo_ctx_memory")
        return v.value

    def sync(self):
        self.check(self.lib.fo_ctx_sync(self.handle), "fo_ctx_sync")

    def set_timing(self, on=True):
        self.check(self.lib.fo_ctx_set_timing(self.handle, int(bool(on))), "fo_ctx_set_timing")

    def set_grid_share(self, share):
        self.check(self.lib.fo_ctx_set_grid_share(self.handle, int(share)), "fo_ctx_set_grid_share")

    def solve_kernel_ms(self):
        """Device time of the last multigrid state / adjoint solve's CG launch(es) (timing on)."""
        v = C.c_double()
        self.check(self.lib.fo_ctx_solve_kernel_ms(self.handle, C.byref(v)), "fo_ctx_solve_kernel_ms")
        return v.value

    def selftest_barrier(self, blocks, skip, limit_ms):
        """(status, blocks that gave up) of the bounded grid barrier with block `skip` absent."""
        g = C.c_int(0)
        st = self.lib.fo_selftest_barrier(self.handle, int(blocks), int(skip), float(limit_ms), C.byref(g))
        return st, g.value

    def mesh_box(self, dim, n, lo, hi):
        return Mesh(self, dim, n, lo, hi)

    def mesh_from_arrays(self, coords, cells):
        """A general simplicial mesh from node coordinates [N_n, d] and cells [N_T, d+1]."""
        return Mesh(self, None, None, None, None, arrays=(coords, cells))

    def close(self):
        if self.handle:
            self.lib.fo_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx, dim, n, lo, hi, arrays=None):
        self.ctx = ctx
        h = C.c_void_p()
        if arrays is not None:
            coords = np.ascontiguousarray(arrays[0], dtype=np.float64)
            cells = np.ascontiguousarray(arrays[1], dtype=np.int32)
            dim = coords.shape[1]
            ctx.check(ctx.lib.fo_mesh_from_arrays(ctx.handle, dim, coords.shape[0], coords.ctypes.data_as(C.c_void_p),
                                                  cells.shape[0], cells.ctypes.data_as(C.c_void_p), C.byref(h)),
                      "fo_mesh_from_arrays")
        else:
            nn = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
            lo3 = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
            hi3 = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
            ctx.check(ctx.lib.fo_mesh_box(ctx.handle, dim, nn, lo3, hi3, C.byref(h)), "fo_mesh_box")
        self.handle = h
        info = _lib.MeshInfo()
        ctx.check(ctx.lib.fo_mesh_query(h, C.byref(info)), "fo_mesh_query")
        self.dim = info.dim
        self.n = tuple(info.n[:dim])
        self.num_nodes, self.num_cells, self.num_elems = info.num_nodes, info.num_cells, info.num_elems
        self.volume, self.h = info.volume, info.h

    def copy_out(self):
        cells = np.empty((self.num_elems, self.dim + 1), dtype=np.int32)
        coords = np.empty((self.num_nodes, self.dim), dtype=np.float64)
        self.ctx.check(self.ctx.lib.fo_mesh_copy_out(self.handle, cells.ctypes.data_as(C.c_void_p),
                                                     coords.ctypes.data_as(C.c_void_p)), "fo_mesh_copy_out")
        return cells, coords

    def node_id(self, ijk):
        nid = 0
        for a in reversed(range(self.dim)):
            nid = nid * (self.n[a] + 1) + int(ijk[a])
        return nid

    def problem(self, desc):
        return Problem(self, desc)

    def dirichlet_extension(self, faces, values, opts=None):
        """fo_dirichlet_extension: values [d N_n] kept on the listed faces [(axis, side)],
        extended by the vector Laplacian elsewhere."""
        mask = 0
        for axis, side in faces:
            mask |= 1 << (2 * axis + side)
        v = _f64(values).reshape(-1)
        out = np.empty_like(v)
        self.ctx.check(self.ctx.lib.fo_dirichlet_extension(self.handle, mask, _dp(v), _dp(out),
                                                           C.byref(opts) if opts else None), "fo_dirichlet_extension")
        return out


class Problem:
    def __init__(self, mesh, desc):
        self.mesh, self.ctx = mesh, mesh.ctx
        self.lib = self.ctx.lib
        h = C.c_void_p()
        self.ctx.check(self.lib.fo_problem_create(mesh.handle, C.byref(desc), C.byref(h)), "fo_problem_create")
        self.handle = h
        self.kind = desc.kind
        self.ncomp = mesh.dim if desc.kind == FO_ELASTIC else 1
        self.n_inst = int(desc.n_inst)       # 0: a single problem
        self.n_cases = max(int(desc.n_cases), 1)
        self.nc = int(desc.n_volume) if desc.n_volume > 0 else (1 if desc.volume_target > 0 else 0)

    def _chk(self, st, what):
        return self.ctx.check(st, what)

    def set_levelset(self, phi):
        if _is_device(phi):
            self._chk(self.lib.fo_set_levelset(self.handle, C.c_void_p(phi.data_ptr()), 1), "fo_set_levelset")
        else:
            a = _f64(phi)
            self._chk(self.lib.fo_set_levelset(self.handle, a.ctypes.data_as(C.c_void_p), 0), "fo_set_levelset")

    def initial_level(self, centers, radii, factor=1.0, ord=2):
        c = _f64(centers).reshape(-1)
        r = _f64(radii)
        o = 0 if ord in (np.inf, "inf", 0) else 2
        self._chk(self.lib.fo_initial_level(self.handle, len(r), _dp(c), _dp(r), factor, o), "fo_initial_level")

    def coefficients(self):
        self._chk(self.lib.fo_coefficients(self.handle), "fo_coefficients")

    def state_solve(self, opts=None, allow_noconv=False):
        st = _lib.SolveStats()
        s = self.lib.fo_state_solve(self.handle, C.byref(opts) if opts else None, C.byref(st))
        if not (allow_noconv and s == _lib.FO_ENOCONV):
            self._chk(s, "fo_state_solve")
        return st

    def adjoint_solve(self, opts=None):
        st = _lib.SolveStats()
        self._chk(self.lib.fo_adjoint_solve(self.handle, C.byref(opts) if opts else None, C.byref(st)),
                  "fo_adjoint_solve")
        return st

    def functionals(self):
        J, Cv = C.c_double(), C.c_double()
        self._chk(self.lib.fo_functionals(self.handle, C.byref(J), C.byref(Cv)), "fo_functionals")
        return J.value, Cv.value

    def shape_derivative(self, lam=0.0, copy=True):
        out = np.empty(self.mesh.dim * self.mesh.num_nodes) if copy else None
        ptr = out.ctypes.data_as(C.c_void_p) if copy else None
        self._chk(self.lib.fo_shape_derivative(self.handle, lam, ptr), "fo_shape_derivative")
        return out

    def descent(self, opts=None):
        btt = C.c_double()
        st = _lib.SolveStats()
        self._chk(self.lib.fo_descent(self.handle, C.byref(opts) if opts else None, C.byref(btt), C.byref(st)),
                  "fo_descent")
        return btt.value, st

    def transport_assemble(self, dt, h, smooth):
        self._chk(self.lib.fo_transport_assemble(self.handle, dt, h, int(smooth)), "fo_transport_assemble")

    def levelset_step(self, t_end, nsteps, h, smooth, opts=None):
        st = _lib.SolveStats()
        self._chk(self.lib.fo_levelset_step(self.handle, t_end, nsteps, h, int(smooth),
                                            C.byref(opts) if opts else None, C.byref(st)), "fo_levelset_step")
        return st

    def reinit(self, nsteps, t_final, h, opts=None):
        st = _lib.SolveStats()
        self._chk(self.lib.fo_reinit(self.handle, nsteps, t_final, h, C.byref(opts) if opts else None,
                                     C.byref(st)), "fo_reinit")
        return st

    def opt_step(self, it, opts, ppl=None):
        log = _lib.IterLog()
        self._chk(self.lib.fo_opt_step(self.handle, it, C.byref(opts), C.byref(ppl.state) if ppl else None,
                                       C.byref(log)), "fo_opt_step")
        return log

    def batch_costs(self):
        """Per-instance costs J_i of a batch."""
        out = np.empty(self.n_inst)
        self._chk(self.lib.fo_batch_costs(self.handle, _dp(out)), "fo_batch_costs")
        return out

    def batch_solve_info(self):
        """(active iterations, final relative residual) per instance of the last batched solve."""
        it = np.empty(self.n_inst, dtype=np.int32)
        res = np.empty(self.n_inst)
        self._chk(self.lib.fo_batch_solve_info(self.handle, it.ctypes.data_as(C.POINTER(C.c_int)), _dp(res)),
                  "fo_batch_solve_info")
        return it, res

    def batch_autotune(self, precision=_lib.FO_MIXED):
        r = _lib.TuneResult()
        self._chk(self.lib.fo_batch_autotune(self.handle, precision, C.byref(r)), "fo_batch_autotune")
        return r

    def batch_mg_autotune(self, precision=_lib.FO_MIXED, rtol=1e-8):
        r = _lib.MgTuneResult()
        self._chk(self.lib.fo_batch_mg_autotune(self.handle, precision, float(rtol), C.byref(r)),
                  "fo_batch_mg_autotune")
        return r

    def _field_len(self, field):
        m = self.mesh
        if field in (FO_FIELD_U, FO_FIELD_P, FO_FIELD_LOAD, _lib.FO_FIELD_V, _lib.FO_FIELD_Q, _lib.FO_FIELD_MEAS):
            return self.ncomp * m.num_nodes * max(self.n_inst, 1) * self.n_cases
        if field in (FO_FIELD_THETA, FO_FIELD_RHS):
            return m.dim * m.num_nodes
        if field in (FO_FIELD_COEF, FO_FIELD_CHI, FO_FIELD_OMEGA0):
            return m.num_elems
        return m.num_nodes

    def get(self, field):
        out = np.empty(self._field_len(field))
        self._chk(self.lib.fo_get(self.handle, field, out.ctypes.data_as(C.c_void_p)), "fo_get")
        if self.n_inst and field in (FO_FIELD_U, FO_FIELD_P, FO_FIELD_LOAD):
            return out.reshape(-1, self.n_inst)  # [N_n, n_inst]
        if self.n_cases > 1 and field in (FO_FIELD_U, FO_FIELD_P, FO_FIELD_LOAD):
            return out.reshape(self.n_cases, -1)  # [n_cases, N_dof]
        return out

    def functionals_v(self):
        """(J summed over the load cases, C[0..nc)) with nc the problem's constraint count."""
        J = C.c_double()
        cv = np.zeros(max(self.nc, 1))
        self._chk(self.lib.fo_functionals_v(self.handle, C.byref(J), _dp(cv), self.nc), "fo_functionals_v")
        return J.value, cv[: self.nc]

    def shape_derivative_v(self, lams, copy=True):
        lv = _f64(np.atleast_1d(lams)) if self.nc else np.zeros(1)
        out = np.empty(self.mesh.dim * self.mesh.num_nodes) if copy else None
        self._chk(self.lib.fo_shape_derivative_v(self.handle, _dp(lv), self.nc, _dp(out) if copy else None),
                  "fo_shape_derivative_v")
        return out

    def set(self, field, values):
        if _is_device(values):
            self._chk(self.lib.fo_set(self.handle, field, C.c_void_p(values.data_ptr()), 1), "fo_set")
        else:
            a = _f64(values)
            self._chk(self.lib.fo_set(self.handle, field, a.ctypes.data_as(C.c_void_p), 0), "fo_set")

    def apply(self, op, x):
        x = _f64(x)
        y = np.empty_like(x)
        self._chk(self.lib.fo_apply(self.handle, op, x.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p), 0),
                  "fo_apply")
        return y

    def close(self):
        if self.handle and self.ctx.handle:
            self.lib.fo_problem_destroy(self.handle)
        self.handle = None


class PPL:
    """Host-side PPL state of the library (fo_ppl_init / fo_ppl_update)."""

    def __init__(self, nc=1):
        self.lib = _lib.load()
        self.state = _lib.PPLState()
        self.lib.fo_ppl_init(C.byref(self.state), nc)

    def update(self, C_values, J):
        cv = _f64(np.atleast_1d(C_values))
        lam = np.zeros(4)
        L = C.c_double()
        self.lib.fo_ppl_update(C.byref(self.state), _dp(cv), J, _dp(lam), C.byref(L))
        return lam[: self.state.nc].copy(), L.value


def launch_count():
    """Kernels the library has launched in this process so far."""
    v = C.c_ulonglong()
    _lib.load().fo_launch_count(C.byref(v))
    return v.value


def stop_check(values, constraints=None, start_to_check=30, tol=1e-2, ctrn_tol=1e-2, prev=10):
    """The stopping criterion of Sec. 5.7 (fo_stop_check) at iteration len(values) - 1: values are
    J (no constraints) or L of iterations 0..i, constraints the vector C of iteration i."""
    lib = _lib.load()
    o = _lib.StopOpts(start_to_check, tol, ctrn_tol, prev)
    v = _f64(values)
    nc = 0 if constraints is None else len(np.atleast_1d(constraints))
    cv = _f64(np.atleast_1d(constraints)) if nc else np.zeros(1)
    stop = C.c_int(0)
    lib.fo_stop_check(_dp(v), len(v), _dp(cv), nc, C.byref(o), C.byref(stop))
    return bool(stop.value)


def adaptime(Btt, opts=None):
    lib = _lib.load()
    opts = opts or run_options()
    t, n = C.c_double(), C.c_int()
    lib.fo_adaptime(Btt, C.byref(opts), C.byref(t), C.byref(n))
    return t.value, n.value


# ------------------------------------------------------------------------------ serving
class ServedRequest:
    """A request for Server.submit: one optimisation step (state, explicit adjoint, cost,
    shape derivative, velocity) on its own box mesh.  `desc` is a model_desc (FO_HEAT or
    FO_ELASTIC); the level set is Gaussian bumps (centers [k, dim]) or nodal values phi."""

    def __init__(self, dim, n, desc, lo=None, hi=None, centers=None, width=0.1, offset=0.2, phi=None, lam=0.0,
                 state=None, velocity=None, want_theta=False):
        r = _lib.Request()
        r.dim = dim
        for a in range(3):
            r.n[a] = int(n[a]) if a < dim else 1
            r.lo[a] = (lo[a] if lo is not None else 0.0) if a < dim else 0.0
            r.hi[a] = (hi[a] if hi is not None else 1.0) if a < dim else 1.0
        r.model = desc
        self._keep = [desc]
        if centers is not None:
            c = _f64(centers).reshape(-1)
            r.n_bumps = len(c) // dim
            r.bump_centers = _dp(c)
            r.bump_width, r.bump_offset = width, offset
            self._keep.append(c)
        else:
            ph = _f64(phi)
            r.phi = _dp(ph)
            self._keep.append(ph)
        r.lam = lam
        r.state = state if state is not None else solve_opts()
        r.velocity = velocity if velocity is not None else solve_opts()
        nn = int(np.prod([int(n[a]) + 1 for a in range(dim)]))
        self.theta = np.empty(dim * nn) if want_theta else None
        if want_theta:
            r.theta_out = _dp(self.theta)
        self.struct = r

    def device_bytes(self):
        return int(_lib.load().fo_request_device_bytes(C.byref(self.struct)))


class Server:
    """Continuous-batching request server (fo_server_*): FIFO admission by device memory,
    `executors` requests in flight on their own streams."""

    def __init__(self, ctx=None, executors=8, mem_budget=8 << 30, queue_capacity=4096, dry_run_ms=0.0, grid_share=None,
                 smallest_first=False):
        self.lib = _lib.load()
        o = _lib.ServerOpts()
        self.lib.fo_server_opts_default(C.byref(o))
        o.executors, o.mem_budget, o.queue_capacity, o.dry_run_ms = executors, mem_budget, queue_capacity, dry_run_ms
        if grid_share is not None:
            o.grid_share = int(grid_share)
        o.policy = 1 if smallest_first else 0
        h = C.c_void_p()
        st = self.lib.fo_server_create(ctx.handle if ctx is not None else None, C.byref(o), C.byref(h))
        if st != FO_OK:
            raise FormoptError(st, "fo_server_create failed")
        self.handle = h
        self._pending = {}          # ticket -> request (keeps its output array alive)

    def submit(self, req):
        """Returns (status, ticket); status FO_EBUSY / FO_ENOMEM_BUDGET / FO_EINVAL leave no ticket."""
        t = C.c_uint64()
        st = self.lib.fo_submit(self.handle, C.byref(req.struct), C.byref(t))
        if st == FO_OK:
            self._pending[t.value] = req
            return st, t.value
        return st, None

    def poll(self, ticket):
        r = _lib.Result()
        done = C.c_int()
        st = self.lib.fo_poll(self.handle, ticket, C.byref(r), C.byref(done))
        if st != FO_OK:
            raise FormoptError(st, "fo_poll")
        return bool(done.value), (r if done.value else None)

    def wait(self, ticket, timeout_s=60.0):
        """The result, or None when the request has not completed within timeout_s."""
        r = _lib.Result()
        st = self.lib.fo_wait(self.handle, ticket, float(timeout_s), C.byref(r))
        if st == _lib.FO_ETIMEOUT:
            return None
        if st != FO_OK:
            raise FormoptError(st, "fo_wait")
        return r

    def release(self, ticket):
        st = self.lib.fo_release(self.handle, ticket)
        if st != FO_OK:
            raise FormoptError(st, "fo_release")
        self._pending.pop(ticket, None)

    def stats(self):
        s = _lib.ServerStats()
        self.lib.fo_server_get_stats(self.handle, C.byref(s))
        return s

    def close(self):
        if self.handle:
            self.lib.fo_server_destroy(self.handle)
            self.handle = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
