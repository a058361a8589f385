"""ctypes declarations of the C ABI in include/formopt_gb300.h (argument marshalling only).

The shared library is the in-tree build ``paper_2601_05709_gb300/_build/libformopt_gb300.so``.
There is no fallback: if the library is missing, loading fails loudly.
"""
import ctypes as C
import os

from . import build as _build

FO_OK, FO_EINVAL, FO_ENOMEM, FO_ENOMEM_BUDGET, FO_ECUDA = 0, -1, -2, -3, -4
FO_ENOCONV, FO_ENAN, FO_ETIMEOUT, FO_EBUSY, FO_ESTATE = -5, -6, -7, -8, -9
STATUS_NAMES = {0: "FO_OK", -1: "FO_EINVAL", -2: "FO_ENOMEM", -3: "FO_ENOMEM_BUDGET", -4: "FO_ECUDA",
                -5: "FO_ENOCONV", -6: "FO_ENAN", -7: "FO_ETIMEOUT", -8: "FO_EBUSY", -9: "FO_ESTATE"}

FO_HEAT, FO_ELASTIC, FO_HELMHOLTZ, FO_LOGISTIC = 0, 1, 2, 3
FO_FP64, FO_MIXED = 0, 1
FO_PC_JACOBI, FO_PC_MG = 0, 1
FO_COEF_CENTROID, FO_COEF_CUT = 0, 1
(FO_FIELD_PHI, FO_FIELD_U, FO_FIELD_P, FO_FIELD_THETA, FO_FIELD_RHS, FO_FIELD_COEF, FO_FIELD_CHI,
 FO_FIELD_LOAD, FO_FIELD_OMEGA0, FO_FIELD_V, FO_FIELD_Q, FO_FIELD_MEAS) = range(12)
FO_OP_STATE, FO_OP_VELOCITY, FO_OP_TRANSPORT_L, FO_OP_TRANSPORT_R, FO_OP_STATE_FP32 = range(5)

D3 = C.c_double * 3
D43 = (C.c_double * 3) * 4


class MeshInfo(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", D3), ("hi", D3), ("num_nodes", C.c_int64),
                ("num_cells", C.c_int64), ("num_elems", C.c_int64), ("volume", C.c_double), ("h", C.c_double)]


class ModelDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("a_in", C.c_double), ("a_out", C.c_double), ("E", C.c_double),
                ("nu", C.c_double), ("k", C.c_double), ("omega", C.c_double), ("dirichlet_faces", C.c_uint32),
                ("f_nodal", C.POINTER(C.c_double)), ("n_point_loads", C.c_int), ("point_node", C.c_int64 * 4),
                ("point_vec", D43), ("n_tractions", C.c_int), ("traction_face", C.c_int * 4),
                ("traction_vec", D43), ("volume_target", C.c_double), ("alpha_mass", C.c_double),
                ("normal_penalty", C.c_double), ("omega0_weight", C.c_double), ("n_omega0", C.c_int),
                ("omega0_lo", D43), ("omega0_hi", D43), ("velocity_dirichlet", C.c_int),
                ("n_inst", C.c_int), ("inst_k", C.POINTER(C.c_double)), ("inst_omega", C.POINTER(C.c_double)),
                ("inst_f", C.POINTER(C.c_double)), ("coef_rule", C.c_int), ("n_cases", C.c_int),
                ("point_case", C.c_int * 4), ("traction_case", C.c_int * 4), ("n_volume", C.c_int),
                ("volume_lo", D43), ("volume_hi", D43), ("volume_V", C.c_double * 4),
                ("growth_rate", C.c_double), ("u_init", C.POINTER(C.c_double)), ("newton_rtol", C.c_double),
                ("newton_atol", C.c_double), ("newton_maxit", C.c_int), ("inverse", C.c_int),
                ("gamma1_faces", C.c_uint32), ("meas", C.POINTER(C.c_double)), ("kv_alpha", C.c_double),
                ("kv_beta", C.c_double)]


class MgTuneResult(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_int), ("nu0", C.c_int), ("inst_levels", C.c_int), ("ms", C.c_double),
                ("iterations", C.c_int), ("candidates", C.c_int), ("tile", C.c_int * 3)]


class TuneResult(C.Structure):
    _fields_ = [("block", C.c_int), ("blocks_per_sm", C.c_int), ("us_per_iteration", C.c_double),
                ("candidates", C.c_int), ("tile", C.c_int * 3)]


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int), ("warm_start", C.c_int),
                ("inner_rtol", C.c_double), ("inner_maxit", C.c_int), ("grid_blocks", C.c_int),
                ("precond", C.c_int), ("mg_bf16", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer_iterations", C.c_int), ("operator_applies", C.c_int),
                ("rel_residual", C.c_double)]


class Request(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("model", ModelDesc), ("n_bumps", C.c_int), ("bump_centers", C.POINTER(C.c_double)),
                ("bump_width", C.c_double), ("bump_offset", C.c_double), ("phi", C.POINTER(C.c_double)),
                ("lam", C.c_double), ("state", SolveOpts), ("velocity", SolveOpts),
                ("theta_out", C.POINTER(C.c_double))]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("message", C.c_char * 128), ("J", C.c_double), ("C", C.c_double),
                ("Btt", C.c_double), ("state", SolveStats), ("adjoint", SolveStats), ("velocity", SolveStats),
                ("dofs", C.c_int64), ("device_bytes", C.c_size_t), ("submit_ms", C.c_double),
                ("start_ms", C.c_double), ("end_ms", C.c_double)]


class ServerOpts(C.Structure):
    _fields_ = [("executors", C.c_int), ("mem_budget", C.c_size_t), ("queue_capacity", C.c_int),
                ("dry_run_ms", C.c_double), ("grid_share", C.c_int), ("policy", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("rejected", C.c_int64),
                ("peak_in_flight", C.c_int64), ("peak_bytes", C.c_size_t)]


class RunOptions(C.Structure):
    _fields_ = [("dfactor", C.c_double), ("t_min", C.c_double), ("t_max", C.c_double), ("s_min", C.c_int),
                ("s_max", C.c_int), ("smooth", C.c_int), ("reinit_step", C.c_int), ("reinit_steps", C.c_int),
                ("reinit_time", C.c_double), ("h", C.c_double), ("state", SolveOpts), ("velocity", SolveOpts),
                ("transport", SolveOpts)]


class PPLState(C.Structure):
    _fields_ = [("nc", C.c_int), ("r", C.c_double), ("delta", C.c_double), ("alpha", C.c_double),
                ("beta", C.c_double), ("z", C.c_double * 4), ("lam", C.c_double * 4), ("mu", C.c_double * 4)]


class IterLog(C.Structure):
    _fields_ = [("J", C.c_double), ("C", C.c_double), ("L", C.c_double), ("lam", C.c_double),
                ("Btt", C.c_double), ("t_end", C.c_double), ("nsteps", C.c_int), ("reinit", C.c_int),
                ("state", SolveStats), ("velocity", SolveStats), ("transport", SolveStats),
                ("reinit_stats", SolveStats), ("ms_state", C.c_double), ("ms_functionals", C.c_double),
                ("ms_shape", C.c_double), ("ms_velocity", C.c_double), ("ms_transport", C.c_double),
                ("ms_reinit", C.c_double), ("ms_state_kernel", C.c_double), ("nc", C.c_int),
                ("Cv", C.c_double * 4), ("lambdav", C.c_double * 4), ("adjoint", SolveStats),
                ("newton_steps", C.c_int)]


class StopOpts(C.Structure):
    _fields_ = [("start_to_check", C.c_int), ("tol", C.c_double), ("ctrn_tol", C.c_double), ("prev", C.c_int)]


VP = C.c_void_p
DP = C.POINTER(C.c_double)
ST = C.c_int

# name -> (restype, argtypes)
FO_MAX_INSTANCES = 128

PROTOTYPES = {
    "fo_ctx_create": (ST, [C.c_int, VP, C.c_size_t, C.POINTER(VP)]),
    "fo_ctx_destroy": (ST, [VP]),
    "fo_last_error": (C.c_char_p, [VP]),
    "fo_ctx_memory": (ST, [VP, C.POINTER(C.c_size_t)]),
    "fo_ctx_sync": (ST, [VP]),
    "fo_ctx_set_timing": (ST, [VP, C.c_int]),
    "fo_ctx_set_grid_share": (ST, [VP, C.c_int]),
    "fo_ctx_solve_kernel_ms": (ST, [VP, DP]),
    "fo_launch_count": (ST, [C.POINTER(C.c_ulonglong)]),
    "fo_mesh_box": (ST, [VP, C.c_int, C.POINTER(C.c_int), DP, DP, C.POINTER(VP)]),
    "fo_mesh_from_arrays": (ST, [VP, C.c_int, C.c_int64, VP, C.c_int64, VP, C.POINTER(VP)]),
    "fo_functionals_v": (ST, [VP, DP, DP, C.c_int]),
    "fo_shape_derivative_v": (ST, [VP, DP, C.c_int, DP]),
    "fo_stop_opts_default": (None, [VP]),
    "fo_stop_check": (None, [DP, C.c_int, DP, C.c_int, VP, C.POINTER(C.c_int)]),
    "fo_mesh_destroy": (ST, [VP]),
    "fo_mesh_query": (ST, [VP, C.POINTER(MeshInfo)]),
    "fo_mesh_copy_out": (ST, [VP, VP, VP]),
    "fo_problem_create": (ST, [VP, C.POINTER(ModelDesc), C.POINTER(VP)]),
    "fo_problem_destroy": (ST, [VP]),
    "fo_set_levelset": (ST, [VP, VP, C.c_int]),
    "fo_initial_level": (ST, [VP, C.c_int, DP, DP, C.c_double, C.c_int]),
    "fo_coefficients": (ST, [VP]),
    "fo_state_solve": (ST, [VP, C.POINTER(SolveOpts), C.POINTER(SolveStats)]),
    "fo_state_solve_noalloc": (ST, [VP, VP, VP, C.POINTER(SolveOpts), C.POINTER(SolveStats)]),
    "fo_selftest_barrier": (ST, [VP, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int)]),
    "fo_adjoint_solve": (ST, [VP, C.POINTER(SolveOpts), C.POINTER(SolveStats)]),
    "fo_functionals": (ST, [VP, DP, DP]),
    "fo_shape_derivative": (ST, [VP, C.c_double, VP]),
    "fo_descent": (ST, [VP, C.POINTER(SolveOpts), DP, C.POINTER(SolveStats)]),
    "fo_transport_assemble": (ST, [VP, C.c_double, C.c_double, C.c_int]),
    "fo_levelset_step": (ST, [VP, C.c_double, C.c_int, C.c_double, C.c_int, C.POINTER(SolveOpts),
                              C.POINTER(SolveStats)]),
    "fo_reinit": (ST, [VP, C.c_int, C.c_double, C.c_double, C.POINTER(SolveOpts), C.POINTER(SolveStats)]),
    "fo_opt_step": (ST, [VP, C.c_int, C.POINTER(RunOptions), C.POINTER(PPLState), C.POINTER(IterLog)]),
    "fo_get": (ST, [VP, C.c_int, VP]),
    "fo_set": (ST, [VP, C.c_int, VP, C.c_int]),
    "fo_apply": (ST, [VP, C.c_int, VP, VP, C.c_int]),
    "fo_levelset_bumps": (ST, [VP, C.c_int, DP, C.c_double, C.c_double]),
    "fo_server_opts_default": (None, [C.POINTER(ServerOpts)]),
    "fo_request_device_bytes": (C.c_size_t, [C.POINTER(Request)]),
    "fo_server_create": (ST, [VP, C.POINTER(ServerOpts), C.POINTER(VP)]),
    "fo_server_destroy": (ST, [VP]),
    "fo_submit": (ST, [VP, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "fo_poll": (ST, [VP, C.c_uint64, C.POINTER(Result), C.POINTER(C.c_int)]),
    "fo_wait": (ST, [VP, C.c_uint64, C.c_double, C.POINTER(Result)]),
    "fo_release": (ST, [VP, C.c_uint64]),
    "fo_server_get_stats": (ST, [VP, C.POINTER(ServerStats)]),
    "fo_batch_costs": (ST, [VP, DP]),
    "fo_batch_solve_info": (ST, [VP, C.POINTER(C.c_int), DP]),
    "fo_batch_autotune": (ST, [VP, C.c_int, C.POINTER(TuneResult)]),
    "fo_batch_mg_autotune": (ST, [VP, C.c_int, C.c_double, C.POINTER(MgTuneResult)]),
    "fo_dirichlet_extension": (ST, [VP, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(SolveOpts)]),
    "fo_ppl_init": (None, [C.POINTER(PPLState), C.c_int]),
    "fo_ppl_update": (None, [C.POINTER(PPLState), DP, C.c_double, DP, DP]),
    "fo_adaptime": (None, [C.c_double, C.POINTER(RunOptions), DP, C.POINTER(C.c_int)]),
    "fo_run_options_default": (None, [C.POINTER(RunOptions)]),
    "fo_solve_opts_default": (None, [C.POINTER(SolveOpts)]),
}

_LIB = None


def load():
    """Load the in-tree library (build it first with __graft_entry__.build())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class FormoptError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
