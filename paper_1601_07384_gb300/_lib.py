"""ctypes declarations of the C ABI in include/stdg.h (argument marshalling only)."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstdg.so")

STATUS = {0: "STDG_OK", -1: "STDG_EINVAL", -2: "STDG_ENOMEM", -3: "STDG_ECUDA", -4: "STDG_ENOCONV",
          -5: "STDG_EMESH", -6: "STDG_ENAN", -7: "STDG_ETIMEOUT", -8: "STDG_EUNSUPPORTED"}
SOLVER = {"gmres": 0, "cg": 1, "kron_cg": 2, "kron_pcg": 3, "fgmres_bj": 4, "fgmres_gnn": 5, "kron_mg": 6,
          "kron_mg_gnn": 7}
PREC = {"fp64": 0, "df32": 1, "mixed_f32": 2, "mixed_bf16": 3}
FIELD = {"zero": 0, "constant": 1, "beltrami": 2, "curl_modes": 3}


class StdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("rel_residual", C.c_double),
                ("seconds", C.c_double), ("fallback", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("picard", C.c_int), ("press_iters", C.c_int * 8), ("visc_iters", C.c_int * 8),
                ("press_residual", C.c_double * 8), ("seconds", C.c_double),
                ("max_divergence", C.c_double), ("fallbacks", C.c_int)]


class SolverOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("restart", C.c_int), ("max_iters", C.c_int), ("graph_batch", C.c_int)]


class ProfileStats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("operator_launches", C.c_int64), ("operator_ms", C.c_double),
                ("kind_launches", C.c_int64 * 4), ("kind_ms", C.c_double * 4), ("phase_ms", C.c_double * 8)]


class Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("c", C.c_double * 3), ("a", C.c_double), ("d", C.c_double),
                ("nu", C.c_double), ("nmodes", C.c_int), ("modes", C.POINTER(C.c_double))]


# stdg_vel_fn, stdg_alloc_fn, stdg_free_fn
VEL_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double), C.c_void_p)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


P = C.c_void_p
I64P = C.POINTER(C.c_int64)
I32P = C.POINTER(C.c_int32)
DP = C.POINTER(C.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "stdg_mesh_create": (C.c_int, [DP, C.c_int64, I64P, C.c_int64, C.POINTER(P)]),
    "stdg_mesh_create_periodic": (C.c_int, [DP, C.c_int64, I64P, C.c_int64, DP, C.POINTER(P)]),
    "stdg_mesh_destroy": (None, [P]),
    "stdg_mesh_info": (C.c_int, [P, I64P, I64P, I64P, I64P]),
    "stdg_mesh_faces": (C.c_int, [P, I64P, I64P, I32P, I32P]),
    "stdg_reference_matrices": (C.c_int, [C.c_int, C.c_int, C.POINTER(P)]),
    "stdg_ref_destroy": (None, [P]),
    "stdg_ref_time_matrix": (C.c_int, [P, DP]),
    "stdg_time_blockdiag": (C.c_int, [DP, C.c_int, DP, DP, DP, C.POINTER(C.c_int)]),
    "stdg_mesh_agglomerate": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                        C.POINTER(C.c_int)]),
    "stdg_ref_eval": (C.c_int, [P, DP, C.c_int64, DP, DP]),
    "stdg_tet_rule": (C.c_int, [C.c_int, DP, DP]),
    "stdg_solver_create": (C.c_int, [P, P, C.c_double, C.POINTER(SolverOptions), P, C.POINTER(P)]),
    "stdg_solver_create_alloc": (C.c_int, [P, P, C.c_double, C.POINTER(SolverOptions), P, ALLOC_FN, FREE_FN, P,
                                           C.POINTER(P)]),
    "stdg_solver_destroy": (None, [P]),
    "stdg_set_dt": (C.c_int, [P, C.c_double]),
    "stdg_set_max_iters": (C.c_int, [P, C.c_int]),
    "stdg_pressure_apply": (C.c_int, [P, P, P, C.c_int]),
    "stdg_pressure_apply_f32": (C.c_int, [P, P, P, C.c_int]),
    "stdg_pressure_apply_factored": (C.c_int, [P, P, P, C.c_int]),
    "stdg_pressure_rhs": (C.c_int, [P, P, P, C.c_int]),
    "stdg_velocity_update": (C.c_int, [P, P, P, P]),
    "stdg_solve": (C.c_int, [P, P, P, C.c_double, C.c_int, C.POINTER(SolveStats)]),
    "stdg_solve_noalloc": (C.c_int, [P, P, P, C.c_double, C.POINTER(SolveStats)]),
    "stdg_set_initial": (C.c_int, [P, C.POINTER(Field)]),
    "stdg_set_boundary": (C.c_int, [P, C.POINTER(Field)]),
    "stdg_set_initial_fn": (C.c_int, [P, VEL_FN, P]),
    "stdg_set_boundary_fn": (C.c_int, [P, VEL_FN, P]),
    "stdg_step": (C.c_int, [P, C.c_double, C.c_int, C.c_int, C.c_double, C.POINTER(StepStats)]),
    "stdg_set_theta": (C.c_int, [P, C.c_double]),
    "stdg_get_state": (C.c_int, [P, P, P, C.c_int, DP]),
    "stdg_set_state": (C.c_int, [P, P, P, C.c_int, C.c_double]),
    "stdg_velocity_moments": (C.c_int, [P, P, P]),
    "stdg_convection": (C.c_int, [P, P, P]),
    "stdg_get_blocks": (C.c_int, [P, DP, DP, DP, DP]),
    "stdg_profile": (C.c_int, [P, C.c_int]),
    "stdg_gnn_init": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_uint64]),
    "stdg_gnn_layout": (C.c_int, [P, I64P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "stdg_gnn_params": (C.c_int, [P, C.POINTER(C.c_float), C.POINTER(C.c_float), I64P]),
    "stdg_gnn_apply": (C.c_int, [P, P, P]),
    "stdg_gnn_loss_grad": (C.c_int, [P, P, P, C.c_int, DP, C.POINTER(C.c_float)]),
    "stdg_gnn_harvest": (C.c_int, [P, P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "stdg_gnn_train": (C.c_int, [P, C.c_int, C.c_double, C.c_int, DP, DP]),
    "stdg_gnn_autoharvest": (C.c_int, [P, C.c_int, C.c_int, C.c_int]),
    "stdg_gnn_autoharvest_mg": (C.c_int, [P, C.c_int, C.c_int]),
    "stdg_profile_read": (C.c_int, [P, C.POINTER(ProfileStats)]),
    "stdg_fma_probe": (C.c_int, [DP, DP, P]),
    "stdg_tc_gemm_bf16": (C.c_int, [P, C.c_int64, P, C.c_int64, P, C.c_int64, C.c_int, C.c_int, C.c_int, P]),
    "stdg_last_error": (C.c_char_p, []),
    "stdg_version": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libstdg.so (fails loudly: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libstdg.so not built ({path}); run paper_1601_07384_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status):
    if status != 0:
        msg = _lib.stdg_last_error().decode(errors="replace") if _lib else ""
        raise StdgError(status, msg)
