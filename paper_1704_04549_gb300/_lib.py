"""ctypes declarations of the libtpp C ABI (include/tpp.h).  Marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtpp.so")

TPP_OK = 0
STATUS_NAMES = {0: "TPP_OK", 1: "TPP_ERR_INVALID_ARG", 2: "TPP_ERR_CUDA",
                3: "TPP_ERR_SINGULAR_FACTOR", 4: "TPP_ERR_NOT_CONVERGED", 5: "TPP_ERR_BREAKDOWN",
                6: "TPP_ERR_SCHUR", 7: "TPP_ERR_NAN", 8: "TPP_ERR_UNSUPPORTED",
                9: "TPP_ERR_WORKSPACE", 10: "TPP_ERR_TIMEOUT"}
TPP_FP64, TPP_FP32, TPP_BF16 = 0, 1, 2
TPP_PC_NONE, TPP_PC_KRON, TPP_PC_BLOCK_JACOBI = 0, 1, 2
TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_MIXED, TPP_FEAT_TWO_SIDED, TPP_FEAT_LEARNED = 1, 2, 4, 8
TPP_FEAT_TIME = 16
TPP_FEAT_BF16 = 32
TPP_FEAT_FULL_BLOCKS = 64
TPP_FEAT_F32_SHIFTS = 128
TPP_TS_BACKWARD_EULER, TPP_TS_DIRK3, TPP_TS_RK4 = 0, 1, 2


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32), ("num_elem", C.c_int64),
                ("nrhs", C.c_int32), ("mu", C.c_int32), ("h", C.c_double),
                ("dt", C.c_double), ("vel_nodes", C.c_void_p), ("vel_face_normal", C.c_void_p),
                ("nbr", C.c_void_p)]


class GmresOpts(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_iters", C.c_int32), ("rtol", C.c_double),
                ("pc", C.c_int32), ("inner_prec", C.c_int32), ("flexible", C.c_int32),
                ("inner_iters", C.c_int32), ("use_graph", C.c_int32), ("inner_rtol", C.c_double)]


class GmresResult(C.Structure):
    _fields_ = [("iters", C.c_int32), ("cycles", C.c_int32), ("status", C.c_int32),
                ("converged", C.c_int32), ("true_rel_res", C.c_double),
                ("est_rel_res", C.c_double), ("inner_iters", C.c_int32), ("reserved", C.c_int32)]


class BuildReport(C.Structure):
    _fields_ = [("num_elem", C.c_int32), ("num_shifted", C.c_int32), ("num_rank1", C.c_int32),
                ("num_schur_fail", C.c_int32), ("max_cond", C.c_double),
                ("min_sigma_ratio", C.c_double), ("max_cond_z", C.c_double),
                ("num_z_unconverged", C.c_int32), ("num_fallback", C.c_int32),
                ("num_schur_relaxed", C.c_int32)]


TPP_FLUX_EULER = 1


class SysProblem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32), ("num_elem", C.c_int64),
                ("nc", C.c_int32), ("flux", C.c_int32), ("gamma", C.c_double),
                ("h", C.c_double), ("dt", C.c_double), ("state", C.c_void_p),
                ("nbr", C.c_void_p)]


class BatchOpts(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_iters", C.c_int32), ("rtol", C.c_double),
                ("prec", C.c_int32), ("max_outer", C.c_int32), ("inner_rtol", C.c_double),
                ("warps", C.c_int32 * 3), ("ctas_per_sm", C.c_int32 * 3),
                ("reg_budget", C.c_int32 * 3), ("iters", C.c_void_p), ("relres", C.c_void_p)]


class BatchReport(C.Structure):
    _fields_ = [("systems", C.c_int64), ("total_iters", C.c_int64), ("max_iters", C.c_int32),
                ("unconverged", C.c_int32), ("max_outer", C.c_int32), ("launches", C.c_int32),
                ("max_relres", C.c_double), ("launch_ms", C.c_double * 3)]


class TimeReport(C.Structure):
    _fields_ = [("steps", C.c_int32), ("gmres_iters", C.c_int32), ("builds", C.c_int32),
                ("solves", C.c_int32), ("max_true_rel_res", C.c_double)]


class Views(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in
                ("sigma", "A1", "B1", "A2", "B2", "SA", "SB", "Q1", "Q2", "T1", "T2", "flags",
                 "cond", "gl_x", "gl_w", "D", "Az", "Azi", "sigz", "zflags", "G", "core", "Qb",
                 "Rb", "qtr", "fA", "fB", "fsig", "fflags")]


EXPORTS = {
    "tpp_workspace_bytes": (C.c_size_t, [C.POINTER(Problem), C.c_int32, C.c_uint32]),
    "tpp_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Problem), C.c_int32, C.c_uint32,
                             C.c_void_p, C.c_size_t, C.c_void_p]),
    "tpp_destroy": (None, [C.c_void_p]),
    "tpp_build_factors": (C.c_int, [C.c_void_p, C.POINTER(BuildReport), C.c_void_p]),
    "tpp_build_block_jacobi": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tpp_set_velocity": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "tpp_gauss_legendre": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tpp_apply_inverse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                    C.c_void_p]),
    "tpp_apply_block_jacobi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                         C.c_void_p]),
    "dg_apply_sumfact": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "dg_apply_sumfact_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                          C.c_void_p]),
    "dg_apply_sumfact_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                       C.c_void_p]),
    "tpp_apply_inverse_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                        C.c_void_p]),
    "tpp_set_metric_terms": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_double, C.c_void_p]),
    "tpp_sys_workspace_bytes": (C.c_size_t, [C.POINTER(SysProblem), C.c_int32, C.c_uint32]),
    "tpp_create_system": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(SysProblem), C.c_int32,
                                    C.c_uint32, C.c_void_p, C.c_size_t, C.c_void_p]),
    "tpp_batch_workspace_bytes": (C.c_size_t, [C.c_void_p, C.c_int32, C.POINTER(BatchOpts)]),
    "tpp_batch_gmres": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                  C.POINTER(BatchOpts), C.POINTER(BatchReport), C.c_void_p,
                                  C.c_size_t, C.c_void_p]),
    "gmres_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(GmresOpts),
                              C.POINTER(GmresResult), C.c_void_p]),
    "tpp_get_views": (C.c_int, [C.c_void_p, C.POINTER(Views)]),
    "tpp_mass_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_void_p,
                                 C.c_void_p]),
    "tpp_time_integrate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_int32,
                                     C.c_int32, C.POINTER(GmresOpts), C.POINTER(TimeReport),
                                     C.c_void_p]),
    "tpp_copy_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "tpp_num_dofs": (C.c_int64, [C.c_void_p]),
    "tpp_num_elem": (C.c_int64, [C.c_void_p]),
    "tpp_last_error": (C.c_char_p, []),
    "tpp_kernel_launch_count": (C.c_int64, []),
    "tpp_probe_fma_rate": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_void_p]),
    "tpp_core_size": (C.c_int32, [C.c_void_p]),
    "tpp_learned_inputs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tpp_build_factors_learned": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double,
                                            C.POINTER(BuildReport), C.c_void_p]),
    "tpp_mlp_num_params": (C.c_int64, [C.c_int32]),
    "tpp_mlp_workspace_bytes": (C.c_size_t, [C.c_int32, C.c_int32]),
    "tpp_mlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_void_p,
                                 C.c_size_t, C.c_void_p]),
    "tpp_mlp_destroy": (None, [C.c_void_p]),
    "tpp_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tpp_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tpp_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "tpp_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                     C.c_float, C.c_void_p, C.c_void_p]),
    "tpp_mlp_gradients": (C.c_void_p, [C.c_void_p]),
    "tpp_mlp_element_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                       C.c_void_p, C.c_void_p]),
    "tpp_solve_learned": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_void_p,
                                    C.c_void_p, C.POINTER(GmresOpts), C.POINTER(GmresResult),
                                    C.POINTER(BuildReport), C.POINTER(C.c_int32), C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libtpp.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_1704_04549_gb300.build.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TppError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().tpp_last_error().decode()
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str):
    if status != TPP_OK:
        raise TppError(status, where)
