"""ctypes mirror of include/llg.h (structures, status codes, prototypes).

Loading fails loudly if the CUDA library has not been built: there is no
fallback implementation anywhere in the package.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libllg_b300.so")

LLG_OK = 0
STATUS = {
    0: "LLG_OK",
    1: "LLG_ERR_INVALID_ARG",
    2: "LLG_ERR_UNSUPPORTED_SIZE",
    3: "LLG_ERR_NOT_CONVERGED",
    4: "LLG_ERR_BREAKDOWN",
    5: "LLG_ERR_DEGENERATE_NODE",
    6: "LLG_ERR_TIMEOUT",
    7: "LLG_ERR_OOM",
    8: "LLG_ERR_CUDA",
}
EX_SPECTRAL, EX_FD2 = 0, 1
PREC_FP64, PREC_FP32_FLEX = 0, 1
PC_FFTHSS, PC_HERMITIAN, PC_NONE = 0, 1, 2
GS_FP64, GS_F32X2 = 0, 1
CHAIN_FP64, CHAIN_F32X2 = 0, 1
PLAN_FIVE, PLAN_CLUSTER = 0, 1

# every symbol the header declares, in declaration order
EXPORTS = [
    "llg_create", "llg_destroy", "llg_last_error", "llg_set_stream", "llg_launch_count", "llg_nodes",
    "llg_saddle_apply", "llg_saddle_apply_f32x2", "llg_ffthss_apply", "llg_ffthss_apply_f32", "llg_ffthss_apply_noalloc",
    "llg_precond_saddle_apply",
    "llg_gmres_solve", "llg_step_euler", "llg_step_midpoint", "llg_adjoint_step", "llg_energy",
    "llg_lower_order_field",
    "llg_ensemble_create", "llg_ensemble_run", "llg_ensemble_set_blocks", "llg_ensemble_max_blocks",
    "llg_ensemble_autotune", "llg_ensemble_set_barrier_test", "llg_ensemble_destroy", "llg_ensemble_last_error",
    "llg_set_pass_plan", "llg_autotune", "llg_set_axis_shape", "llg_profile_begin", "llg_profile_end", "llg_krylov_orthogonality", "llg_probe_fma_rate",
    "llg_check_conversions",
]
KCLASS = {"xfwd": 1, "axis": 2, "xinv": 3, "arnoldi": 4}


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3)]


class Params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("c_ex", C.c_double), ("k", C.c_double), ("theta", C.c_double),
                ("lam", C.c_double), ("h_ext", C.c_double * 3), ("exchange", C.c_int), ("h_field", C.c_void_p),
                ("k_an", C.c_double), ("e_an", C.c_double * 3), ("demag", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("restart", C.c_int), ("max_iters", C.c_int), ("rtol", C.c_double), ("precision", C.c_int),
                ("picard_max", C.c_int), ("picard_tol", C.c_double), ("diagnostics", C.c_int),
                ("preconditioner", C.c_int), ("gs_arith", C.c_int),
                ("chain_arith", C.c_int)]


class Problem(C.Structure):
    _fields_ = [("n", C.c_int * 2), ("L", C.c_double * 2), ("prm", Params), ("m", C.c_void_p), ("x", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("picard_iters", C.c_int), ("applies", C.c_int),
                ("rel_res_true", C.c_double), ("max_len_drift", C.c_double), ("energy_before", C.c_double),
                ("energy_after", C.c_double), ("dissipation_residual", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load the library (raises if it is missing: the package has no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"CUDA library {LIB_PATH} is missing; build it with "
            "`python -m paper_2607_15290_b300.build` (nvcc, sm_103a)")
    L = C.CDLL(LIB_PATH)
    P, vp, d = C.POINTER, C.c_void_p, C.POINTER(C.c_double)
    ctx = vp
    L.llg_create.argtypes = [P(Grid), vp, P(vp)]
    L.llg_destroy.argtypes = [ctx]
    L.llg_last_error.argtypes = [ctx]
    L.llg_last_error.restype = C.c_char_p
    L.llg_set_stream.argtypes = [ctx, vp]
    L.llg_launch_count.argtypes = [ctx]
    L.llg_launch_count.restype = C.c_longlong
    L.llg_nodes.argtypes = [ctx]
    L.llg_nodes.restype = C.c_longlong
    L.llg_saddle_apply.argtypes = [ctx, P(Params), vp, vp, vp, C.c_int]
    L.llg_saddle_apply_f32x2.argtypes = [ctx, P(Params), vp, vp, vp, C.c_int]
    L.llg_ffthss_apply.argtypes = [ctx, P(Params), vp, vp, vp, C.c_int]
    L.llg_ffthss_apply_f32.argtypes = [ctx, P(Params), vp, vp, vp, C.c_int]
    L.llg_ffthss_apply_noalloc.argtypes = [P(Grid), P(Params), vp, vp, vp, C.c_int, vp]
    L.llg_precond_saddle_apply.argtypes = [ctx, P(Params), vp, vp, vp]
    L.llg_gmres_solve.argtypes = [ctx, P(Params), P(Opts), vp, vp, vp, P(Info)]
    L.llg_step_euler.argtypes = [ctx, P(Params), P(Opts), vp, vp, vp, P(Info)]
    L.llg_step_midpoint.argtypes = [ctx, P(Params), P(Opts), vp, vp, vp, vp, P(Info)]
    L.llg_adjoint_step.argtypes = [ctx, P(Params), P(Opts), vp, vp, vp, vp, d, d, P(Info)]
    L.llg_energy.argtypes = [ctx, P(Params), vp, d]
    L.llg_lower_order_field.argtypes = [ctx, P(Params), vp, vp]
    L.llg_autotune.argtypes = [ctx, C.c_int, C.c_char_p, C.c_int]
    L.llg_set_axis_shape.argtypes = [ctx, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
    L.llg_set_pass_plan.argtypes = [ctx, C.c_int]
    L.llg_ensemble_create.argtypes = [P(Problem), C.c_int, P(Opts), vp, P(vp)]
    L.llg_ensemble_run.argtypes = [vp, C.c_int, P(Info), P(C.c_int)]
    L.llg_ensemble_set_blocks.argtypes = [vp, C.c_int]
    L.llg_ensemble_max_blocks.argtypes = [vp]
    L.llg_ensemble_autotune.argtypes = [vp, P(C.c_int)]
    L.llg_ensemble_set_barrier_test.argtypes = [vp, C.c_longlong, C.c_int]
    L.llg_ensemble_destroy.argtypes = [vp]
    L.llg_ensemble_last_error.argtypes = [vp]
    L.llg_ensemble_last_error.restype = C.c_char_p
    L.llg_profile_begin.argtypes = [ctx, C.c_int]
    L.llg_profile_end.argtypes = [ctx, d, P(C.c_longlong), d, d]
    L.llg_krylov_orthogonality.argtypes = [ctx, d, P(C.c_int)]
    L.llg_probe_fma_rate.argtypes = [ctx, C.c_int, d]
    L.llg_check_conversions.argtypes = [ctx, C.c_longlong, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    for name in EXPORTS:
        if name not in ("llg_last_error", "llg_launch_count", "llg_nodes", "llg_ensemble_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L
