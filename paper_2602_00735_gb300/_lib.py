"""ctypes declarations of libraspml.so (include/raspml.h). Marshalling only."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libraspml.so")

OK, NOT_CONVERGED = 0, 1
ERRORS = {-1: "EBADARG", -2: "ENOMEM", -3: "ECUDA", -4: "EPIVOT", -5: "ENAN", -6: "ETIMEOUT", -7: "ESTATE"}

#: every entry point declared in include/raspml.h
SYMBOLS = ("ras_pml_setup", "ras_pml_info", "ras_pml_num_unknowns", "ras_pml_assemble_rhs", "ras_pml_assemble_rhs_noalloc",
           "ras_pml_factor", "ras_pml_apply",
           "ras_pml_matvec", "helmholtz_solve", "helmholtz_solve_host", "ras_pml_richardson",
           "ras_pml_history", "ras_pml_set_timing", "ras_pml_get_timing", "ras_pml_error_string",
           "ras_pml_destroy", "ras_pml_tune", "ras_pml_set_shapes", "ras_pml_batch_set_shapes",
           "ras_pml_batch_setup", "ras_pml_batch_info", "ras_pml_batch_layout", "ras_pml_batch_assemble_rhs",
           "ras_pml_batch_factor", "ras_pml_batch_tune", "ras_pml_batch_apply", "ras_pml_batch_matvec",
           "ras_pml_batch_solve", "ras_pml_batch_destroy",
           "ras_pml_net_create", "ras_pml_net_param_count", "ras_pml_net_set_params", "ras_pml_net_get_params",
           "ras_pml_net_forward", "ras_pml_net_loss_grad", "ras_pml_net_adam_step", "ras_pml_net_set_gamma",
           "ras_pml_net_get_gamma", "ras_pml_net_train", "ras_pml_net_destroy", "ras_pml_attach_net",
           "ras_pml_get_params", "ras_pml_net_correct", "ras_pml_set_copy_wait_limit",
           "ras_pml_fma_peak")
VOID_SYMBOLS = ("ras_pml_error_string", "ras_pml_destroy", "ras_pml_batch_destroy", "ras_pml_net_destroy",
                "ras_pml_net_get_gamma")


class Params(ctypes.Structure):
    _fields_ = [("k", c_double), ("x0", c_double), ("y0", c_double), ("x1", c_double), ("y1", c_double),
                ("kappa_g", c_double), ("h", c_double), ("px", c_int), ("py", c_int),
                ("ovlp_cells", c_int), ("pml_cells", c_int), ("g_amp", c_double), ("g_ramp", c_double),
                ("local_bc", c_int), ("factor_prec", c_int), ("ortho", c_int),
                ("g_profile", c_int), ("form", c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n", c_int64), ("Mx", c_int32), ("My", c_int32), ("num_sub", c_int32),
                ("ovlp_cells", c_int32), ("pml_cells", c_int32), ("max_local_n", c_int32),
                ("max_band", c_int32), ("sum_local_n", c_int64), ("sum_band_n", c_int64),
                ("factor_bytes", c_int64), ("apply_bytes", c_double), ("min_pivot_ratio", c_double),
                ("factored", c_int32), ("factor_prec", c_int32), ("bad_subdomain", c_int32),
                ("last_iters", c_int32)]


class Timing(ctypes.Structure):
    _fields_ = [("factor_ms", c_double), ("solve_ms", c_double), ("apply_ms", c_double),
                ("spmv_ms", c_double), ("ortho_ms", c_double), ("applies", c_int32), ("reorths", c_int32),
                ("launches", c_int32), ("learned_dirs", c_int32), ("learned_gain", c_double)]


class TuneReport(ctypes.Structure):
    _fields_ = [("factor_threads", c_int32), ("factor_rank", c_int32), ("apply_cols", c_int32),
                ("n_factor", c_int32), ("n_apply", c_int32), ("factor_cand_threads", c_int32 * 10),
                ("factor_cand_rank", c_int32 * 10), ("factor_ms", ctypes.c_float * 10),
                ("apply_cand", c_int32 * 4), ("apply_ms", ctypes.c_float * 4), ("wide_cluster", c_int32),
                ("n_wide", c_int32), ("wide_cand", c_int32 * 4), ("wide_ms", ctypes.c_float * 4)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("nprob", c_int32), ("num_sub", c_int32), ("ntot", c_int64), ("sum_n", c_int64),
                ("sum_local_n", c_int64), ("max_band", c_int32), ("factor_prec", c_int32),
                ("factor_bytes", c_int64), ("apply_bytes", c_double), ("min_pivot_ratio", c_double),
                ("factored", c_int32), ("bad_problem", c_int32), ("bad_subdomain", c_int32),
                ("factor_threads", c_int32), ("factor_rank", c_int32), ("apply_cols", c_int32), ("steps", c_int32),
                ("cycles", c_int32),
                ("kcap", c_int32)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libraspml.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    H = c_void_p
    lib.ras_pml_setup.argtypes = [POINTER(Params), c_void_p, POINTER(c_void_p)]
    lib.ras_pml_info.argtypes = [H, POINTER(Info)]
    lib.ras_pml_num_unknowns.argtypes = [H, POINTER(c_int64)]
    lib.ras_pml_assemble_rhs.argtypes = [H, c_void_p, c_void_p, c_int, c_double, c_void_p]
    lib.ras_pml_assemble_rhs_noalloc.argtypes = [H, c_void_p, c_void_p, c_int, c_double, c_void_p]
    lib.ras_pml_factor.argtypes = [H]
    lib.ras_pml_apply.argtypes = [H, c_void_p, c_void_p]
    lib.ras_pml_matvec.argtypes = [H, c_void_p, c_void_p]
    lib.helmholtz_solve.argtypes = [H, c_void_p, c_void_p, c_double, c_int, c_int, POINTER(c_int),
                                    POINTER(c_double)]
    lib.helmholtz_solve_host.argtypes = lib.helmholtz_solve.argtypes
    lib.ras_pml_richardson.argtypes = [H, c_void_p, c_void_p, c_double, c_int, POINTER(c_int), POINTER(c_double)]
    lib.ras_pml_history.argtypes = [H, c_void_p, c_int, POINTER(c_int)]
    lib.ras_pml_set_timing.argtypes = [H, c_int]
    lib.ras_pml_set_copy_wait_limit.argtypes = [ctypes.c_longlong]
    lib.ras_pml_fma_peak.argtypes = [c_int, POINTER(c_double)]
    lib.ras_pml_get_timing.argtypes = [H, POINTER(Timing)]
    lib.ras_pml_error_string.argtypes = [c_int]
    lib.ras_pml_error_string.restype = ctypes.c_char_p
    lib.ras_pml_destroy.argtypes = [H]
    lib.ras_pml_destroy.restype = None
    lib.ras_pml_tune.argtypes = [H, POINTER(TuneReport)]
    lib.ras_pml_set_shapes.argtypes = [H, c_int, c_int, c_int, c_int]
    lib.ras_pml_batch_set_shapes.argtypes = [H, c_int, c_int, c_int, c_int]
    lib.ras_pml_batch_setup.argtypes = [POINTER(Params), c_int, c_void_p, POINTER(c_void_p)]
    lib.ras_pml_batch_info.argtypes = [H, POINTER(BatchInfo)]
    lib.ras_pml_batch_layout.argtypes = [H, c_void_p, c_void_p]
    lib.ras_pml_batch_assemble_rhs.argtypes = [H, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ras_pml_batch_factor.argtypes = [H]
    lib.ras_pml_batch_tune.argtypes = [H, POINTER(TuneReport)]
    lib.ras_pml_batch_apply.argtypes = [H, c_void_p, c_void_p]
    lib.ras_pml_batch_matvec.argtypes = [H, c_void_p, c_void_p]
    lib.ras_pml_batch_solve.argtypes = [H, c_void_p, c_void_p, c_double, c_int, c_int, c_void_p, c_void_p]
    lib.ras_pml_batch_destroy.argtypes = [H]
    lib.ras_pml_batch_destroy.restype = None
    lib.ras_pml_net_create.argtypes = [c_int, c_int, ctypes.c_uint64, c_void_p, POINTER(c_void_p)]
    lib.ras_pml_net_param_count.argtypes = [H]
    lib.ras_pml_net_set_params.argtypes = [H, c_void_p, c_int]
    lib.ras_pml_net_get_params.argtypes = [H, c_void_p, c_int]
    lib.ras_pml_net_forward.argtypes = [H, c_void_p, c_void_p, c_int]
    lib.ras_pml_net_loss_grad.argtypes = [H, c_void_p, c_void_p, c_int, POINTER(c_double), c_void_p]
    lib.ras_pml_net_adam_step.argtypes = [H, ctypes.c_float]
    lib.ras_pml_net_set_gamma.argtypes = [H, c_double]
    lib.ras_pml_net_get_gamma.argtypes = [H]
    lib.ras_pml_net_get_gamma.restype = c_double
    lib.ras_pml_net_train.argtypes = [H, H, c_int, c_void_p, c_int, c_int, ctypes.c_float, ctypes.c_uint64, c_void_p,
                                      POINTER(c_double)]
    lib.ras_pml_attach_net.argtypes = [H, H]
    lib.ras_pml_get_params.argtypes = [H, POINTER(Params)]
    lib.ras_pml_net_correct.argtypes = [H, H, c_void_p, c_void_p]
    lib.ras_pml_net_destroy.argtypes = [H]
    lib.ras_pml_net_destroy.restype = None
    for name in SYMBOLS:
        if name not in VOID_SYMBOLS:
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


class RasPmlError(RuntimeError):
    def __init__(self, fn: str, status: int):
        msg = load().ras_pml_error_string(status).decode()
        super().__init__(f"{fn} returned {status} ({ERRORS.get(status, '?')}): {msg}")
        self.status = status


def check(fn: str, status: int, allow_not_converged: bool = False) -> int:
    if status == OK or (allow_not_converged and status == NOT_CONVERGED):
        return status
    raise RasPmlError(fn, status)
