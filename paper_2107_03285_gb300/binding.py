"""ctypes binding of libsgn (include/sgn.h): argument marshalling only.

Every step of the SGN path runs in the library's CUDA kernels; this module
allocates the caller-owned device buffer with PyTorch, passes raw pointers
and the current CUDA stream, and raises on non-OK status.  There is no CPU
fallback: if libsgn.so is missing or cannot load, importing it fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsgn.so")

# status codes (sgn_status)
OK, EINVAL, ECUDA, ENOMEM, EINVERTED, ENEWTON, EPIVOT, EREFINE, ESTATE, ENONFINITE, ETIMEOUT = range(11)
FP64, MIXED = 0, 1
SOLVE_AUTO, SOLVE_REFINE, SOLVE_BICGSTAB = 0, 1, 2
RHS_KKT, RHS_PAPER = 0, 1
STORE_FP64, STORE_MIXED, STORE_KFACT, STORE_KFACT_MIXED = 1, 2, 4, 8
BATCH_EQUILIBRIUM, BATCH_KKT = 0, 1
PROF_KINDS = ["update", "panel_update", "pivot", "trsm", "front_assembly", "elements", "solve", "vector"]

EXPORTED = ["sgn_setup", "sgn_get_info", "sgn_device_bytes", "sgn_bind", "sgn_set_stream",
            "sgn_set_objective", "sgn_destroy", "sgn_strerror", "sgn_assemble", "sgn_factor",
            "sgn_solve", "sgn_step_host", "sgn_equilibrium", "sgn_gradient", "sgn_factor_k",
            "sgn_export_kkt", "sgn_profile", "sgn_profile_read", "sgn_launch_count", "sgn_assemble_static", "sgn_step_graph",
            "sgn_last_error", "sgn_selftest_wait_timeout", "sgn_batch_setup", "sgn_batch_info", "sgn_batch_residuals",
            "sgn_factor_ex", "sgn_objective_value", "sgn_lbfgs_direction", "sgn_lbfgs_work_bytes",
            "sgn_optimize_lbfgs", "sgn_factor_inertia",
            # learned warm start (include/sgn_learn.h)
            "sgn_learn_create", "sgn_learn_device_bytes", "sgn_learn_bind", "sgn_learn_destroy",
            "sgn_rbf_params", "sgn_learn_basis", "sgn_learn_train", "sgn_learn_predict",
            "sgn_equilibrium_warm", "sgn_learn_param_count", "sgn_learn_params", "sgn_learn_grads",
            "sgn_learn_apply", "sgn_learn_basis_get"]


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_nodes", C.c_int32), ("n_elem", C.c_int32),
                ("X_h", C.POINTER(C.c_double)), ("conn_h", C.POINTER(C.c_int32)),
                ("fixed_h", C.POINTER(C.c_uint8)), ("E0", C.c_double), ("nu", C.c_double)]


class SetupOpts(C.Structure):
    _fields_ = [("leaf_nodes", C.c_int32), ("panel", C.c_int32), ("update_ctas", C.c_int32)]


class Objective(C.Structure):
    _fields_ = [("n_track", C.c_int32), ("track_dof_h", C.POINTER(C.c_int64)),
                ("target_h", C.POINTER(C.c_double)), ("weight_h", C.POINTER(C.c_double)),
                ("alpha", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_free", C.c_int64), ("n_elem", C.c_int64),
                ("n_x", C.c_int64), ("n_p", C.c_int64), ("n_kkt", C.c_int64), ("nnz_kkt", C.c_int64),
                ("n_supernodes", C.c_int64), ("n_levels", C.c_int64), ("max_front", C.c_int64),
                ("nnz_factor", C.c_int64), ("factor_flops", C.c_double), ("kfactor_flops", C.c_double),
                ("setup_seconds", C.c_double)]


class FactorReport(C.Structure):
    _fields_ = [("n_pos", C.c_int64), ("n_neg", C.c_int64), ("n_zero", C.c_int64),
                ("n_2x2", C.c_int64), ("n_perturbed", C.c_int64), ("seconds", C.c_double),
                ("tensor_core_updates", C.c_int64)]


class SolveOpts(C.Structure):
    _fields_ = [("max_refine", C.c_int32), ("tol", C.c_double), ("method", C.c_int32), ("max_krylov", C.c_int32),
                ("regularized", C.c_int32)]


class InertiaOpts(C.Structure):
    _fields_ = [("delta0", C.c_double), ("growth", C.c_double), ("max_tries", C.c_int32)]


class SolveReport(C.Structure):
    _fields_ = [("refine_steps", C.c_int32), ("residual", C.c_double), ("seconds", C.c_double),
                ("history", C.c_double * 32), ("krylov_iters", C.c_int32)]


class FactorOpts(C.Structure):
    _fields_ = [("eps_x", C.c_double), ("eps_lambda", C.c_double)]


class LbfgsOpts(C.Structure):
    _fields_ = [("m", C.c_int32), ("max_iter", C.c_int32), ("tol_g", C.c_double), ("precision", C.c_int32),
                ("eq_precision", C.c_int32), ("armijo", C.c_double), ("max_halvings", C.c_int32)]


class LbfgsReport(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("restarts", C.c_int32), ("trials", C.c_int32),
                ("equilibrium_iters", C.c_int32), ("seconds", C.c_double), ("f", C.c_double * 64),
                ("gnorm", C.c_double * 64), ("step", C.c_double * 64)]


class KernelProfile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("seconds", C.c_double), ("flops", C.c_double)]


class NewtonOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("tol", C.c_double), ("precision", C.c_int32)]


class NewtonReport(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("residual", C.c_double),
                ("initial_residual", C.c_double), ("seconds", C.c_double), ("solves", C.c_int32),
                ("history", C.c_double * 32), ("step_length", C.c_double * 32)]


class LearnOpts(C.Structure):
    _fields_ = [("n_rbf", C.c_int32), ("centers_h", C.POINTER(C.c_double)), ("width", C.c_double),
                ("n_modes", C.c_int32), ("hidden", C.c_int32), ("max_snap", C.c_int32), ("batch", C.c_int32)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libsgn.so not built ({path}); run `python -m paper_2107_03285_gb300.build`")
    lib = C.CDLL(path)
    P, VP = C.POINTER, C.c_void_p
    dp = P(C.c_double)
    sig = {
        "sgn_setup": (C.c_int, [P(Mesh), P(SetupOpts), P(VP)]),
        "sgn_get_info": (C.c_int, [VP, P(Info)]),
        "sgn_device_bytes": (C.c_int, [VP, C.c_int32, P(C.c_size_t)]),
        "sgn_bind": (C.c_int, [VP, VP, C.c_size_t, C.c_int32, VP]),
        "sgn_set_stream": (C.c_int, [VP, VP]),
        "sgn_set_objective": (C.c_int, [VP, P(Objective)]),
        "sgn_destroy": (None, [VP]),
        "sgn_strerror": (C.c_char_p, [C.c_int]),
        "sgn_assemble": (C.c_int, [VP, VP, VP]),
        "sgn_assemble_static": (C.c_int, [VP, VP, VP]),
        "sgn_step_graph": (C.c_int, [VP, C.c_int, C.c_int32, VP, VP, VP, VP, VP, dp]),
        "sgn_factor": (C.c_int, [VP, C.c_int, P(FactorReport)]),
        "sgn_factor_ex": (C.c_int, [VP, C.c_int, P(FactorOpts), P(FactorReport)]),
        "sgn_objective_value": (C.c_int, [VP, VP, VP, dp]),
        "sgn_factor_inertia": (C.c_int, [VP, C.c_int, P(InertiaOpts), dp, P(FactorReport)]),
        "sgn_lbfgs_direction": (C.c_int, [VP, C.c_int32, VP, VP, VP, VP]),
        "sgn_lbfgs_work_bytes": (C.c_int, [VP, C.c_int32, P(C.c_size_t)]),
        "sgn_optimize_lbfgs": (C.c_int, [VP, VP, VP, VP, VP, C.c_size_t, P(LbfgsOpts), P(LbfgsReport)]),
        "sgn_solve": (C.c_int, [VP, C.c_int, VP, VP, VP, VP, P(SolveOpts), P(SolveReport)]),
        "sgn_step_host": (C.c_int, [VP, C.c_int, dp, dp, dp, dp, dp, P(SolveReport)]),
        "sgn_equilibrium": (C.c_int, [VP, VP, VP, VP, P(NewtonOpts), P(NewtonReport)]),
        "sgn_gradient": (C.c_int, [VP, VP]),
        "sgn_factor_k": (C.c_int, [VP]),
        "sgn_export_kkt": (C.c_int, [VP, P(C.c_int64), P(C.c_int64), P(C.c_int64), dp]),
        "sgn_profile": (C.c_int, [VP, C.c_int32]),
        "sgn_profile_read": (C.c_int, [VP, P(KernelProfile), C.c_int32]),
        "sgn_launch_count": (C.c_int64, [VP]),
        "sgn_last_error": (C.c_char_p, [VP]),
        "sgn_selftest_wait_timeout": (C.c_int, [VP]),
        "sgn_batch_setup": (C.c_int, [C.c_int32, P(Mesh), P(Objective), P(SetupOpts), P(VP)]),
        "sgn_batch_info": (C.c_int, [VP, P(C.c_int32), P(C.c_int64), P(C.c_int64)]),
        "sgn_batch_residuals": (C.c_int, [VP, C.c_int32, dp]),
        "sgn_learn_create": (C.c_int, [VP, P(LearnOpts), P(VP)]),
        "sgn_learn_device_bytes": (C.c_int, [VP, P(C.c_size_t)]),
        "sgn_learn_bind": (C.c_int, [VP, VP, C.c_size_t]),
        "sgn_learn_destroy": (None, [VP]),
        "sgn_rbf_params": (C.c_int, [VP, VP, VP]),
        "sgn_learn_basis": (C.c_int, [VP, VP, C.c_int32, C.c_uint64, dp]),
        "sgn_learn_train": (C.c_int, [VP, VP, VP, C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_uint64,
                                      P(C.c_float)]),
        "sgn_learn_predict": (C.c_int, [VP, VP, VP]),
        "sgn_equilibrium_warm": (C.c_int, [VP, VP, VP, VP, VP, P(NewtonOpts), P(NewtonReport),
                                           P(C.c_int32)]),
        "sgn_learn_param_count": (C.c_int64, [VP]),
        "sgn_learn_params": (C.c_int, [VP, P(C.c_float), C.c_int32]),
        "sgn_learn_grads": (C.c_int, [VP, P(C.c_float), P(C.c_float), C.c_int32, P(C.c_float),
                                      P(C.c_float)]),
        "sgn_learn_apply": (C.c_int, [VP, P(C.c_float), C.c_float, C.c_float]),
        "sgn_learn_basis_get": (C.c_int, [VP, dp, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class SGNError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__(f"{where}: status {code} ({msg})")
        self.code = code


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _check(code, where, h=None):
    if code != OK:
        msg = lib().sgn_strerror(code).decode()
        if h is not None:
            detail = lib().sgn_last_error(h).decode()
            if detail and detail != msg:
                msg = f"{msg}; {detail}"
        raise SGNError(code, where, msg)
    return code


def _dptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))
