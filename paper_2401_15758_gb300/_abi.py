"""ctypes declarations of the C ABI in include/sc4dvar.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

# status codes
OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_NOT_SPD = -3
ERR_BREAKDOWN = -4
ERR_NOT_CONVERGED = -5
ERR_TIMEOUT = -6
ERR_OOM = -7
ERR_STATE = -8

MODEL_BURGERS1D = 1
MODEL_BVE2D = 2
MODEL_BURGERS1D_DIRICHLET = 3
MODEL_BVE_GYRE = 4
RK4, RK3_TVD = 0, 1
PRIOR_DIRICHLET_INV_HELMHOLTZ = 3
FP64 = 0
FP32 = 1
DF64 = 2      # double blocks, double-float sweeps (periodic Burgers Hessian products)
GEMM_3XTF32, GEMM_SIMT, GEMM_TF32, GEMM_BF16 = 0, 1, 2, 3
PRIOR_SYMBOL = 0
PRIOR_SE = 1
PRIOR_INV_HELMHOLTZ = 2
SKETCH_NONE = 0
SKETCH_RANDSVD = 1
SKETCH_NYSTROM = 2
SKETCH_SINGLEVIEW = 3
STREAM_SKETCH = 100
STREAM_KAPPA = 200
STREAM_PSI = 1000
GN_MAX_ITERS = 64


class ProblemDesc(C.Structure):
    _fields_ = [
        ("model", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("nu", C.c_double), ("dt", C.c_double), ("n_steps", C.c_int),
        ("n_obs_times", C.c_int), ("obs_steps", C.POINTER(C.c_int)),
        ("n_obs", C.c_int), ("obs_idx", C.POINTER(C.c_int)), ("sigma_obs", C.c_double),
        ("prior_kind", C.c_int), ("prior_sigma", C.c_double), ("prior_length", C.c_double),
        ("prior_symbol", C.POINTER(C.c_double)),
        ("forcing_amp", C.c_double), ("forcing_k", C.c_int), ("n_checkpoints", C.c_int),
        ("integrator", C.c_int),
    ]


class SketchOpts(C.Structure):
    _fields_ = [
        ("method", C.c_int), ("l", C.c_int), ("l2", C.c_int), ("adaptive", C.c_int),
        ("l_hat", C.c_int), ("l_max", C.c_int), ("eps_sk", C.c_double),
        ("seed", C.c_uint64), ("gn_iter", C.c_int), ("prec", C.c_int), ("gemm", C.c_int),
    ]


class PcgOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("prec", C.c_int), ("refine", C.c_int)]


class PcgInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("relres", C.c_double),
                ("status", C.c_int)]


class GnOpts(C.Structure):
    _fields_ = [("iters", C.c_int), ("gtol", C.c_double), ("sketch", SketchOpts),
                ("eps_re", C.c_double), ("pcg", PcgOpts), ("line_search", C.c_int),
                ("ls_c1", C.c_double), ("ls_c2", C.c_double), ("ls_alpha1", C.c_double),
                ("solve", C.c_int)]


class GnInfo(C.Structure):
    _fields_ = [
        ("iters_done", C.c_int),
        ("J", C.c_double * GN_MAX_ITERS), ("g_inf", C.c_double * GN_MAX_ITERS),
        ("pcg_its", C.c_int * GN_MAX_ITERS), ("relres", C.c_double * GN_MAX_ITERS),
        ("sketched", C.c_int * GN_MAX_ITERS), ("rank", C.c_int * GN_MAX_ITERS),
        ("kappa_re", C.c_double * GN_MAX_ITERS),
        ("alpha", C.c_double * GN_MAX_ITERS), ("ls_evals", C.c_int * GN_MAX_ITERS),
        ("ls_status", C.c_int * GN_MAX_ITERS),
    ]


class GnState(C.Structure):
    _fields_ = [("next_iter", C.c_int), ("g0_inf", C.c_double), ("sketch_iter", C.c_int)]


class Counters(C.Structure):
    _fields_ = [("fwd", C.c_int64), ("tlm_online", C.c_int64), ("adj_online", C.c_int64),
                ("tlm_offline", C.c_int64), ("adj_offline", C.c_int64),
                ("tlm_kappa", C.c_int64), ("adj_kappa", C.c_int64), ("qr_shifted", C.c_int64)]


P = C.c_void_p
I = C.c_int
D = C.c_double
U64 = C.c_uint64

SIGNATURES = {
    "sc4dvar_last_error": (C.c_char_p, []),
    "sc4dvar_version": (I, []),
    "sc4dvar_launch_count": (C.c_longlong, []),
    "sc4dvar_problem_create": (I, [C.POINTER(ProblemDesc), C.POINTER(P)]),
    "sc4dvar_problem_destroy": (I, [P]),
    "sc4dvar_problem_dims": (I, [P, C.POINTER(I), C.POINTER(I)]),
    "sc4dvar_set_background": (I, [P, P, P]),
    "sc4dvar_set_observations": (I, [P, P, P]),
    "sc4dvar_prior_sqrt_apply": (I, [P, P, I, I, P, I, P]),
    "sc4dvar_prior_symbol": (I, [P, P]),
    "sc4dvar_forecast": (I, [P, P, P, P, P]),
    "sc4dvar_fwd": (I, [P, P, C.POINTER(D), P, P]),
    "sc4dvar_gradient": (I, [P, P, P]),
    "sc4dvar_tlm_block": (I, [P, P, I, I, P, I, I, P]),
    "sc4dvar_adj_block": (I, [P, P, I, I, P, I, I, P]),
    "sc4dvar_gn_hessian_apply_block": (I, [P, P, I, I, P, I, I, I, P]),
    "sc4dvar_gn_hessian_apply_block_noalloc": (I, [P, P, I, I, P, I, I, I, P]),
    "sc4dvar_build_precond": (I, [P, C.POINTER(SketchOpts), P, P, C.POINTER(P), P]),
    "sc4dvar_tall_gemm": (I, [I, I, I, I, D, P, I, P, I, I, D, P, I, I, P]),
    "sc4dvar_precond_destroy": (I, [P]),
    "sc4dvar_precond_info": (I, [P, C.POINTER(I), P, P]),
    "sc4dvar_precond_apply": (I, [P, P, I, I, P, I, P]),
    "sc4dvar_kappa_estimate": (I, [P, P, U64, U64, I, C.POINTER(D), P]),
    "sc4dvar_pcg": (I, [P, P, P, P, C.POINTER(PcgOpts), C.POINTER(PcgInfo), P]),
    "sc4dvar_sketchsolv": (I, [P, P, P, P]),
    "sc4dvar_qr_update": (I, [I, I, I, I, I, P, I, P, I, P, I, P, I, P]),
    "sc4dvar_gauss_newton": (I, [P, C.POINTER(GnOpts), P, C.POINTER(GnInfo), P]),
    "sc4dvar_gauss_newton_resume": (I, [P, C.POINTER(GnOpts), P, C.POINTER(GnState), C.POINTER(P),
                                        C.POINTER(GnInfo), P]),
    "sc4dvar_precond_import": (I, [P, I, P, P, C.POINTER(P)]),
    "sc4dvar_counters": (I, [P, C.POINTER(Counters)]),
    "sc4dvar_counters_reset": (I, [P]),
    "sc4dvar_counters_set": (I, [P, C.POINTER(Counters)]),
    "sc4dvar_gaussian": (I, [U64, U64, I, I, C.c_int64, P, P]),
    "sc4dvar_batch_create": (I, [C.POINTER(P), I, C.POINTER(P)]),
    "sc4dvar_batch_destroy": (I, [P]),
    "sc4dvar_batch_hessian_apply": (I, [P, C.POINTER(P), C.POINTER(P), C.POINTER(I), I, I, P]),
    "sc4dvar_batch_pcg_start": (I, [P, C.POINTER(P), C.POINTER(P), D, I, P]),
    "sc4dvar_batch_pcg_step": (I, [P, I, P]),
    "sc4dvar_batch_pcg_status": (I, [P, C.POINTER(D), C.POINTER(I), C.POINTER(I), P]),
    "sc4dvar_batch_pcg_solution": (I, [P, C.POINTER(P), P]),
    "sc4dvar_autotune": (I, [P, I, C.POINTER(I)]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsc4dvar.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libsc4dvar.so not found at {path}; run paper_2401_15758_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class Sc4dvarError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sc4dvar error {code}: {msg}")
        self.code = code


def check(code: int):
    if code != OK:
        msg = _lib.sc4dvar_last_error().decode(errors="replace") if _lib else ""
        raise Sc4dvarError(code, msg)
    return code
