"""ctypes binding of libcoxgb.so: the C ABI in include/coxgb.h and include/nmfgb.h, same names.

Argument marshalling only; every step of the iteration runs in the CUDA
library.  Loading fails loudly when the library has not been built."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcoxgb.so")

COX_OK = 0
COX_ERR_ARG = -1
COX_ERR_CODE3 = -2
COX_ERR_OOM = -3
COX_ERR_CUDA = -4
COX_ERR_TIMEOUT = -5
COX_ERR_NONFINITE = -6
COX_ERR_NOT_CONVERGED = -7
COX_ERR_STATE = -8
COX_ERR_UNSUPPORTED = -9

COX_X_INT8_HOST = 0
COX_X_F64_HOST = 1
COX_X_PACKED2_HOST = 2
COX_X_PACKED2_DEV = 3

COX_SPLIT_E4M3 = 0
COX_FP64 = 1
COX_FP32_GEMV = 2
COX_SPLIT_E2M1 = 3

# every symbol include/coxgb.h declares
EXPORTS = [
    "cox_default_options", "cox_setup", "cox_destroy", "cox_lipschitz", "cox_lambda_max",
    "cox_loss_grad", "cox_prox_step", "cox_prox_step_host", "cox_sync", "cox_last_objective",
    "cox_path_fit", "cox_get_state", "cox_set_state", "cox_get_info", "cox_get_mu_order",
    "cox_strerror", "cox_set_precision", "cox_profile", "cox_profile_read", "cox_lipschitz_noalloc",
    "cox_autotune", "cox_eta", "cox_plan_shape", "cox_rank_by_entry", "cox_path_seq", "cox_set_covariates",
    "cox_get_gamma", "cox_set_gamma", "cox_grad_gamma", "cox_prox_step_eta", "cox_last_loss_l1",
    "cox_set_active_set", "cox_plan_shape_prec",
]
# every symbol include/nmfgb.h declares
NMF_EXPORTS = [
    "nmf_setup", "nmf_destroy", "nmf_set_factors", "nmf_get_factors", "nmf_iterate", "nmf_objective",
    "nmf_sync", "nmf_get_info", "nmf_time_products",
]
NMF_MAX_RANK = 80
NMF_MULTIPLICATIVE = 0
NMF_APG = 1
COX_MAX_COVARIATES = 16


class cox_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("center", ctypes.c_int), ("device", ctypes.c_int),
                ("tile_m", ctypes.c_int), ("stages", ctypes.c_int), ("lag", ctypes.c_int),
                ("wait_limit_s", ctypes.c_double), ("chunks", ctypes.c_int), ("window", ctypes.c_int),
                ("issue", ctypes.c_int), ("active_set", ctypes.c_int)]


class cox_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int64), ("n_pad", ctypes.c_int64),
                ("p_pad", ctypes.c_int64), ("precision", ctypes.c_int), ("center", ctypes.c_int),
                ("tile_m", ctypes.c_int), ("stages", ctypes.c_int), ("sm_count", ctypes.c_int),
                ("device_bytes", ctypes.c_int64), ("n_tie_groups", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("chunks", ctypes.c_int), ("ring", ctypes.c_int),
                ("issue", ctypes.c_int), ("issue_xtv", ctypes.c_int), ("active_cols", ctypes.c_int64),
                ("active_rebuilds", ctypes.c_int64)]


class cox_tune_choice(ctypes.Structure):
    _fields_ = [("tile_m", ctypes.c_int), ("chunks", ctypes.c_int), ("stages", ctypes.c_int),
                ("candidates", ctypes.c_int), ("ms", ctypes.c_double), ("issue", ctypes.c_int)]


class cox_plan(ctypes.Structure):
    _fields_ = [("tile_m", ctypes.c_int), ("chunks", ctypes.c_int), ("stages", ctypes.c_int),
                ("ring", ctypes.c_int), ("decoder_groups", ctypes.c_int), ("named_barriers", ctypes.c_int),
                ("limb_cols", ctypes.c_int), ("tmem_cols", ctypes.c_int), ("smem_bytes", ctypes.c_longlong),
                ("issue", ctypes.c_int), ("issuers", ctypes.c_int), ("mmas_per_commit", ctypes.c_int),
                ("limb_stages", ctypes.c_int)]


class nmf_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("r", ctypes.c_int), ("limb_cols", ctypes.c_int),
                ("stages", ctypes.c_int), ("sm_count", ctypes.c_int), ("grid_xwt", ctypes.c_int),
                ("grid_vtx", ctypes.c_int), ("units_xwt", ctypes.c_int64), ("units_vtx", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("launches", ctypes.c_int64)]


class CoxError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


_lib = None


def load(path: str | None = None):
    """Load libcoxgb.so (built by ``paper_2010_16114_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libcoxgb.so is not built ({path}); run paper_2010_16114_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.cox_default_options.restype = None
    lib.cox_default_options.argtypes = [ctypes.POINTER(cox_options)]
    lib.cox_setup.restype = I
    lib.cox_setup.argtypes = [ctypes.POINTER(P), P, I64, I64, I, P, P, ctypes.POINTER(cox_options)]
    lib.cox_destroy.restype = None
    lib.cox_destroy.argtypes = [P]
    lib.cox_lipschitz.restype = I
    lib.cox_lipschitz.argtypes = [P, P, D, I, ctypes.POINTER(D)]
    lib.cox_lipschitz_noalloc.restype = I
    lib.cox_lipschitz_noalloc.argtypes = [P, P, D, I, ctypes.POINTER(D)]
    lib.cox_lambda_max.restype = I
    lib.cox_lambda_max.argtypes = [P, ctypes.POINTER(D)]
    lib.cox_loss_grad.restype = I
    lib.cox_loss_grad.argtypes = [P, P, I, P, P, P]
    lib.cox_prox_step.restype = I
    lib.cox_prox_step.argtypes = [P, P, P, I, D, P]
    lib.cox_prox_step_host.restype = I
    lib.cox_prox_step_host.argtypes = [P, P, P, I, D, P]
    lib.cox_sync.restype = I
    lib.cox_sync.argtypes = [P, P]
    lib.cox_last_objective.restype = I
    lib.cox_last_objective.argtypes = [P, P, I, P]
    lib.cox_path_fit.restype = I
    lib.cox_path_fit.argtypes = [P, P, I, I, D, D, I, P, P, P, P]
    lib.cox_get_state.restype = I
    lib.cox_get_state.argtypes = [P, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.cox_set_state.restype = I
    lib.cox_set_state.argtypes = [P, P, ctypes.c_size_t]
    lib.cox_get_info.restype = I
    lib.cox_get_info.argtypes = [P, ctypes.POINTER(cox_info)]
    lib.cox_get_mu_order.restype = I
    lib.cox_get_mu_order.argtypes = [P, P, P]
    lib.cox_set_precision.restype = I
    lib.cox_set_precision.argtypes = [P, I]
    lib.cox_profile.restype = I
    lib.cox_profile.argtypes = [P, I]
    lib.cox_profile_read.restype = I
    lib.cox_profile_read.argtypes = [P, P, P]
    lib.cox_eta.restype = I
    lib.cox_eta.argtypes = [P, P, I, P, P]
    lib.cox_autotune.restype = I
    lib.cox_autotune.argtypes = [P, I, I, ctypes.POINTER(cox_tune_choice), ctypes.POINTER(cox_tune_choice)]
    lib.cox_plan_shape.restype = I
    lib.cox_plan_shape.argtypes = [I, I, I, I, I, ctypes.POINTER(cox_plan)]
    lib.cox_plan_shape_prec.restype = I
    lib.cox_plan_shape_prec.argtypes = [I, I, I, I, I, I, ctypes.POINTER(cox_plan)]
    lib.cox_rank_by_entry.restype = I
    lib.cox_rank_by_entry.argtypes = [I64, I, P, P, I, P, P, ctypes.POINTER(I64)]
    lib.cox_path_seq.restype = I
    lib.cox_path_seq.argtypes = [P, P, I, I, D, D, I, P, P, P, P, P]
    lib.cox_set_active_set.restype = I
    lib.cox_set_active_set.argtypes = [P, I]
    lib.cox_prox_step_eta.restype = I
    lib.cox_prox_step_eta.argtypes = [P, P, P, P, I, D, P]
    lib.cox_last_loss_l1.restype = I
    lib.cox_last_loss_l1.argtypes = [P, P, P, I, P]
    lib.cox_set_covariates.restype = I
    lib.cox_set_covariates.argtypes = [P, P, I]
    for nm in ("cox_get_gamma", "cox_set_gamma", "cox_grad_gamma"):
        getattr(lib, nm).restype = I
        getattr(lib, nm).argtypes = [P, P, I]
    lib.nmf_setup.restype = I
    lib.nmf_setup.argtypes = [P, I64, I64, I, I, ctypes.POINTER(P)]
    lib.nmf_destroy.restype = I
    lib.nmf_destroy.argtypes = [P]
    lib.nmf_set_factors.restype = I
    lib.nmf_set_factors.argtypes = [P, P, P, P]
    lib.nmf_get_factors.restype = I
    lib.nmf_get_factors.argtypes = [P, P, P, P]
    lib.nmf_iterate.restype = I
    lib.nmf_iterate.argtypes = [P, I, I64, D, P]
    lib.nmf_objective.restype = I
    lib.nmf_objective.argtypes = [P, ctypes.POINTER(D), P]
    lib.nmf_sync.restype = I
    lib.nmf_sync.argtypes = [P, P]
    lib.nmf_get_info.restype = I
    lib.nmf_get_info.argtypes = [P, ctypes.POINTER(nmf_info)]
    lib.nmf_time_products.restype = I
    lib.nmf_time_products.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(D), P]
    lib.cox_strerror.restype = ctypes.c_char_p
    lib.cox_strerror.argtypes = [I]
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().cox_strerror(code).decode()
    except ImportError:
        return f"error {code}"


def check(code: int, where: str, allow=(COX_OK,)) -> int:
    if code not in allow:
        raise CoxError(code, where)
    return code


# thin same-name wrappers -------------------------------------------------------------

def cox_default_options() -> cox_options:
    o = cox_options()
    load().cox_default_options(ctypes.byref(o))
    return o


def cox_setup(X_ptr, n, p, x_format, time_ptr, event_ptr, opt: cox_options | None):
    h = ctypes.c_void_p()
    rc = load().cox_setup(ctypes.byref(h), X_ptr, n, p, x_format, time_ptr, event_ptr,
                          ctypes.byref(opt) if opt is not None else None)
    return rc, h


def cox_destroy(h):
    load().cox_destroy(h)


def cox_lipschitz(h, start_ptr=None, tol=0.0, maxiter=0):
    L = ctypes.c_double()
    rc = load().cox_lipschitz(h, start_ptr, tol, maxiter, ctypes.byref(L))
    return rc, L.value


def cox_lipschitz_noalloc(h, start_ptr=None, tol=0.0, maxiter=0):
    L = ctypes.c_double()
    rc = load().cox_lipschitz_noalloc(h, start_ptr, tol, maxiter, ctypes.byref(L))
    return rc, L.value


def cox_lambda_max(h):
    v = ctypes.c_double()
    rc = load().cox_lambda_max(h, ctypes.byref(v))
    return rc, v.value


def cox_loss_grad(h, beta_ptr, k, loss_ptr, grad_ptr, stream_ptr):
    return load().cox_loss_grad(h, beta_ptr, k, loss_ptr, grad_ptr, stream_ptr)


def cox_prox_step(h, beta_ptr, lam_ptr, k, step, stream_ptr):
    return load().cox_prox_step(h, beta_ptr, lam_ptr, k, step, stream_ptr)


def cox_prox_step_host(h, beta_ptr, lam_ptr, k, step, stream_ptr):
    return load().cox_prox_step_host(h, beta_ptr, lam_ptr, k, step, stream_ptr)


def cox_sync(h, stream_ptr):
    return load().cox_sync(h, stream_ptr)


def cox_last_objective(h, obj_ptr, k, stream_ptr):
    return load().cox_last_objective(h, obj_ptr, k, stream_ptr)


def cox_path_fit(h, lam_ptr, k, max_iter, tol, step, warm, beta_ptr, iters_ptr, obj_ptr, stream_ptr):
    return load().cox_path_fit(h, lam_ptr, k, max_iter, tol, step, warm, beta_ptr, iters_ptr, obj_ptr,
                               stream_ptr)


def cox_get_state(h, buf_ptr, size_ref):
    return load().cox_get_state(h, buf_ptr, size_ref)


def cox_set_state(h, buf_ptr, size):
    return load().cox_set_state(h, buf_ptr, size)


def cox_get_info(h):
    info = cox_info()
    rc = load().cox_get_info(h, ctypes.byref(info))
    return rc, info


def cox_get_mu_order(h, mu_ptr, order_ptr):
    return load().cox_get_mu_order(h, mu_ptr, order_ptr)


def cox_set_precision(h, precision: int) -> int:
    return load().cox_set_precision(h, precision)


def cox_profile(h, enable: int) -> int:
    return load().cox_profile(h, enable)


def cox_profile_read(h, ms_ptr, launches_ptr) -> int:
    return load().cox_profile_read(h, ms_ptr, launches_ptr)


def cox_eta(h, beta_ptr, k: int, eta_ptr, stream) -> int:
    return load().cox_eta(h, beta_ptr, k, eta_ptr, stream)


def cox_autotune(h, k: int, reps: int):
    xb, xtv = cox_tune_choice(), cox_tune_choice()
    rc = load().cox_autotune(h, k, reps, ctypes.byref(xb), ctypes.byref(xtv))
    return rc, xb, xtv


def cox_plan_shape(k: int, tile_m: int = 0, chunks: int = 0, stages: int = 0, issue: int = 0):
    """(rc, cox_plan) of the tensor-core products for k columns; host only."""
    out = cox_plan()
    rc = load().cox_plan_shape(k, tile_m, chunks, stages, issue, ctypes.byref(out))
    return rc, out


def cox_plan_shape_prec(precision: int, k: int, tile_m: int = 0, chunks: int = 0, stages: int = 0,
                        issue: int = 0):
    """(rc, cox_plan) of either operand form of the tensor-core products; host only."""
    out = cox_plan()
    rc = load().cox_plan_shape_prec(precision, k, tile_m, chunks, stages, issue, ctypes.byref(out))
    return rc, out


def cox_strerror(code: int) -> str:
    return strerror(code)


def cox_path_seq(h, lam_ptr, L, max_iter, tol, step, warm, B_ptr, G_ptr, iters_ptr, obj_ptr, stream_ptr):
    return load().cox_path_seq(h, lam_ptr, L, max_iter, tol, step, warm, B_ptr, G_ptr, iters_ptr, obj_ptr,
                               stream_ptr)


def cox_set_covariates(h, Z_ptr, q: int) -> int:
    return load().cox_set_covariates(h, Z_ptr, q)


def cox_get_gamma(h, out_ptr, k: int) -> int:
    return load().cox_get_gamma(h, out_ptr, k)


def cox_set_gamma(h, in_ptr, k: int) -> int:
    return load().cox_set_gamma(h, in_ptr, k)


def cox_grad_gamma(h, out_ptr, k: int) -> int:
    return load().cox_grad_gamma(h, out_ptr, k)


def cox_prox_step_eta(h, beta_ptr, eta_ptr, lam_ptr, k, step, stream_ptr):
    return load().cox_prox_step_eta(h, beta_ptr, eta_ptr, lam_ptr, k, step, stream_ptr)


def cox_last_loss_l1(h, f_ptr, l1_ptr, k, stream_ptr):
    return load().cox_last_loss_l1(h, f_ptr, l1_ptr, k, stream_ptr)


def cox_set_active_set(h, on: int) -> int:
    return load().cox_set_active_set(h, on)


def nmf_setup(X_ptr, m: int, n: int, r: int, device: int, out_ptr) -> int:
    return load().nmf_setup(X_ptr, m, n, r, device, out_ptr)


def nmf_destroy(h) -> int:
    return load().nmf_destroy(h)


def nmf_set_factors(h, V_ptr, W_ptr, stream_ptr) -> int:
    return load().nmf_set_factors(h, V_ptr, W_ptr, stream_ptr)


def nmf_get_factors(h, V_ptr, W_ptr, stream_ptr) -> int:
    return load().nmf_get_factors(h, V_ptr, W_ptr, stream_ptr)


def nmf_iterate(h, algo: int, iters: int, eps: float, stream_ptr) -> int:
    return load().nmf_iterate(h, algo, iters, eps, stream_ptr)


def nmf_objective(h, f_ptr, stream_ptr) -> int:
    return load().nmf_objective(h, f_ptr, stream_ptr)


def nmf_sync(h, stream_ptr) -> int:
    return load().nmf_sync(h, stream_ptr)


def nmf_get_info(h, info_ptr) -> int:
    return load().nmf_get_info(h, info_ptr)


def nmf_time_products(h, reps: int, a_ptr, b_ptr, stream_ptr) -> int:
    return load().nmf_time_products(h, reps, a_ptr, b_ptr, stream_ptr)
