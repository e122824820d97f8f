"""Python front end of libcoxgb: one handle per data set.

Coefficients are torch tensors of shape (k, p) on the handle's CUDA device
(row c = penalty c), which is the library's p x k column-major layout.
float32 for the genotype modes, float64 for precision "fp64".
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

PRECISIONS = {"split_e4m3": L.COX_SPLIT_E4M3, "fp64": L.COX_FP64, "fp32_gemv": L.COX_FP32_GEMV,
              "split_e2m1": L.COX_SPLIT_E2M1}


def _vp(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(x))


def _stream_ptr(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def plan_shape(k: int, tile_m: int = 0, chunks: int = 0, stages: int = 0, issue: int = 0,
               precision: str = "split_e4m3") -> dict:
    """The tensor-core products' pipeline plan for k columns (cox_plan_shape_prec):
    shape, issue mode, shared-memory depth, TMEM slots, barriers and memory, for
    the e4m3 or the e2m1 operand form.  Host only; raises CoxError for a shape or
    depth the pipeline does not allow."""
    rc, p = L.cox_plan_shape_prec(PRECISIONS[precision], int(k), int(tile_m), int(chunks), int(stages),
                                  int(issue))
    L.check(rc, "cox_plan_shape_prec")
    return {f: getattr(p, f) for f, _ in L.cox_plan._fields_}


def rank_by_entry(lambdas, beta):
    """Section 6 SNP ranking (cox_rank_by_entry, host): SNPs with a nonzero
    coefficient on the path ordered by the largest lambda at which they are
    nonzero, ties by |beta| there, then by index.  beta: (k, p) coefficients
    (row c at lambdas[c]), a tensor (any device) or an array, float32 or
    float64.  Returns (order, entry): entry[j] = index of SNP j's entry lambda
    or -1."""
    if isinstance(beta, torch.Tensor):
        beta = beta.detach().cpu().numpy()
    B = np.ascontiguousarray(beta)
    if B.dtype not in (np.float32, np.float64):
        B = B.astype(np.float64)
    if B.ndim == 1:
        B = B[None]
    k, p = B.shape
    lams = np.ascontiguousarray(np.atleast_1d(np.asarray(lambdas, dtype=np.float64)))
    if len(lams) != k:
        raise ValueError(f"{len(lams)} lambdas for {k} coefficient rows")
    order = np.zeros(p, np.int64)
    entry = np.zeros(p, np.int64)
    cnt = ctypes.c_int64()
    L.check(L.load().cox_rank_by_entry(p, k, _vp(lams), _vp(B), int(B.dtype == np.float64), _vp(order),
                                       _vp(entry), ctypes.byref(cnt)), "cox_rank_by_entry")
    return order[:cnt.value], entry


class CoxProblem:
    """A data set (X, y, delta) laid out on the GPU (``cox_setup``).

    X may be
      * a numpy uint8 (n, p) array of genotype codes {0,1,2};
      * a numpy float64 (n, p) array (precision "fp64");
      * a uint8 array/tensor of row-major 2-bit codes, shape (n, ceil(p/4)),
        on the host or on the device, with ``p`` given."""

    def __init__(self, X, time, event, precision: str = "split_e4m3", center: bool | None = None,
                 p: int | None = None, device: int | None = None, tile_m: int = 0, stages: int = 0,
                 lag: int = 10, wait_limit_s: float = 2.0, chunks: int = 0, window: int = 0, issue: int = 0,
                 active_set: bool = False):
        lib = L.load()
        opt = L.cox_default_options()
        opt.precision = PRECISIONS[precision]
        opt.center = int(center if center is not None else precision != "fp64")
        opt.device = -1 if device is None else int(device)
        opt.tile_m = int(tile_m)
        opt.stages = int(stages)
        opt.chunks = int(chunks)
        opt.window = int(window)
        opt.issue = int(issue)
        opt.active_set = int(bool(active_set))
        opt.lag = int(lag)
        opt.wait_limit_s = float(wait_limit_s)
        time = np.ascontiguousarray(time, dtype=np.float64)
        event = np.ascontiguousarray(event, dtype=np.uint8)
        n = len(time)
        self._keep = None
        if isinstance(X, torch.Tensor) and X.is_cuda:
            assert X.dtype == torch.uint8 and p is not None
            fmt, xp = L.COX_X_PACKED2_DEV, _vp(X.contiguous())
            self._keep = X
        elif isinstance(X, np.ndarray) and X.dtype == np.float64:
            fmt, p = L.COX_X_F64_HOST, X.shape[1]
            X = np.ascontiguousarray(X)
            xp = _vp(X)
        elif p is not None and X.shape[1] == (p + 3) // 4 and X.dtype == np.uint8 and X.shape[1] != p:
            X = np.ascontiguousarray(X)
            fmt, xp = L.COX_X_PACKED2_HOST, _vp(X)
        else:
            X = np.ascontiguousarray(X, dtype=np.uint8)
            fmt, p = L.COX_X_INT8_HOST, X.shape[1]
            xp = _vp(X)
        rc, h = L.cox_setup(xp, n, p, fmt, _vp(time), _vp(event), opt)
        L.check(rc, "cox_setup")
        self.h = h
        self.n, self.p = n, p
        self.q = 0
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        dev = torch.cuda.current_device() if device is None else device
        self.device = torch.device("cuda", dev)
        self._lib = lib

    # -- life cycle -------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            L.cox_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- queries ------------------------------------------------------------------------
    def info(self):
        rc, info = L.cox_get_info(self.h)
        L.check(rc, "cox_get_info")
        return {f: getattr(info, f) for f, _ in L.cox_info._fields_}

    def mu_order(self):
        mu = np.zeros(self.p)
        order = np.zeros(self.n, np.int64)
        L.check(L.cox_get_mu_order(self.h, _vp(mu), _vp(order)), "cox_get_mu_order")
        return mu, order

    def set_active_set(self, on: bool):
        """Stream only the SNP columns with a nonzero coefficient in X B (cox_set_active_set)."""
        L.check(L.cox_set_active_set(self.h, int(bool(on))), "cox_set_active_set")

    def set_precision(self, precision: str):
        """Switch between "split_e4m3" and "fp32_gemv" on the same resident data."""
        L.check(L.cox_set_precision(self.h, PRECISIONS[precision]), "cox_set_precision")
        self.precision = precision

    def autotune(self, k: int, reps: int = 3):
        """Time every compiled pipeline shape of both products for k columns and
        keep the fastest (cox_autotune); returns the choices."""
        rc, xb, xtv = L.cox_autotune(self.h, int(k), int(reps))
        L.check(rc, "cox_autotune")
        f = [n for n, _ in L.cox_tune_choice._fields_]
        return {"x_b": {n: getattr(xb, n) for n in f}, "xt_v": {n: getattr(xtv, n) for n in f}}

    def profile(self, enable: bool):
        L.check(L.cox_profile(self.h, int(enable)), "cox_profile")

    def profile_read(self):
        """(total ms, launches) per kernel class: X B, X^T V (+step), scans, other."""
        ms = np.zeros(4)
        n = np.zeros(4, np.int64)
        L.check(L.cox_profile_read(self.h, _vp(ms), _vp(n)), "cox_profile_read")
        return ms, n

    def lipschitz(self, start: np.ndarray | None = None, tol: float = 0.0, maxiter: int = 0) -> float:
        """L = 2 ||X_c||_2^2 / n by the power method (defaults: tol 1e-6, 1000 iterations)."""
        s = None if start is None else np.ascontiguousarray(start, dtype=np.float64)
        rc, v = L.cox_lipschitz(self.h, _vp(s), float(tol), int(maxiter))
        L.check(rc, "cox_lipschitz")
        return v

    def lambda_max(self) -> float:
        rc, v = L.cox_lambda_max(self.h)
        L.check(rc, "cox_lambda_max")
        return v

    def zeros(self, k: int) -> torch.Tensor:
        return torch.zeros((k, self.p), dtype=self.dtype, device=self.device)

    def _beta(self, beta: torch.Tensor) -> torch.Tensor:
        if beta.dim() == 1:
            beta = beta[None]
        if beta.dtype != self.dtype or not beta.is_cuda or beta.shape[1] != self.p or not beta.is_contiguous():
            raise ValueError(f"beta must be a contiguous {self.dtype} CUDA tensor of shape (k, {self.p})")
        return beta

    # -- the iteration ---------------------------------------------------------------------
    def loss_grad(self, beta: torch.Tensor, stream=None):
        """f(beta_c) per row and grad f (same shape as beta)."""
        b = self._beta(beta)
        k = b.shape[0]
        loss = np.zeros(k)
        grad = torch.empty_like(b)
        rc = L.cox_loss_grad(self.h, _vp(b), k, _vp(loss), _vp(grad), _stream_ptr(stream))
        L.check(rc, "cox_loss_grad")
        return loss, grad.view_as(beta)

    def eta(self, beta: torch.Tensor, stream=None) -> torch.Tensor:
        """eta = X_c beta, shape (k, n), subjects in the handle's sorted order."""
        b = self._beta(beta)
        k = b.shape[0]
        out = torch.empty((k, self.n), dtype=torch.float64, device=b.device)
        L.check(L.cox_eta(self.h, _vp(b), k, _vp(out), _stream_ptr(stream)), "cox_eta")
        return out

    def prox_step(self, beta: torch.Tensor, lambdas, step: float, stream=None):
        """One iteration in place on beta (asynchronous)."""
        b = self._beta(beta)
        k = b.shape[0]
        lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lambdas, dtype=np.float64), (k,)))
        rc = L.cox_prox_step(self.h, _vp(b), _vp(lam), k, float(step), _stream_ptr(stream))
        L.check(rc, "cox_prox_step")
        return beta

    def prox_step_eta(self, beta: torch.Tensor, eta: torch.Tensor, lambdas, step: float, stream=None):
        """One iteration of a column shard from the summed eta (k, n) float64 on
        the device (cox_prox_step_eta), in place on this shard's beta."""
        b = self._beta(beta)
        k = b.shape[0]
        if eta.dtype != torch.float64 or not eta.is_cuda or tuple(eta.shape) != (k, self.n) or not eta.is_contiguous():
            raise ValueError(f"eta must be a contiguous float64 CUDA tensor of shape ({k}, {self.n})")
        lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lambdas, dtype=np.float64), (k,)))
        L.check(L.cox_prox_step_eta(self.h, _vp(b), _vp(eta), _vp(lam), k, float(step), _stream_ptr(stream)),
                "cox_prox_step_eta")
        return beta

    def last_loss_l1(self, k: int, stream=None):
        """(f, ||beta||_1 of this handle's columns) at the iterate entering the last step."""
        f = np.zeros(k)
        l1 = np.zeros(k)
        L.check(L.cox_last_loss_l1(self.h, _vp(f), _vp(l1), k, _stream_ptr(stream)), "cox_last_loss_l1")
        return f, l1

    def prox_step_host(self, beta: np.ndarray, lambdas, step: float, stream=None):
        """One iteration on a host array (k, p), copied in and out."""
        k = beta.shape[0] if beta.ndim == 2 else 1
        lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lambdas, dtype=np.float64), (k,)))
        rc = L.cox_prox_step_host(self.h, _vp(beta), _vp(lam), k, float(step), _stream_ptr(stream))
        L.check(rc, "cox_prox_step_host")
        return beta

    def sync(self, stream=None):
        L.check(L.cox_sync(self.h, _stream_ptr(stream)), "cox_sync")

    def last_objective(self, k: int, stream=None) -> np.ndarray:
        out = np.zeros(k)
        L.check(L.cox_last_objective(self.h, _vp(out), k, _stream_ptr(stream)), "cox_last_objective")
        return out

    def path_fit(self, lambdas, step: float, max_iter: int = 1000, tol: float = 1e-6,
                 beta: torch.Tensor | None = None, warm: int = 0, stream=None):
        """Fit k penalties; returns (beta (k,p), iterations, objectives, converged)."""
        lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64).ravel())
        k = len(lam)
        if beta is None:
            beta = self.zeros(k)
        b = self._beta(beta)
        iters = np.zeros(k, np.int32)
        obj = np.zeros(k)
        rc = L.cox_path_fit(self.h, _vp(lam), k, int(max_iter), float(tol), float(step), int(warm), _vp(b),
                            _vp(iters), _vp(obj), _stream_ptr(stream))
        L.check(rc, "cox_path_fit", allow=(L.COX_OK, L.COX_ERR_NOT_CONVERGED))
        return beta, iters, obj, rc == L.COX_OK

    def path_seq(self, lambdas, step: float, max_iter: int = 1000, tol: float = 1e-6, warm: bool = True,
                 stream=None):
        """The Section 6 path, one penalty after another (cox_path_seq), each from
        the previous one's solution when warm.  Returns (B (L, p), G (L, q),
        iterations, objectives, converged)."""
        lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64).ravel())
        nl = len(lam)
        B = self.zeros(nl)
        G = np.zeros((nl, max(self.q, 1)))
        iters = np.zeros(nl, np.int32)
        obj = np.zeros(nl)
        rc = L.cox_path_seq(self.h, _vp(lam), nl, int(max_iter), float(tol), float(step), int(bool(warm)), _vp(B),
                            _vp(G), _vp(iters), _vp(obj), _stream_ptr(stream))
        L.check(rc, "cox_path_seq", allow=(L.COX_OK, L.COX_ERR_NOT_CONVERGED))
        return B, G[:, :self.q], iters, obj, rc == L.COX_OK

    # -- unpenalised covariates (Section 6) ---------------------------------------------
    def set_covariates(self, Z):
        """Covariates that enter without a penalty: Z (n, q) in subject order, or None."""
        if Z is None:
            L.check(L.cox_set_covariates(self.h, None, 0), "cox_set_covariates")
            self.q = 0
            return
        Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64).reshape(self.n, -1))
        L.check(L.cox_set_covariates(self.h, _vp(Z), Z.shape[1]), "cox_set_covariates")
        self.q = Z.shape[1]

    def gamma(self, k: int) -> np.ndarray:
        """The handle's unpenalised coefficients for k columns, shape (k, q)."""
        out = np.zeros((k, max(self.q, 1)))
        L.check(L.cox_get_gamma(self.h, _vp(out), k), "cox_get_gamma")
        return out[:, :self.q]

    def set_gamma(self, gamma, k: int):
        g = None if gamma is None else np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).reshape(k, self.q))
        L.check(L.cox_set_gamma(self.h, _vp(g), k), "cox_set_gamma")

    def grad_gamma(self, k: int) -> np.ndarray:
        """d f / d gamma at the last evaluation for k columns, shape (k, q)."""
        out = np.zeros((k, max(self.q, 1)))
        L.check(L.cox_grad_gamma(self.h, _vp(out), k), "cox_grad_gamma")
        return out[:, :self.q]

    def get_state(self) -> bytes:
        size = ctypes.c_size_t()
        L.check(L.cox_get_state(self.h, None, ctypes.byref(size)), "cox_get_state")
        buf = ctypes.create_string_buffer(size.value)
        L.check(L.cox_get_state(self.h, buf, ctypes.byref(size)), "cox_get_state")
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        L.check(L.cox_set_state(self.h, buf, len(blob)), "cox_set_state")
