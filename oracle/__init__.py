"""FP64 CPU oracle for the l1-regularised Cox proximal-gradient iteration.

TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code
with the CUDA solver (``paper_2010_16114_gb300``), and neither imports the
other.

The arithmetic lives in ``cox_oracle.c`` (plain loops, FP64, no FMA
contraction); this module only marshals numpy arrays.  Every function cites
the passage of arXiv 2010.16114 (DistStat.jl) it follows:

* ``risk`` / ``risk_bruteforce`` -- Section 5.3, W_j, pi_ij and P delta;
  Breslow ties per Section 6.
* ``eta`` / ``grad`` -- Section 5.3, X beta and Delta = X^T (I - P) delta
  (divided by n; the 1/n normalisation is this build's reading);
  ``eta_u8`` / ``grad_u8`` the same with genotype columns held as bytes.
* ``prox`` / ``soft_threshold`` -- Section 4.2 soft threshold, applied as
  S(beta + sigma g, sigma lambda) (Section 5.3 iteration).
* ``opnorm2`` -- Section 4.4 power method; ``lipschitz`` = 2 ||X_c||_2^2 / n
  from the step-size remark in Section 5.3.
* ``ista`` -- the Section 5.3 iteration repeated.
* ``ista_unpen`` -- the iteration with an unpenalised block (Section 6: sex
  and principal components enter unpenalised).
* ``path`` -- the Section 6 lambda path with the lag stopping rule.
* ``rank_by_entry`` -- the Section 6 SNP ranking by entry lambda.
* ``nmf`` / ``nmf_objective`` -- Section 5.1 nonnegative matrix factorization:
  the multiplicative (Lee-Seung) and alternating projected gradient updates,
  and ||X - V W||_F^2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cox_oracle.c")
_LIBS = {False: os.path.join(_HERE, "liboracle.so"), True: os.path.join(_HERE, "liboracle_ld.so")}

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_f64 = ctypes.c_double


def build(force: bool = False) -> None:
    """Compile the FP64 oracle and its long-double twin with gcc."""
    for ld, path in _LIBS.items():
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + ".tmp"
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
            if ld:
                cmd.append("-DORC_LONG_DOUBLE")
            subprocess.check_call(cmd + ["-o", tmp, _SRC, "-lm"])
            os.replace(tmp, path)


_loaded: dict = {}


def _lib(long_double: bool = False):
    if long_double not in _loaded:
        build()
        lib = ctypes.CDLL(_LIBS[long_double])
        for name in ("orc_risk", "orc_risk_bruteforce"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [_i64, _p, _p, _p, _p, _p, _p]
        lib.orc_argsort.restype = ctypes.c_int
        lib.orc_argsort.argtypes = [_i64, _p, _p]
        lib.orc_eta.restype = None
        lib.orc_eta.argtypes = [_i64, _i64, _p, _p, _p, _p]
        lib.orc_grad.restype = None
        lib.orc_grad.argtypes = [_i64, _i64, _p, _p, _p, _p, _p]
        lib.orc_eta_u8.restype = None
        lib.orc_eta_u8.argtypes = [_i64, _i64, _p, _p, _p, _p]
        lib.orc_grad_u8.restype = None
        lib.orc_grad_u8.argtypes = [_i64, _i64, _p, _p, _p, _p, _p]
        lib.orc_soft_threshold.restype = _f64
        lib.orc_soft_threshold.argtypes = [_f64, _f64]
        lib.orc_prox.restype = None
        lib.orc_prox.argtypes = [_i64, _p, _p, _f64, _f64, _p]
        lib.orc_objective.restype = ctypes.c_int
        lib.orc_objective.argtypes = [_i64, _i64, _p, _p, _p, _p, _p, _f64, _p]
        lib.orc_ista.restype = ctypes.c_int
        lib.orc_ista.argtypes = [_i64, _i64, _p, _p, _p, _p, _f64, _f64, _i64, _p, _p, _p]
        lib.orc_opnorm2.restype = _f64
        lib.orc_opnorm2.argtypes = [_i64, _i64, _p, _p, _p, _f64, _i64, _p]
        lib.orc_ista_unpen.restype = ctypes.c_int
        lib.orc_ista_unpen.argtypes = [_i64, _i64, _p, _p, _i64, _p, _p, _p, _f64, _f64, _i64, _p, _p, _p]
        lib.orc_path.restype = ctypes.c_int
        lib.orc_path.argtypes = [_i64, _i64, _p, _p, _i64, _p, _p, _p, _f64, _i64, _p, _f64, _i64, _i64,
                                 ctypes.c_int, _p, _p, _p]
        lib.orc_nmf_objective.restype = _f64
        lib.orc_nmf_objective.argtypes = [_i64, _i64, _i64, _p, _p, _p]
        lib.orc_nmf.restype = ctypes.c_int
        lib.orc_nmf.argtypes = [_i64, _i64, _i64, _p, _p, _p, _i64, ctypes.c_int, _f64]
        lib.orc_rank_by_entry.restype = _i64
        lib.orc_rank_by_entry.argtypes = [_i64, _i64, _p, _p, _p, _p]
        _loaded[long_double] = lib
    return _loaded[long_double]


def _f(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _cols(X) -> np.ndarray:
    """(n, m) matrix -> column-major float64 buffer."""
    return np.asfortranarray(X, dtype=np.float64)


def argsort(y) -> np.ndarray:
    """Stable ascending order of the observed times (Section 5.3 sorting)."""
    y = _f(y)
    ord_ = np.zeros(len(y), np.int64)
    _lib().orc_argsort(len(y), _ptr(y), _ptr(ord_))
    return ord_


def risk(y, delta, eta, long_double: bool = False):
    """(W, u, f) by sorted cumulative sums: W_i = sum_{y_j >= y_i} exp(eta_j - c),
    u = P delta, f = -l(beta)/n (Section 5.3; Breslow ties, Section 6)."""
    y, delta, eta = _f(y), _u8(delta), _f(eta)
    n = len(y)
    W, u, loss = np.zeros(n), np.zeros(n), _f64()
    rc = _lib(long_double).orc_risk(n, _ptr(y), _ptr(delta), _ptr(eta), _ptr(W), _ptr(u),
                                    ctypes.byref(loss))
    if rc != 0:
        raise FloatingPointError(f"orc_risk returned {rc}")
    return W, u, loss.value


def risk_bruteforce(y, delta, eta, long_double: bool = False):
    """Same as ``risk`` from the O(n^2) definitions of W_j and pi_ij
    (Section 5.3; Appendix B's P delta double loop).  Tiny n only."""
    y, delta, eta = _f(y), _u8(delta), _f(eta)
    n = len(y)
    W, u, loss = np.zeros(n), np.zeros(n), _f64()
    rc = _lib(long_double).orc_risk_bruteforce(n, _ptr(y), _ptr(delta), _ptr(eta), _ptr(W),
                                               _ptr(u), ctypes.byref(loss))
    if rc != 0:
        raise FloatingPointError(f"orc_risk_bruteforce returned {rc}")
    return W, u, loss.value


def eta(Xcols, mu, beta, long_double: bool = False) -> np.ndarray:
    """eta = X_c beta over the given columns (Section 5.3, X beta)."""
    Xc = _cols(Xcols)
    n, m = Xc.shape
    beta = _f(beta)
    mu = None if mu is None else _f(mu)
    out = np.zeros(n)
    _lib(long_double).orc_eta(n, m, _ptr(Xc), _ptr(mu), _ptr(beta), _ptr(out))
    return out


def grad(Xcols, mu, delta, u, long_double: bool = False) -> np.ndarray:
    """g = X_c^T (delta - u) / n over the given columns (Section 5.3, Delta / n)."""
    Xc = _cols(Xcols)
    n, m = Xc.shape
    mu = None if mu is None else _f(mu)
    g = np.zeros(m)
    _lib(long_double).orc_grad(n, m, _ptr(Xc), _ptr(mu), _ptr(_u8(delta)), _ptr(_f(u)), _ptr(g))
    return g


def eta_u8(Xt, mu, beta) -> np.ndarray:
    """``eta`` with the columns given as bytes: Xt is (m, n) uint8, row t =
    column t of X (Section 5.3, X beta).  Bitwise equal to ``eta``."""
    Xt = np.ascontiguousarray(Xt, dtype=np.uint8)
    m, n = Xt.shape
    out = np.zeros(n)
    _lib().orc_eta_u8(n, m, _ptr(Xt), _ptr(None if mu is None else _f(mu)), _ptr(_f(beta)), _ptr(out))
    return out


def grad_u8(Xt, mu, delta, u) -> np.ndarray:
    """``grad`` with the columns given as bytes: Xt is (m, n) uint8, row t =
    column t of X (Section 5.3, Delta / n).  Bitwise equal to ``grad``."""
    Xt = np.ascontiguousarray(Xt, dtype=np.uint8)
    m, n = Xt.shape
    g = np.zeros(m)
    _lib().orc_grad_u8(n, m, _ptr(Xt), _ptr(None if mu is None else _f(mu)), _ptr(_u8(delta)), _ptr(_f(u)),
                       _ptr(g))
    return g


def soft_threshold(x: float, t: float) -> float:
    """Section 4.2 soft threshold."""
    return _lib().orc_soft_threshold(float(x), float(t))


def prox(beta, g, sigma: float, lam: float) -> np.ndarray:
    """S(beta + sigma g, sigma lambda) elementwise (Section 5.3)."""
    beta, g = _f(beta), _f(g)
    out = np.zeros_like(beta)
    _lib().orc_prox(len(beta), _ptr(beta), _ptr(g), sigma, lam, _ptr(out))
    return out


def objective(X, mu, y, delta, beta, lam: float) -> float:
    """F_lambda(beta) = f(beta) + lambda ||beta||_1."""
    Xc = _cols(X)
    n, p = Xc.shape
    F = _f64()
    rc = _lib().orc_objective(n, p, _ptr(Xc), _ptr(None if mu is None else _f(mu)), _ptr(_f(y)),
                              _ptr(_u8(delta)), _ptr(_f(beta)), lam, ctypes.byref(F))
    if rc != 0:
        raise FloatingPointError(f"orc_objective returned {rc}")
    return F.value


def ista(X, mu, y, delta, sigma: float, lam: float, iters: int, beta0=None):
    """ISTA (Section 5.3) for ``iters`` iterations from beta0 (default 0).
    Returns (beta, F_trace, g_last): F_trace[t] = F_lambda(beta_t)."""
    Xc = _cols(X)
    n, p = Xc.shape
    beta = np.zeros(p) if beta0 is None else _f(beta0).copy()
    F = np.zeros(max(iters, 1))
    g = np.zeros(p)
    rc = _lib().orc_ista(n, p, _ptr(Xc), _ptr(None if mu is None else _f(mu)), _ptr(_f(y)),
                         _ptr(_u8(delta)), sigma, lam, iters, _ptr(beta), _ptr(F), _ptr(g))
    if rc != 0:
        raise FloatingPointError(f"orc_ista returned {rc}")
    return beta, F[:iters], g


def opnorm2(X, mu, v0, tol: float = 1e-6, maxiter: int = 1000):
    """||X_c||_2 by the power method (Section 4.4).  Returns (norm, iterations)."""
    Xc = _cols(X)
    n, p = Xc.shape
    it = _i64()
    v = _lib().orc_opnorm2(n, p, _ptr(Xc), _ptr(None if mu is None else _f(mu)), _ptr(_f(v0)),
                           tol, maxiter, ctypes.byref(it))
    return v, it.value


def lipschitz(X, mu, v0, tol: float = 1e-6, maxiter: int = 1000) -> float:
    """L = 2 ||X_c||_2^2 / n: the Section 5.3 step sigma = 1 / (2 ||X||_2^2)
    rescaled to the 1/n-normalised loss, with the centred design."""
    nrm, _ = opnorm2(X, mu, v0, tol, maxiter)
    return 2.0 * nrm * nrm / X.shape[0]


def lambda_max(X, mu, y, delta) -> float:
    """Smallest lambda with beta = 0 optimal: ||g(0)||_inf."""
    W, u, _ = risk(y, delta, np.zeros(len(y)))
    return float(np.max(np.abs(grad(X, mu, delta, u))))


def _zcols(Z, n: int) -> np.ndarray:
    """Z (n x q, any layout) as a column-major float64 array; None -> q = 0."""
    if Z is None:
        return np.zeros((n, 0))
    Z = np.asarray(Z, dtype=np.float64)
    if Z.ndim == 1:
        Z = Z[:, None]
    return Z


def ista_unpen(X, mu, Z, y, delta, sigma: float, lam: float, iters: int, beta0=None, gamma0=None):
    """ISTA with an unpenalised block Z (Section 6: sex and principal
    components enter unpenalised): beta thresholded, gamma a plain gradient
    step.  Returns (beta, gamma, F_trace)."""
    Xc = _cols(X)
    n, p = Xc.shape
    Zc = _cols(_zcols(Z, n))
    q = Zc.shape[1]
    beta = np.zeros(p) if beta0 is None else _f(beta0).copy()
    gamma = np.zeros(max(q, 1)) if gamma0 is None else _f(gamma0).copy()
    F = np.zeros(max(iters, 1))
    rc = _lib().orc_ista_unpen(n, p, _ptr(Xc), _ptr(None if mu is None else _f(mu)), q, _ptr(Zc),
                               _ptr(_f(y)), _ptr(_u8(delta)), sigma, lam, iters, _ptr(beta), _ptr(gamma),
                               _ptr(F))
    if rc != 0:
        raise FloatingPointError(f"orc_ista_unpen returned {rc}")
    return beta, gamma[:q], F[:iters]


def path(X, mu, Z, y, delta, sigma: float, lams, tol: float = 1e-5, lag: int = 10,
         max_iter: int = 1000, warm: bool = False):
    """The Section 6 lambda path: each lambda solved by ISTA (with the
    unpenalised block Z, may be None) until |F_t - F_{t-lag}| / |F_t + 1| < tol
    or max_iter, from zero or, warm, from the previous lambda's solution.
    Returns (B (L x p), G (L x q), iters (L))."""
    Xc = _cols(X)
    n, p = Xc.shape
    Zc = _cols(_zcols(Z, n))
    q = Zc.shape[1]
    lams = _f(lams)
    L = len(lams)
    B = np.zeros((L, p))
    G = np.zeros((L, max(q, 1)))
    it = np.zeros(L, np.int64)
    rc = _lib().orc_path(n, p, _ptr(Xc), _ptr(None if mu is None else _f(mu)), q, _ptr(Zc), _ptr(_f(y)),
                         _ptr(_u8(delta)), sigma, L, _ptr(lams), tol, lag, max_iter, int(bool(warm)),
                         _ptr(B), _ptr(G), _ptr(it))
    if rc != 0:
        raise FloatingPointError(f"orc_path returned {rc}")
    return B, G[:, :q], it


def rank_by_entry(lams, B):
    """Section 6 SNP ranking: SNPs with a nonzero coefficient on the path,
    ordered by the largest lambda at which they are nonzero, ties by |beta|
    there, then by index.  B is L x p (row l = coefficients at lams[l]).
    Returns (order, entry): entry[j] = index of SNP j's entry lambda or -1."""
    lams = _f(lams)
    B = np.ascontiguousarray(B, dtype=np.float64)
    L, p = B.shape
    order = np.zeros(max(p, 1), np.int64)
    entry = np.zeros(max(p, 1), np.int64)
    cnt = _lib().orc_rank_by_entry(p, L, _ptr(lams), _ptr(B), _ptr(order), _ptr(entry))
    if cnt < 0:
        raise MemoryError("orc_rank_by_entry")
    return order[:cnt], entry[:p]


def nmf_objective(X, V, W) -> float:
    """||X - V W||_F^2 (Section 5.1), X (m, n), V (m, r), W (r, n)."""
    X, V, W = _f(X), _f(V), _f(W)
    m, n = X.shape
    r = V.shape[1]
    return _lib().orc_nmf_objective(m, n, r, _ptr(X), _ptr(V), _ptr(W))


def nmf(X, V, W, iters: int, algo: str = "mult", eps: float = 1e-10):
    """``iters`` NMF iterations (Section 5.1): V from W, then W from the new V,
    by the multiplicative ("mult") or alternating projected gradient ("apg")
    update.  Returns the updated (V, W)."""
    X = _f(X)
    V = _f(V).copy()
    W = _f(W).copy()
    m, n = X.shape
    r = V.shape[1]
    rc = _lib().orc_nmf(m, n, r, _ptr(X), _ptr(V), _ptr(W), iters, {"mult": 0, "apg": 1}[algo], eps)
    if rc != 0:
        raise ValueError(f"orc_nmf returned {rc}")
    return V, W
