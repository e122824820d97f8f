"""Python front end of the NMF entry points (include/nmfgb.h): X ~ V W by the
multiplicative or the alternating projected gradient updates of arXiv
2010.16114, Section 5.1.  Argument marshalling only: the products, updates and
reductions run in libcoxgb.so."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L

ALGOS = {"mult": L.NMF_MULTIPLICATIVE, "apg": L.NMF_APG}


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class NMF:
    """X (m x n, nonnegative) held on the device in bf16, rank r factors.

    ``stream`` arguments are CUDA stream handles as integers (``torch.cuda.Stream().cuda_stream``)
    or None for the legacy default stream."""

    def __init__(self, X: np.ndarray, r: int, device: int = -1):
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.ndim != 2:
            raise ValueError("X must be a matrix")
        self.m, self.n = X.shape
        self.r = int(r)
        h = ctypes.c_void_p()
        L.check(L.nmf_setup(_ptr(X), self.m, self.n, self.r, device, ctypes.byref(h)), "nmf_setup")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            L.nmf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_factors(self, V: np.ndarray, W: np.ndarray, stream=None):
        V = np.ascontiguousarray(V, dtype=np.float32)
        W = np.ascontiguousarray(W, dtype=np.float32)
        if V.shape != (self.m, self.r) or W.shape != (self.r, self.n):
            raise ValueError("V must be m x r and W r x n")
        L.check(L.nmf_set_factors(self._h, _ptr(V), _ptr(W), stream), "nmf_set_factors")

    def factors(self, stream=None):
        V = np.empty((self.m, self.r), np.float32)
        W = np.empty((self.r, self.n), np.float32)
        L.check(L.nmf_get_factors(self._h, _ptr(V), _ptr(W), stream), "nmf_get_factors")
        return V, W

    def iterate(self, iters: int, algo: str = "mult", eps: float = 1e-10, stream=None):
        L.check(L.nmf_iterate(self._h, ALGOS[algo], int(iters), float(eps), stream), "nmf_iterate")

    def sync(self, stream=None):
        L.check(L.nmf_sync(self._h, stream), "nmf_sync")

    def objective(self, stream=None) -> float:
        f = ctypes.c_double()
        L.check(L.nmf_objective(self._h, ctypes.byref(f), stream), "nmf_objective")
        return f.value

    def time_products(self, reps: int = 10, stream=None):
        """Mean milliseconds of one X W^T and one X^T V launch."""
        a, b = ctypes.c_double(), ctypes.c_double()
        L.check(L.nmf_time_products(self._h, int(reps), ctypes.byref(a), ctypes.byref(b), stream),
                "nmf_time_products")
        return a.value, b.value

    def info(self) -> dict:
        i = L.nmf_info()
        L.check(L.nmf_get_info(self._h, ctypes.byref(i)), "nmf_get_info")
        return {k: getattr(i, k) for k, _ in L.nmf_info._fields_}
