"""Seeded synthetic inputs for the l1-regularised Cox workloads.

Input generation only: this package holds none of the Cox method's
arithmetic.  Both the FP64 oracle (``oracle/``) and the CUDA solver library
consume what it produces; neither is imported here.

Workload recipes (shapes of the paper's simulated Cox data, Section 5.3, and
of its UK Biobank analysis, Section 6), keyed by what they are:

* ``normal_1k_2k`` -- n=1000 subjects, p=2000 predictors, x_ij ~ N(0,1), 20
  causal effects ~ N(0, 0.5^2), T ~ Exp(rate exp(x'beta)), C ~ Exp(r) with r
  set so 30% are censored, no ties; lambda = 0.5 lambda_max, 200 iterations,
  FP64.
* ``geno_100k_50k``, ``geno_200k_10k``, ``geno_400k_100k_k32``,
  ``geno_400k_500k_k16`` -- n x p genotypes x_ij ~ Binomial(2, MAF_j),
  MAF_j ~ U(lo, hi), causal effects on centred genotypes,
  T = E / (h0 exp(eta)), C ~ U(1, dmax), y = ceil(min(T, C)) in whole days
  (ties), h0 set to hit the event rate; k penalties (1 unless the name says).

NMF inputs (Section 5.1 experiments, ``nmf_inputs``): X m x n on the grid
k / 256 (uniform, exact in bf16), V m x r and W r x n uniform on [0, 1) in FP32;
the seed ``NMF_SEED`` stands for the paper's ``rand!`` draws.

Each recipe carries its own seed; ``scaled`` keeps recipe and seed and
changes only the sizes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_DEV_SRC = os.path.join(_HERE, "synth_dev.cu")
_DEV_LIB = os.path.join(_HERE, "libsynth_dev.so")



def build_host(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_device(force: bool = False) -> str:
    """Compile synth_dev.cu into libsynth_dev.so for sm_103a."""
    if force or not os.path.exists(_DEV_LIB) or os.path.getmtime(_DEV_LIB) < os.path.getmtime(_DEV_SRC):
        tmp = _DEV_LIB + ".tmp"
        subprocess.check_call(["nvcc", "-O3", "-shared", "-Xcompiler", "-fPIC",
                               "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
                               "-o", tmp, _DEV_SRC])
        os.replace(tmp, _DEV_LIB)
    return _DEV_LIB


_lib = None
_dev = None

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_f64 = ctypes.c_double


def _host():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_host())
        lib.syn_draw.restype = _u64
        lib.syn_draw.argtypes = [_u64, _u64, _u64, _u64]
        lib.syn_maf.argtypes = [_u64, _i64, _f64, _f64, _p, _p]
        lib.syn_genotypes.argtypes = [_u64, _p, _i64, _i64, _i64, _i64, _p]
        lib.syn_genotype_cols.argtypes = [_u64, _p, _i64, _p, _i64, _p]
        lib.syn_genotype_cols_u8.argtypes = [_u64, _p, _i64, _p, _i64, _p]
        lib.syn_genotypes_packed.argtypes = [_u64, _p, _i64, _i64, _i64, _p]
        lib.syn_normals.argtypes = [_u64, _i64, _i64, _i64, _i64, _p]
        lib.syn_normal_vec.argtypes = [_u64, _u64, _i64, _p]
        lib.syn_uniform_vec.argtypes = [_u64, _u64, _i64, _p]
        lib.syn_causal.restype = ctypes.c_int
        lib.syn_causal.argtypes = [_u64, _i64, _i64, _f64, _p, _p]
        lib.syn_times_exp.restype = ctypes.c_int
        lib.syn_times_exp.argtypes = [_u64, _i64, _p, _f64, _p, _p, _p]
        lib.syn_nmf_x.argtypes = [_u64, _i64, _i64, _i64, _p]
        lib.syn_nmf_factor.argtypes = [_u64, ctypes.c_int, _i64, _p]
        lib.syn_times_days.restype = ctypes.c_int
        lib.syn_times_days.argtypes = [_u64, _i64, _p, _f64, _i64, _p, _p, _p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass(frozen=True)
class Recipe:
    """One workload recipe; ``scaled`` keeps the recipe and changes sizes."""
    name: str
    seed: int
    kind: str            # "normal" or "geno"
    n: int
    p: int
    k: int
    n_causal: int
    effect_sd: float
    maf_lo: float = 0.05
    maf_hi: float = 0.5
    cens_frac: float = 0.30   # normal: censored fraction
    event_frac: float = 0.20  # geno: event fraction
    dmax: int = 3650          # geno: longest follow-up in days
    lam_hi: float = 0.5       # lambda grid top, as a fraction of lambda_max
    lam_lo: float = 0.5       # lambda grid bottom (log-spaced, inclusive)
    iters: int = 200
    center: bool = True

    def scaled(self, n: int | None = None, p: int | None = None, k: int | None = None,
               n_causal: int | None = None) -> "Recipe":
        n = self.n if n is None else n
        p = self.p if p is None else p
        nc = self.n_causal if n_causal is None else n_causal
        return replace(self, n=n, p=p, k=self.k if k is None else k, n_causal=min(nc, max(1, p // 4)))

    def lambda_fracs(self) -> np.ndarray:
        """Fractions of lambda_max: k values log-spaced from lam_hi to lam_lo."""
        if self.k == 1:
            return np.array([self.lam_hi])
        return np.exp(np.linspace(np.log(self.lam_hi), np.log(self.lam_lo), self.k))


WORKLOADS = {r.name: r for r in (
    Recipe("normal_1k_2k", 2010161140, "normal", 1000, 2000, 1, 20, 0.5, cens_frac=0.30,
           lam_hi=0.5, lam_lo=0.5, iters=200, center=False),
    Recipe("geno_100k_50k", 2010161141, "geno", 100_000, 50_000, 1, 50, 0.1, 0.05, 0.5,
           event_frac=0.20, dmax=3650, lam_hi=0.5, lam_lo=0.5, iters=50),
    Recipe("geno_200k_10k", 2010161142, "geno", 200_000, 10_000, 1, 50, 0.1, 0.05, 0.5,
           event_frac=0.20, dmax=3650, lam_hi=0.5, lam_lo=0.5, iters=50),
    Recipe("geno_400k_100k_k32", 2010161143, "geno", 400_000, 100_000, 32, 100, 0.1, 0.05, 0.5,
           event_frac=0.10, dmax=3650, lam_hi=1.0, lam_lo=0.01, iters=50),
    Recipe("geno_400k_500k_k16", 2010161144, "geno", 400_000, 500_000, 16, 500, 0.05, 0.01, 0.5,
           event_frac=0.05, dmax=5000, lam_hi=1.0, lam_lo=0.01, iters=1000),
)}


class Workload:
    """Generated survival data plus on-demand access to X.

    ``y``/``delta`` are in subject order.  X is never materialised unless
    asked for: ``dense()`` gives the whole matrix (small cases), ``cols(j)``
    regenerates chosen columns, ``packed_rows()`` gives the row-major 2-bit
    packed form (4 codes per byte, SNP j at bits 2*(j%4))."""

    def __init__(self, recipe: Recipe):
        self.r = recipe
        lib = _host()
        n, p, seed = recipe.n, recipe.p, recipe.seed
        nc = min(recipe.n_causal, p)
        self.causal_idx = np.zeros(nc, np.int64)
        self.causal_eff = np.zeros(nc, np.float64)
        if lib.syn_causal(seed, p, nc, recipe.effect_sd, _ptr(self.causal_idx), _ptr(self.causal_eff)) != 0:
            raise RuntimeError("syn_causal failed")
        self.beta_true = np.zeros(p)
        self.beta_true[self.causal_idx] = self.causal_eff
        if recipe.kind == "geno":
            self.maf = np.zeros(p)
            self.thr = np.zeros(p, np.uint32)
            lib.syn_maf(seed, p, recipe.maf_lo, recipe.maf_hi, _ptr(self.maf), _ptr(self.thr))
            xc = self.cols(self.causal_idx)
            xc = xc - xc.mean(axis=0, keepdims=True)
            eta = xc @ self.causal_eff
        else:
            self.maf = None
            self.thr = None
            xc = self.cols(self.causal_idx)
            eta = xc @ self.causal_eff
        self.eta_true = np.ascontiguousarray(eta, dtype=np.float64)
        self.y = np.zeros(n)
        self.delta = np.zeros(n, np.uint8)
        if recipe.kind == "geno":
            h0 = ctypes.c_double()
            rc = lib.syn_times_days(seed, n, _ptr(self.eta_true), recipe.event_frac, recipe.dmax,
                                    _ptr(self.y), _ptr(self.delta), ctypes.byref(h0))
            self.h0 = h0.value
        else:
            r = ctypes.c_double()
            rc = lib.syn_times_exp(seed, n, _ptr(self.eta_true), recipe.cens_frac,
                                   _ptr(self.y), _ptr(self.delta), ctypes.byref(r))
            self.h0 = r.value
        if rc != 0:
            raise RuntimeError("survival time generation failed")

    @property
    def n(self):
        return self.r.n

    @property
    def p(self):
        return self.r.p

    def cols(self, idx) -> np.ndarray:
        """Columns ``idx`` of X as float64, shape (n, len(idx)), C-order."""
        idx = np.ascontiguousarray(np.atleast_1d(idx), dtype=np.int64)
        out = np.zeros((len(idx), self.r.n), np.float64)
        lib = _host()
        if self.r.kind == "geno":
            lib.syn_genotype_cols(self.r.seed, _ptr(self.thr), self.r.n, _ptr(idx), len(idx), _ptr(out))
        else:
            tmp = np.zeros(self.r.n)
            for c, j in enumerate(idx):
                lib.syn_normals(self.r.seed, 0, self.r.n, int(j), 1, _ptr(tmp))
                out[c] = tmp
        return np.ascontiguousarray(out.T)

    def cols_u8(self, idx, threads: int = 1) -> np.ndarray:
        """Genotype columns ``idx`` as uint8, shape (len(idx), n): row c is
        column idx[c] of X (column-major X restricted to idx).  With threads > 1
        the columns are generated in parallel blocks (the C calls release the
        interpreter lock)."""
        assert self.r.kind == "geno"
        idx = np.ascontiguousarray(np.atleast_1d(idx), dtype=np.int64)
        n, m = self.r.n, len(idx)
        out = np.zeros((m, n), np.uint8)
        lib = _host()

        def block(c0, c1):
            lib.syn_genotype_cols_u8(self.r.seed, _ptr(self.thr), n,
                                     ctypes.c_void_p(idx.ctypes.data + 8 * c0), c1 - c0,
                                     ctypes.c_void_p(out.ctypes.data + c0 * n))

        if threads <= 1 or m < 2:
            block(0, m)
        else:
            from concurrent.futures import ThreadPoolExecutor
            step = max(1, -(-m // (4 * threads)))
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda c0: block(c0, min(m, c0 + step)), range(0, m, step)))
        return out

    def rows_u8(self, rows) -> np.ndarray:
        """Genotype rows ``rows`` as uint8, shape (len(rows), p)."""
        assert self.r.kind == "geno"
        rows = np.atleast_1d(np.asarray(rows, dtype=np.int64))
        out = np.zeros((len(rows), self.r.p), np.uint8)
        lib = _host()
        for c, i in enumerate(rows):
            lib.syn_genotypes(self.r.seed, _ptr(self.thr), int(i), 1, 0, self.r.p,
                              ctypes.c_void_p(out.ctypes.data + c * self.r.p))
        return out

    def dense(self) -> np.ndarray:
        """Whole X: uint8 codes (geno) or float64 (normal), row-major n x p."""
        n, p = self.r.n, self.r.p
        if self.r.kind == "geno":
            out = np.zeros((n, p), np.uint8)
            _host().syn_genotypes(self.r.seed, _ptr(self.thr), 0, n, 0, p, _ptr(out))
        else:
            out = np.zeros((n, p), np.float64)
            _host().syn_normals(self.r.seed, 0, n, 0, p, _ptr(out))
        return out

    def packed_rows(self, i0: int = 0, ni: int | None = None) -> np.ndarray:
        """Row-major 2-bit packed codes, shape (ni, ceil(p/4)) uint8."""
        assert self.r.kind == "geno"
        ni = self.r.n - i0 if ni is None else ni
        out = np.zeros((ni, (self.r.p + 3) // 4), np.uint8)
        _host().syn_genotypes_packed(self.r.seed, _ptr(self.thr), self.r.p, i0, ni, _ptr(out))
        return out

    def packed_rows_device(self, out_ptr: int, stream_ptr: int = 0, thr_dev_ptr: int | None = None,
                           i0: int = 0, ni: int | None = None):
        """Write the row-major packed codes straight into device memory."""
        global _dev
        assert self.r.kind == "geno"
        if _dev is None:
            _dev = ctypes.CDLL(build_device())
            _dev.syn_dev_genotypes_packed.restype = ctypes.c_int
            _dev.syn_dev_genotypes_packed.argtypes = [_u64, _p, _i64, _i64, _i64, _p, _p]
        ni = self.r.n - i0 if ni is None else ni
        rc = _dev.syn_dev_genotypes_packed(self.r.seed, ctypes.c_void_p(thr_dev_ptr), self.r.p, i0, ni,
                                           ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream_ptr))
        if rc != 0:
            raise RuntimeError(f"syn_dev_genotypes_packed failed ({rc})")

    def normal_vec(self, stream: int, m: int) -> np.ndarray:
        out = np.zeros(m)
        _host().syn_normal_vec(self.r.seed, stream, m, _ptr(out))
        return out

    def uniform_vec(self, stream: int, m: int) -> np.ndarray:
        out = np.zeros(m)
        _host().syn_uniform_vec(self.r.seed, stream, m, _ptr(out))
        return out


def workload(name: str, **sizes) -> Workload:
    """Generate recipe ``name`` (optionally at other sizes, same recipe and seed)."""
    r = WORKLOADS[name]
    if sizes:
        r = r.scaled(**sizes)
    return Workload(r)


def normal_vec(seed: int, stream: int, m: int) -> np.ndarray:
    out = np.zeros(m)
    _host().syn_normal_vec(seed, stream, m, _ptr(out))
    return out


NMF_SEED = 2010161150


def nmf_x(m: int, n: int, seed: int = NMF_SEED, i0: int = 0) -> np.ndarray:
    """Rows [i0, i0 + m) of the NMF data matrix (float32, values k / 256)."""
    out = np.empty((m, n), np.float32)
    _host().syn_nmf_x(seed, i0, m, n, _ptr(out))
    return out


def nmf_inputs(m: int, n: int, r: int, seed: int = NMF_SEED):
    """(X, V0, W0): X m x n on the grid k / 256, V0 m x r and W0 r x n uniform
    on [0, 1), all float32."""
    X = nmf_x(m, n, seed)
    V = np.empty((m, r), np.float32)
    W = np.empty((r, n), np.float32)
    _host().syn_nmf_factor(seed, 0, m * r, _ptr(V))
    _host().syn_nmf_factor(seed, 1, r * n, _ptr(W))
    return X, V, W
