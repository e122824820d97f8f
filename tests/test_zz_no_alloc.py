"""The allocation-free step size (cox_lipschitz_noalloc) agrees with
cox_lipschitz.

The entry point serves callers that cannot allocate device memory when they
call it (memory already held by another allocator; loops that cannot absorb
the device-wide synchronisation of cudaFree).  Its work vectors live in a
fixed 16 MiB array inside the library, shared by all calls.  This file is
collected last so that, run after the whole suite, the shared array already
holds data from earlier calls; it must also pass alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from helpers import dense_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2010_16114_gb300 as P
    P.build()
    from paper_2010_16114_gb300 import _lib
    return _lib


def _both(L, prob, v0, tol, maxiter):
    vp = v0.ctypes.data_as(ctypes.c_void_p) if v0 is not None else None
    rc1, a = L.cox_lipschitz(prob.h, vp, tol, maxiter)
    rc2, b = L.cox_lipschitz_noalloc(prob.h, vp, tol, maxiter)
    assert rc1 == L.COX_OK and rc2 == L.COX_OK
    return a, b


@pytest.mark.parametrize("precision", ["split_e4m3", "fp64"])
def test_noalloc_matches_allocating_call_twice(L, precision):
    from paper_2010_16114_gb300.cox import CoxProblem
    if precision == "fp64":
        w, X, Xf, mu = dense_problem("normal_1k_2k", n=700, p=300)
        Xin = Xf
    else:
        w, X, Xf, mu = dense_problem("geno_100k_50k", n=3000, p=700)
        Xin = X
    v0 = synth.normal_vec(95376, 7, w.p)
    with CoxProblem(Xin, w.y, w.delta, precision=precision) as prob:
        for call in range(2):  # two calls in a row share the array
            a, b = _both(L, prob, v0, 1e-6, 1000)
            assert abs(a - b) <= 1e-12 * abs(a), (call, a, b)
        a, b = _both(L, prob, None, 1e-8, 50)  # default start vector, other limits
        assert abs(a - b) <= 1e-12 * abs(a)


def test_noalloc_rejects_sizes_beyond_the_array(L):
    """n_pad float entries alone exceed 16 MiB: a clear argument error."""
    from paper_2010_16114_gb300.cox import CoxProblem
    n, p = 4_300_000, 1
    X = (np.arange(n) % 3).astype(np.uint8).reshape(n, p)
    y = np.arange(n, dtype=np.float64)
    d = np.zeros(n, np.uint8)
    d[::3] = 1
    with CoxProblem(X, y, d) as prob:
        rc, _ = L.cox_lipschitz_noalloc(prob.h, None, 1e-6, 5)
        assert rc == L.COX_ERR_ARG
        rc, Lv = L.cox_lipschitz(prob.h, None, 1e-6, 5)  # the allocating call still works
        assert rc == L.COX_OK and Lv > 0
