"""GB300 l1-regularised Cox proportional-hazards proximal gradient.

The hot path -- eta = X_c beta, Breslow risk-set scans, X_c^T (delta - u),
soft threshold -- runs in libcoxgb.so (hand-written CUDA for sm_103a) behind
the C ABI in include/coxgb.h.  This package builds that library, binds it
with ctypes (``_lib``, same names as the C calls) and offers a thin Python
front end (``CoxProblem``) and a ``torch.autograd.Function`` (``CoxNLL``).
The same library carries the Section 5.1 NMF (include/nmfgb.h, front end ``NMF``).
There is no CPU fallback: without the built library every call raises.
"""
from ._lib import CoxError, load  # noqa: F401
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("CoxProblem",):
        from .cox import CoxProblem
        return CoxProblem
    if name == "NMF":
        from .nmf import NMF
        return NMF
    if name in ("CoxNLL", "cox_nll"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
