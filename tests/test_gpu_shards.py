"""One-GPU simulation of the column-sharded iteration (the paper's Section 5.3
layout with X split by columns over devices): each of G = 3 handles holds a
block of SNP columns, and the shards' linear predictors add up to the full
one, eta = sum_g (X_g)_c B_g, which is the all-reduce a multi-GPU run would do
before the replicated risk-set scans."""
import numpy as np
import pytest

import oracle
from helpers import dense_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _betas(p, k, seed):
    r = np.random.default_rng(seed)
    B = np.zeros((k, p), np.float32)
    for c in range(k):
        nz = r.choice(p, size=max(1, p // 4), replace=False)
        B[c, nz] = r.normal(0, 0.05, len(nz))
    return B


@pytest.mark.parametrize("precision", ["split_e4m3", "split_e2m1", "fp64"])
def test_column_shards_sum_to_eta(precision):
    import paper_2010_16114_gb300 as P
    from paper_2010_16114_gb300.cox import CoxProblem
    P.build()
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=3000, p=2500)
    k = 4
    B = _betas(w.p, k, 7)
    split = precision.startswith("split")
    Xin = X if split else Xf
    dt = torch.float32 if split else torch.float64
    kw = {} if split else {"center": True}
    with CoxProblem(Xin, w.y, w.delta, precision=precision, **kw) as full:
        eta_full = full.eta(torch.tensor(B, dtype=dt, device="cuda")).cpu().numpy()
        _, order = full.mu_order()
    eta_sum = np.zeros_like(eta_full)
    for cols in np.array_split(np.arange(w.p), 3):
        Xg = np.ascontiguousarray(Xin[:, cols])
        with CoxProblem(Xg, w.y, w.delta, precision=precision, **kw) as prob:
            eta_sum += prob.eta(torch.tensor(np.ascontiguousarray(B[:, cols]), dtype=dt, device="cuda")).cpu().numpy()
            _, og = prob.mu_order()
            assert np.array_equal(og, order)  # same subjects, same (stable) time order
    scale = (np.abs(Xf) @ np.abs(B.astype(np.float64)).T).max()
    tol = (2.0 ** -15 if split else 1e-12) * scale
    assert np.abs(eta_sum - eta_full).max() <= tol
    for c in range(k):
        eta_o = oracle.eta(Xf, mu, B[c].astype(np.float64))[order]
        assert np.abs(eta_full[c] - eta_o).max() <= tol
        assert np.abs(eta_sum[c] - eta_o).max() <= tol
