"""The active-set first product (cox_options.active_set): X B over only the SNP
columns where some penalty's coefficient is nonzero (Section 6: the UK Biobank
path selected a few hundred of 470,194 SNPs).  Against the dense product on
the same data and against the oracle; the fallback to the dense copy when the
support is large; and the path fit with the set on."""
import numpy as np
import pytest

import oracle
import synth
from helpers import dense_problem, rel_l2, support_matches

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    import paper_2010_16114_gb300 as P
    P.build()
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=3000, p=1500)
    L = oracle.lipschitz(Xf, mu, synth.normal_vec(95376, 7, w.p))
    lmax = oracle.lambda_max(Xf, mu, w.y, w.delta)
    return w, X, Xf, mu, L, lmax


def test_active_set_matches_dense_and_oracle(data):
    """Large penalties keep the supports small, so every iteration after the
    first streams the active columns only; the set is rebuilt as it grows."""
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu, L, lmax = data
    lams = np.array([0.6, 0.45, 0.35]) * lmax
    sigma, iters = 1.0 / L, 20
    with CoxProblem(X, w.y, w.delta, active_set=True) as pa, CoxProblem(X, w.y, w.delta) as pd:
        ba, bd = pa.zeros(3), pd.zeros(3)
        for _ in range(iters):
            pa.prox_step(ba, lams, sigma)
            pd.prox_step(bd, lams, sigma)
        info = pa.info()
        Ba = ba.cpu().numpy().astype(np.float64)
        Bd = bd.cpu().numpy().astype(np.float64)
    support = np.count_nonzero(np.any(Ba != 0, axis=0))
    assert 0 < support <= info["active_cols"] < w.p // 4
    assert info["active_rebuilds"] >= 2
    for c, lam in enumerate(lams):
        b_prev, _, _ = oracle.ista(Xf, mu, w.y, w.delta, sigma, lam, iters - 1)
        b_o, _, g = oracle.ista(Xf, mu, w.y, w.delta, sigma, lam, 1, b_prev)
        assert rel_l2(Ba[c], Bd[c]) <= 1e-5, (c, rel_l2(Ba[c], Bd[c]))
        assert rel_l2(Ba[c], b_o) <= 1e-4
        assert support_matches(Ba[c], b_o, b_prev + sigma * g, sigma * lam)


def test_large_support_takes_the_dense_copy(data):
    """With a support beyond a quarter of the columns the dense product runs:
    the iterates are then bitwise those of a handle without the active set."""
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu, L, lmax = data
    lams = np.array([0.02, 0.01]) * lmax
    with CoxProblem(X, w.y, w.delta, active_set=True) as pa, CoxProblem(X, w.y, w.delta) as pd:
        ba, bd = pa.zeros(2), pd.zeros(2)
        for _ in range(6):
            pa.prox_step(ba, lams, 1.0 / L)
            pd.prox_step(bd, lams, 1.0 / L)
        assert np.count_nonzero(np.any(ba.cpu().numpy() != 0, axis=0)) > w.p // 4
        assert torch.equal(ba, bd)


def test_path_fit_with_active_set(data):
    """The path fit with the set on (plain launches) stops where the dense fit
    stops and lands on the same coefficients within the split gates."""
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu, L, lmax = data
    lams = np.array([0.7, 0.5]) * lmax
    with CoxProblem(X, w.y, w.delta, active_set=True) as pa, CoxProblem(X, w.y, w.delta) as pd:
        Ba, ita, oba, _ = pa.path_fit(lams, 1.0 / L, max_iter=200, tol=0.0)
        Bd, itd, obd, _ = pd.path_fit(lams, 1.0 / L, max_iter=200, tol=0.0)
        assert list(ita) == list(itd) == [200, 200]
        for c in range(2):
            assert rel_l2(Ba[c].cpu().numpy(), Bd[c].cpu().numpy()) <= 1e-5
            assert abs(oba[c] - obd[c]) <= 1e-7 * abs(obd[c])
