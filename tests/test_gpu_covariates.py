"""GPU parity of the Section 6 workflow: unpenalised covariates (sex and
principal components enter the UK Biobank model without a penalty), the
lambda path run one penalty after another from the previous solution, and
the SNP ranking by entry lambda on that path's output.  Expected values from
the oracle (orc_ista_unpen, orc_path, orc_rank_by_entry), all through the C
ABI.

Tolerances as the other parity tests: beta relative L2 <= 1e-4 after a fixed
number of iterations with the same support outside a 1e-6 threshold margin;
gamma (FP64 arithmetic on an FP32-accurate V) relative L2 <= 1e-5; loss 1e-7
relative; gradients 1e-5 relative L2.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import dense_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2010_16114_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


@pytest.fixture(scope="module")
def data():
    """The genotype recipe at n = 3000, p = 400 with q = 3 covariates: a sex
    indicator and two principal-component-like scores."""
    w, X, Xf, mu = dense_problem("geno_400k_500k_k16", n=3000, p=400)
    n = w.n
    Z = np.column_stack([(w.uniform_vec(31, n) < 0.5).astype(np.float64),
                         w.normal_vec(32, n), 0.5 * w.normal_vec(33, n)])
    v0 = synth.normal_vec(95376, 7, w.p)
    L = oracle.lipschitz(Xf, mu, v0)
    lmax = oracle.lambda_max(Xf, mu, w.y, w.delta)
    return w, X, Xf, mu, Z, L, lmax


def _problem(X, w, Z, **kw):
    from paper_2010_16114_gb300.cox import CoxProblem
    prob = CoxProblem(X, w.y, w.delta, **kw)
    prob.set_covariates(Z)
    return prob


@pytest.mark.parametrize("precision", ["split_e4m3", "split_e2m1", "fp32_gemv"])
def test_loss_and_gradients_with_covariates(pkg, data, precision):
    w, X, Xf, mu, Z, L, lmax = data
    r = np.random.default_rng(4)
    k = 2
    B = np.zeros((k, w.p))
    for c in range(k):
        nz = r.choice(w.p, 30, replace=False)
        B[c, nz] = r.normal(0, 0.05, 30)
    G = r.normal(0, 0.3, (k, Z.shape[1]))
    with _problem(X, w, Z, precision=precision) as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        prob.set_gamma(G, k)
        loss, grad = prob.loss_grad(beta)
        gg = prob.grad_gamma(k)
        assert np.array_equal(prob.gamma(k), G)  # a gradient evaluation leaves gamma alone
        Bg = grad.cpu().numpy().astype(np.float64)
        for c in range(k):
            bc = beta[c].cpu().numpy().astype(np.float64)
            eta = oracle.eta(Xf, mu, bc) + oracle.eta(Z, None, G[c])
            _, u, f = oracle.risk(w.y, w.delta, eta)
            assert abs(loss[c] - f) <= 1e-7 * abs(f), (c, loss[c], f)
            assert rel_l2(Bg[c], -oracle.grad(Xf, mu, w.delta, u)) <= 1e-5
            assert rel_l2(gg[c], -oracle.grad(Z, None, w.delta, u)) <= 1e-5


@pytest.mark.parametrize("precision", ["split_e4m3", "split_e2m1", "fp32_gemv"])
def test_iterations_with_covariates_match_oracle(pkg, data, precision):
    """20 batched iterations for 3 penalties: beta thresholded, gamma a plain
    gradient step (orc_ista_unpen)."""
    w, X, Xf, mu, Z, L, lmax = data
    lams = np.array([0.6, 0.25, 0.1]) * lmax
    sigma, iters = 0.5 / L, 20
    with _problem(X, w, Z, precision=precision) as prob:
        beta = prob.zeros(3)
        for _ in range(iters):
            prob.prox_step(beta, lams, sigma)
        prob.sync()
        Bg = beta.cpu().numpy().astype(np.float64)
        Gg = prob.gamma(3)
        F_last = prob.last_objective(3)
    for c, lam in enumerate(lams):
        b_o, g_o, F_o = oracle.ista_unpen(Xf, mu, Z, w.y, w.delta, sigma, lam, iters)
        assert rel_l2(Gg[c], g_o) <= 1e-5, (c, Gg[c], g_o)
        assert abs(F_last[c] - F_o[-1]) <= 1e-6 * abs(F_o[-1])
        if np.linalg.norm(b_o) == 0:
            assert np.all(Bg[c] == 0)
        else:
            assert rel_l2(Bg[c], b_o) <= 1e-4, (c, rel_l2(Bg[c], b_o))


def test_sequential_warm_path_and_ranking(pkg, data):
    """Five penalties from 0.9 to 0.05 lambda_max, each 40 iterations from the
    previous solution (tol = 0: the count is fixed, so no stopping-rule tie can
    split the two sides), with the covariate block; then the SNP ranking of
    Section 6 on the GPU path's coefficients against the oracle's ranking of
    its own path."""
    from paper_2010_16114_gb300.cox import rank_by_entry
    w, X, Xf, mu, Z, L, lmax = data
    lams = lmax * np.exp(np.linspace(np.log(0.9), np.log(0.05), 5))
    sigma, iters = 0.5 / L, 40
    with _problem(X, w, Z) as prob:
        B, G, it, obj, conv = prob.path_seq(lams, sigma, max_iter=iters, tol=0.0, warm=True)
        Bg = B.cpu().numpy().astype(np.float64)
    assert list(it) == [iters] * len(lams) and not conv
    B_o, G_o, it_o = oracle.path(Xf, mu, Z, w.y, w.delta, sigma, lams, tol=0.0, lag=10, max_iter=iters, warm=True)
    assert list(it_o) == [iters] * len(lams)
    for l in range(len(lams)):
        assert rel_l2(G[l], G_o[l]) <= 1e-5, (l, G[l], G_o[l])
        if np.linalg.norm(B_o[l]) == 0:
            assert np.all(Bg[l] == 0)
        else:
            assert rel_l2(Bg[l], B_o[l]) <= 1e-4, (l, rel_l2(Bg[l], B_o[l]))
    # ranking: entry lambda per SNP where the support is unambiguous on both sides
    order_g, entry_g = rank_by_entry(lams, B)
    order_o, entry_o = oracle.rank_by_entry(lams, B_o)
    scale = np.abs(B_o).max()
    clear = np.all((B_o == 0) | (np.abs(B_o) > 1e-4 * scale), axis=0) & \
        np.all((Bg == 0) | (np.abs(Bg) > 1e-4 * scale), axis=0)
    assert clear.sum() >= 0.9 * w.p
    assert np.array_equal(entry_g[clear], entry_o[clear])
    assert len(order_g) > 0
    # ranked SNPs come in order of their entry lambda (largest first)
    assert np.all(np.diff(lams[entry_g[order_g]]) <= 0)


def test_cold_path_equals_batched_columns(pkg, data):
    """Without warm starts each penalty of the sequential path starts from zero,
    like a column of the batched path fit (fixed counts)."""
    w, X, Xf, mu, Z, L, lmax = data
    lams = np.array([0.5, 0.2]) * lmax
    with _problem(X, w, Z) as prob:
        B, G, it, _, _ = prob.path_seq(lams, 0.5 / L, max_iter=30, tol=0.0, warm=False)
        Bb, itb, _, _ = prob.path_fit(lams, 0.5 / L, max_iter=30, tol=0.0)
        Gb = prob.gamma(2)
    assert list(it) == list(itb) == [30, 30]
    assert torch.equal(B, Bb)
    assert np.array_equal(G, Gb)


def test_checkpoint_resume_with_covariates(pkg, data):
    w, X, Xf, mu, Z, L, lmax = data
    lams = np.array([0.3, 0.05]) * lmax
    with _problem(X, w, Z) as prob:
        full, it_full, ob_full, _ = prob.path_fit(lams, 0.5 / L, max_iter=60, tol=0.0)
        g_full = prob.gamma(2)
        prob.path_fit(lams, 0.5 / L, max_iter=30, tol=0.0)
        blob = prob.get_state()
    with _problem(X, w, Z) as prob2:
        prob2.set_state(blob)
        res, it_res, ob_res, _ = prob2.path_fit(lams, 0.5 / L, max_iter=60, tol=0.0, beta=prob2.zeros(2), warm=2)
        assert list(it_res) == [60, 60]
        assert torch.equal(res, full)
        assert np.array_equal(prob2.gamma(2), g_full)
        assert np.array_equal(ob_res, ob_full)
