"""GPU parity of the e2m1 operand form of the tensor-core products
(COX_SPLIT_E2M1: kind::mxf4 with unit block scales, codes as e2m1 nibbles, eight
e2m1 limbs per coefficient) against the FP64 oracle, through the C ABI.

Tolerances, as for the e4m3 form: eight limbs on the grid of halves hold each
coefficient to within 2^-23 of its column's largest magnitude, the products of
codes and limbs and their sums over an accumulation window are exact in FP32, so
the gradient is within relative L2 1e-5, the loss within 1e-7, beta within 1e-4
after a fixed number of iterations, with identical support outside a 1e-6
threshold margin.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import dense_problem, oracle_loss_grad, rel_l2, support_matches

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2010_16114_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


def _problem(X, w, **kw):
    from paper_2010_16114_gb300.cox import CoxProblem
    return CoxProblem(X, w.y, w.delta, precision="split_e2m1", **kw)


def _random_betas(p, k, seed):
    r = np.random.default_rng(seed)
    B = np.zeros((k, p))
    for c in range(k):
        nz = r.choice(p, size=max(1, p // (3 + c)), replace=False)
        B[c, nz] = r.normal(0, 0.05, len(nz))
    return B


def _check_loss_grad(prob, w, Xf, mu, B, cols):
    beta = torch.tensor(B, dtype=torch.float32, device="cuda")
    loss, grad = prob.loss_grad(beta)
    G = grad.cpu().numpy()
    for c in cols:
        bc = beta[c].cpu().numpy().astype(np.float64)
        f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, bc)
        assert abs(loss[c] - f_o) <= 1e-7 * abs(f_o), (c, loss[c], f_o)
        assert rel_l2(G[c], g_o) <= 1e-5, (c, rel_l2(G[c], g_o))


@pytest.fixture(scope="module", params=[(3000, 700), (1000, 129), (4099, 1500)],
                ids=lambda s: f"n{s[0]}_p{s[1]}")
def geno(request):
    n, p = request.param
    return dense_problem("geno_100k_50k", n=n, p=p)


@pytest.mark.parametrize("k", [1, 3, 9, 16])
def test_e2m1_loss_grad_geno(pkg, geno, k):
    w, X, Xf, mu = geno
    B = _random_betas(w.p, k, 11 + k)
    with _problem(X, w) as prob:
        _check_loss_grad(prob, w, Xf, mu, B, range(k))


@pytest.fixture(scope="module")
def multi_window():
    return dense_problem("geno_100k_50k", n=9100, p=8700)


# every compiled e2m1 shape: (k, row tiles, K chunks per stage) over the 64-
# and 128-column limb classes
SHAPES4 = [(3, 2, 2), (8, 1, 4), (16, 2, 2), (5, 1, 4)]


@pytest.mark.parametrize("k,tile_m,chunks", SHAPES4, ids=lambda v: str(v))
def test_e2m1_every_pipeline_shape(pkg, multi_window, k, tile_m, chunks):
    """Each compiled e2m1 shape on row groups spanning several accumulation
    windows (16 chunks forced) in both products, ragged n = 9100, p = 8700."""
    w, X, Xf, mu = multi_window
    B = _random_betas(w.p, k, 41 + k)
    with _problem(X, w, tile_m=tile_m, chunks=chunks, window=16, issue=1) as prob:
        _check_loss_grad(prob, w, Xf, mu, B, sorted({0, k // 3, (2 * k) // 3, k - 1}))
        info = prob.info()
        assert (info["tile_m"], info["chunks"], info["issue"]) == (tile_m, chunks, 1)


def test_e2m1_default_windows(pkg, multi_window):
    """The default 256-chunk accumulation windows (one window per row group here)."""
    w, X, Xf, mu = multi_window
    B = _random_betas(w.p, 16, 7)
    with _problem(X, w) as prob:
        _check_loss_grad(prob, w, Xf, mu, B, [0, 5, 10, 15])


def test_e2m1_prox_whole_and_split_row_groups(pkg):
    """p = 40001 over n = 3000: the X^T V product's row groups run whole in one
    CTA (step from its own sums) and cut between CTAs (partials, last-CTA step)."""
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=3000, p=40001)
    k = 3
    B = _random_betas(w.p, k, 61)
    with _problem(X, w) as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        loss, grad = prob.loss_grad(beta)
        G = grad.cpu().numpy()
        step, lam = 0.05, 1e-4
        prob.prox_step(beta, [lam] * k, step)
        Bn = beta.cpu().numpy().astype(np.float64)
        for c in range(k):
            bc = B[c].astype(np.float32).astype(np.float64)
            f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, bc)
            assert rel_l2(G[c], g_o) <= 1e-5, (c, rel_l2(G[c], g_o))
            z = bc - step * g_o
            b1 = np.sign(z) * np.maximum(np.abs(z) - step * lam, 0.0)
            dz = 1e-5 * step * np.linalg.norm(g_o)
            amb = np.abs(np.abs(z) - step * lam) <= max(1e-6, dz)
            assert np.all(((Bn[c] != 0) == (b1 != 0)) | amb)
            np.testing.assert_allclose(Bn[c], b1, rtol=1e-4, atol=dz + 1e-7 * np.abs(bc).max())


def test_e2m1_iterations_match_oracle(pkg, geno):
    """20 batched iterations for 3 penalties against the oracle's iterates: beta
    relative L2 <= 1e-4, same support outside the threshold margin."""
    w, X, Xf, mu = geno
    v0 = synth.normal_vec(95376, 7, w.p)
    L = oracle.lipschitz(Xf, mu, v0)
    lmax = oracle.lambda_max(Xf, mu, w.y, w.delta)
    lams = np.array([0.8, 0.3, 0.1]) * lmax
    sigma = 1.0 / L
    iters = 20
    with _problem(X, w) as prob:
        beta = prob.zeros(3)
        for _ in range(iters):
            prob.prox_step(beta, lams, sigma)
        prob.sync()
        Bg = beta.cpu().numpy().astype(np.float64)
    for c, lam in enumerate(lams):
        b_prev, _, _ = oracle.ista(Xf, mu, w.y, w.delta, sigma, lam, iters - 1)
        b_o, _, g_last = oracle.ista(Xf, mu, w.y, w.delta, sigma, lam, 1, b_prev)
        z = b_prev + sigma * g_last
        if np.linalg.norm(b_o) == 0:
            assert np.all(Bg[c] == 0)
            continue
        assert rel_l2(Bg[c], b_o) <= 1e-4, (c, rel_l2(Bg[c], b_o))
        assert support_matches(Bg[c], b_o, z, sigma * lam)


def test_e2m1_agrees_with_e4m3(pkg, multi_window):
    """The two operand forms on one data set: gradients within the split gate of
    each other, and switching forms on a handle (cox_set_precision) replans."""
    w, X, Xf, mu = multi_window
    B = _random_betas(w.p, 16, 5)
    beta = torch.tensor(B, dtype=torch.float32, device="cuda")
    from paper_2010_16114_gb300.cox import CoxProblem
    with CoxProblem(X, w.y, w.delta, precision="split_e4m3") as prob:
        l4, g4 = prob.loss_grad(beta)
        g4 = g4.cpu().numpy()
        prob.set_precision("split_e2m1")
        l2, g2 = prob.loss_grad(beta)
        g2 = g2.cpu().numpy()
    for c in range(16):
        assert rel_l2(g2[c], g4[c]) <= 2e-5
        assert abs(l2[c] - l4[c]) <= 2e-7 * abs(l4[c])


def test_e2m1_active_set_matches_dense(pkg):
    """The active-set X B on the e2m1 form: sparse beta, the gathered copy of the
    active SNPs against the dense product and the oracle."""
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=3000, p=20000)
    k = 4
    r = np.random.default_rng(3)
    B = np.zeros((k, w.p))
    for c in range(k):
        nz = r.choice(w.p, size=300, replace=False)
        B[c, nz] = r.normal(0, 0.05, 300)
    with _problem(X, w, active_set=True) as prob:
        _check_loss_grad(prob, w, Xf, mu, B, range(k))
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        prob.prox_step(beta, [1e-4] * k, 0.05)
        ba = beta.cpu().numpy()
    with _problem(X, w) as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        prob.prox_step(beta, [1e-4] * k, 0.05)
        bd = beta.cpu().numpy()
    for c in range(k):
        assert rel_l2(ba[c], bd[c]) <= 1e-5
