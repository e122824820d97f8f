"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances, stated per result:
  * FP64 path (normal_1k_2k recipe): beta and gradient relative L2 <= 1e-10 (FP64
    sums in a different order than the oracle's).
  * split-e4m3 tensor-core path and FP32 baseline: gradient relative L2 <= 1e-5
    (four e4m3 limbs hold each coefficient to <= 2^-16 relative; FP32
    accumulation), loss relative error <= 1e-7, beta relative L2 <= 1e-4 after
    a fixed number of iterations, identical support outside a 1e-6 threshold
    margin.
Sizes are chosen so the oracle finishes in seconds while n and p span several
128-wide tiles with a ragged tail.
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


def _problem(pkg, X, w, precision, **kw):
    from paper_2010_16114_gb300.cox import CoxProblem
    return CoxProblem(X, w.y, w.delta, precision=precision, **kw)


# ---------------------------------------------------------------- FP64 path
def test_fp64_normal_1k_2k_200_iterations(pkg):
    """The dense normal workload as specified: n=1000, p=2000, lambda = 0.5 lambda_max, step 1/L,
    200 iterations in FP64; beta and gradient within 1e-10 of the oracle."""
    w, X, Xf, mu = dense_problem("normal_1k_2k")
    v0 = synth.normal_vec(95376, 7, w.p)
    L = oracle.lipschitz(Xf, mu, v0)
    lmax = oracle.lambda_max(Xf, mu, w.y, w.delta)
    lam, sigma = 0.5 * lmax, 1.0 / L
    beta_o, F_o, _ = oracle.ista(Xf, mu, w.y, w.delta, sigma, lam, 200)
    with _problem(pkg, Xf, w, "fp64", center=False) as prob:
        assert abs(prob.lambda_max() - lmax) <= 1e-12 * lmax
        beta = prob.zeros(1)
        for _ in range(200):
            prob.prox_step(beta, [lam], sigma)
        prob.sync()
        b = beta.cpu().numpy()[0]
        assert rel_l2(b, beta_o) <= 1e-10
        assert (b != 0).sum() == (beta_o != 0).sum()
        f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, beta_o)
        loss, grad = prob.loss_grad(beta)
        assert abs(loss[0] - f_o) <= 1e-12 * abs(f_o)
        assert rel_l2(grad.cpu().numpy()[0], g_o) <= 1e-10
        Lg = prob.lipschitz(v0)
        assert abs(Lg - L) <= 1e-6 * L


# ---------------------------------------------------------------- genotype paths
GENO_SIZES = [(3000, 700), (1000, 129), (4099, 1500)]


@pytest.fixture(scope="module", params=GENO_SIZES, ids=lambda s: f"n{s[0]}_p{s[1]}")
def geno(request):
    n, p = request.param
    return dense_problem("geno_100k_50k", n=n, p=p)


def _random_betas(p, k, seed):
    r = np.random.default_rng(seed)
    B = np.zeros((k, p))
    for c in range(k):
        nz = r.choice(p, size=max(1, p // (3 + c)), replace=False)
        B[c, nz] = r.normal(0, 0.05, len(nz))
    return B


@pytest.mark.parametrize("precision", ["split_e4m3", "fp32_gemv"])
@pytest.mark.parametrize("k", [1, 3, 16])
def test_loss_grad_geno(pkg, geno, precision, k):
    w, X, Xf, mu = geno
    B = _random_betas(w.p, k, 11 + k)
    with _problem(pkg, X, w, precision) as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        loss, grad = prob.loss_grad(beta)
        G = grad.cpu().numpy()
        for c in range(k):
            bc = beta[c].cpu().numpy().astype(np.float64)  # the FP32 master the GPU saw
            f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, bc)
            assert abs(loss[c] - f_o) <= 1e-7 * abs(f_o), (c, loss[c], f_o)
            assert rel_l2(G[c], g_o) <= 1e-5, (c, rel_l2(G[c], g_o))


@pytest.fixture(scope="module")
def multi_window():
    return dense_problem("geno_100k_50k", n=9100, p=8700)


@pytest.mark.parametrize("k", [3, 16])
def test_loss_grad_multi_window(pkg, multi_window, k):
    """Row groups whose K range spans several accumulation windows (windows of
    16 chunks of 128 forced) in both products, with ragged n and p:
    n = 9100, p = 8700."""
    w, X, Xf, mu = multi_window
    B = _random_betas(w.p, k, 29 + k)
    with _problem(pkg, X, w, "split_e4m3", window=16) as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        loss, grad = prob.loss_grad(beta)
        G = grad.cpu().numpy()
        for c in range(k):
            bc = beta[c].cpu().numpy().astype(np.float64)
            f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, bc)
            assert abs(loss[c] - f_o) <= 1e-7 * abs(f_o), (c, loss[c], f_o)
            assert rel_l2(G[c], g_o) <= 1e-5, (c, rel_l2(G[c], g_o))


def test_prox_whole_and_split_row_groups(pkg):
    """p = 40001 SNPs over n = 3000 subjects: in the X^T V product a CTA's unit
    range holds whole row groups (the step is applied from its own sums) and
    groups cut between CTAs (partials and the last-CTA step); both against the
    oracle for the gradient and one step."""
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=3000, p=40001)
    k = 3
    B = _random_betas(w.p, k, 61)
    with _problem(pkg, X, w, "split_e4m3") as prob:
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


# every compiled pipeline shape (row tiles, K chunks per stage, issue mode) of
# each limb-column class: 1 = one issuer per row tile, 2 = two issuers on
# alternate stages, 3 = one per row tile committing after every second stage
SHAPES = [(k, t, c, 1) for k in (3, 8, 16) for (t, c) in ((2, 2), (2, 1), (1, 2))] + \
         [(32, 2, 1, 1), (32, 1, 2, 1), (32, 1, 1, 1), (32, 2, 2, 1), (20, 2, 2, 1), (64, 1, 1, 1)] + \
         [(16, 2, 3, 1), (10, 2, 3, 1)] + \
         [(3, 2, 2, 2), (8, 2, 2, 2), (16, 2, 2, 2), (32, 1, 2, 2)] + \
         [(3, 2, 2, 3), (16, 2, 2, 3), (16, 2, 1, 3), (32, 2, 1, 3), (64, 1, 1, 3)]


@pytest.mark.parametrize("k,tile_m,chunks,issue", SHAPES, ids=lambda v: str(v))
def test_every_pipeline_shape(pkg, multi_window, k, tile_m, chunks, issue):
    """Each compiled shape, forced through the options, on row groups that span
    several accumulation windows (16 chunks): the gradients of 4 sampled columns."""
    w, X, Xf, mu = multi_window
    B = _random_betas(w.p, k, 41 + k)
    with _problem(pkg, X, w, "split_e4m3", tile_m=tile_m, chunks=chunks, window=16, issue=issue) as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        loss, grad = prob.loss_grad(beta)
        info = prob.info()
        assert (info["tile_m"], info["chunks"], info["issue"], info["issue_xtv"]) == (tile_m, chunks, issue, issue)
        G = grad.cpu().numpy()
        for c in sorted({0, k // 3, (2 * k) // 3, k - 1}):
            bc = beta[c].cpu().numpy().astype(np.float64)
            f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, bc)
            assert abs(loss[c] - f_o) <= 1e-7 * abs(f_o), (c, loss[c], f_o)
            assert rel_l2(G[c], g_o) <= 1e-5, (c, rel_l2(G[c], g_o))


@pytest.mark.parametrize("k", [16, 32])
def test_autotune_choice_is_used_and_exact(pkg, multi_window, k):
    """Every compiled shape and issue mode of both products is timed (k = 32:
    the 128 limb-column shapes, alternating issuers included), the fastest is
    planned, and the result matches the oracle."""
    w, X, Xf, mu = multi_window
    B = _random_betas(w.p, k, 53)
    with _problem(pkg, X, w, "split_e4m3") as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        ref_loss, ref_grad = prob.loss_grad(beta)
        tune = prob.autotune(k, reps=2)
        for prod in ("x_b", "xt_v"):
            t = tune[prod]
            assert t["candidates"] >= 3 and t["ms"] > 0 and t["tile_m"] in (1, 2) and t["chunks"] in (1, 2, 3)
        loss, grad = prob.loss_grad(beta)
        info = prob.info()
        assert (info["tile_m"], info["chunks"], info["stages"]) == \
            (tune["x_b"]["tile_m"], tune["x_b"]["chunks"], tune["x_b"]["stages"])
        G = grad.cpu().numpy()
        for c in (0, 7, k - 1):
            f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, beta[c].cpu().numpy().astype(np.float64))
            assert rel_l2(G[c], g_o) <= 1e-5
            assert abs(loss[c] - f_o) <= 1e-7 * abs(f_o)


@pytest.mark.parametrize("precision", ["split_e4m3", "fp32_gemv"])
def test_prox_iterations_geno(pkg, geno, precision):
    """20 batched iterations for 3 penalties vs the oracle's iterates."""
    w, X, Xf, mu = geno
    v0 = synth.normal_vec(95376, 7, w.p)
    L = oracle.lipschitz(Xf, mu, v0)
    lmax = oracle.lambda_max(Xf, mu, w.y, w.delta)
    lams = np.array([0.8, 0.3, 0.1]) * lmax
    sigma = 1.0 / L
    iters = 20
    with _problem(pkg, X, w, precision) as prob:
        beta = prob.zeros(3)
        for _ in range(iters):
            prob.prox_step(beta, lams, sigma)
        prob.sync()
        Bg = beta.cpu().numpy().astype(np.float64)
        for c, lam in enumerate(lams):
            b_prev, _, g_prev = oracle.ista(Xf, mu, w.y, w.delta, sigma, lam, iters - 1)
            b_o, _, g_last = oracle.ista(Xf, mu, w.y, w.delta, sigma, lam, 1, b_prev)
            z = b_prev + sigma * g_last
            if np.linalg.norm(b_o) == 0:
                assert np.all(Bg[c] == 0)
                continue
            assert rel_l2(Bg[c], b_o) <= 1e-4, (c, rel_l2(Bg[c], b_o))
            assert support_matches(Bg[c], b_o, z, sigma * lam)


def test_lambda_max_and_lipschitz_geno(pkg, geno):
    w, X, Xf, mu = geno
    v0 = synth.normal_vec(95376, 7, w.p)
    L = oracle.lipschitz(Xf, mu, v0)
    lmax = oracle.lambda_max(Xf, mu, w.y, w.delta)
    with _problem(pkg, X, w, "split_e4m3") as prob:
        assert abs(prob.lambda_max() - lmax) <= 1e-5 * lmax
        assert abs(prob.lipschitz(v0) - L) <= 1e-4 * L


# ---------------------------------------------------------------- edge cases
def _edge_case(kind, n=700, p=300):
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=n, p=p)
    y, d = w.y.copy(), w.delta.copy()
    if kind == "all_censored":
        d[:] = 0
    elif kind == "all_events":
        d[:] = 1
    elif kind == "all_tied":
        y[:] = 5.0
    elif kind == "one_event":
        d[:] = 0
        d[np.argmax(y)] = 1
    return w, X, Xf, mu, y, d


@pytest.mark.parametrize("kind", ["all_censored", "all_events", "all_tied", "one_event"])
def test_degenerate_cases(pkg, kind):
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu, y, d = _edge_case(kind)
    B = _random_betas(w.p, 2, 5)
    with CoxProblem(X, y, d, precision="split_e4m3") as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        loss, grad = prob.loss_grad(beta)
        G = grad.cpu().numpy()
        for c in range(2):
            f_o, g_o = oracle_loss_grad(Xf, mu, y, d, beta[c].cpu().numpy().astype(np.float64))
            if np.linalg.norm(g_o) == 0:
                assert np.all(np.abs(G[c]) <= 1e-12)
                assert loss[c] == 0.0
            else:
                # f = (1/n) sum_i delta_i (log W_i - eta_i): a difference of O(|eta|)
                # terms, so its error follows the limb error of eta (~2^-17 of
                # sum_j |x_ij beta_j|), not |f| -- with one event f is nearly zero.
                eta_o = oracle.eta(Xf, mu, beta[c].cpu().numpy().astype(np.float64))
                eta_scale = np.abs(X.astype(np.float64)) @ np.abs(beta[c].cpu().numpy().astype(np.float64))
                atol = 2.0 ** -16 * d.mean() * max(eta_scale.max(), np.abs(eta_o).max())
                assert abs(loss[c] - f_o) <= 1e-7 * abs(f_o) + atol
                assert rel_l2(G[c], g_o) <= 1e-5


def test_single_predictor_and_tiny_n(pkg):
    for n, p in [(1, 1), (2, 1), (5, 3), (130, 1)]:
        w, X, Xf, mu = dense_problem("geno_100k_50k", n=n, p=p)
        d = w.delta.copy()
        d[0] = 1
        from paper_2010_16114_gb300.cox import CoxProblem
        with CoxProblem(X, w.y, d, precision="split_e4m3") as prob:
            beta = torch.full((1, p), 0.3, dtype=torch.float32, device="cuda")
            loss, grad = prob.loss_grad(beta)
            f_o, g_o = oracle_loss_grad(Xf, mu, w.y, d, np.full(p, 0.3))
            assert abs(loss[0] - f_o) <= 1e-7 * max(1.0, abs(f_o))
            assert np.allclose(grad.cpu().numpy()[0], g_o, rtol=1e-5, atol=1e-7)


def test_invalid_code_rejected(pkg):
    from paper_2010_16114_gb300._lib import COX_ERR_CODE3, CoxError
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=200, p=50)
    X = X.copy()
    X[17, 33] = 3
    with pytest.raises(CoxError) as ei:
        CoxProblem(X, w.y, w.delta)
    assert ei.value.code == COX_ERR_CODE3


def test_packed_inputs_match_int8(pkg):
    """Row-major 2-bit input (host and device) gives the same handle as uint8."""
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=1500, p=333)
    pk = w.packed_rows()
    beta = torch.tensor(_random_betas(w.p, 2, 3), dtype=torch.float32, device="cuda")
    with CoxProblem(X, w.y, w.delta) as a:
        la, ga = a.loss_grad(beta)
        mua, oa = a.mu_order()
    with CoxProblem(pk, w.y, w.delta, p=w.p) as b:
        lb, gb = b.loss_grad(beta)
    pkd = torch.from_numpy(pk).cuda()
    with CoxProblem(pkd, w.y, w.delta, p=w.p) as c:
        lc, gc = c.loss_grad(beta)
        muc, oc = c.mu_order()
    assert np.array_equal(la, lb) and np.array_equal(la, lc)
    assert torch.equal(ga, gb) and torch.equal(ga, gc)
    assert np.array_equal(mua, muc) and np.array_equal(oa, oc)
    np.testing.assert_array_equal(mua, Xf.mean(0))


def test_repeatable_bitwise(pkg):
    """Same inputs, same launch: bit-identical loss, gradient and iterates."""
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=3000, p=700)
    with CoxProblem(X, w.y, w.delta) as prob:
        b1 = prob.zeros(4)
        b2 = prob.zeros(4)
        lams = [1e-3, 5e-4, 2e-4, 1e-4]
        for _ in range(5):
            prob.prox_step(b1, lams, 0.5)
        for _ in range(5):
            prob.prox_step(b2, lams, 0.5)
        prob.sync()
        assert torch.equal(b1, b2)


@pytest.mark.parametrize("window", [2, 6, 10])
def test_alternating_issuers_odd_windows(pkg, multi_window, window):
    """Two issuers on alternate stages with windows of 1, 3 or 5 stages (two
    chunks each): windows where one issuer has no stage, or more stages than
    the other, and group ends inside a window (36 stages per row group).  Gradient and one step for 16
    columns against the oracle."""
    w, X, Xf, mu = multi_window
    k = 16
    B = _random_betas(w.p, k, 71 + window)
    with _problem(pkg, X, w, "split_e4m3", tile_m=2, chunks=2, window=window, issue=2) as prob:
        beta = torch.tensor(B, dtype=torch.float32, device="cuda")
        loss, grad = prob.loss_grad(beta)
        G = grad.cpu().numpy()
        for c in (0, 5, 15):
            bc = beta[c].cpu().numpy().astype(np.float64)
            f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, bc)
            assert abs(loss[c] - f_o) <= 1e-7 * abs(f_o), (c, loss[c], f_o)
            assert rel_l2(G[c], g_o) <= 1e-5, (c, rel_l2(G[c], g_o))
