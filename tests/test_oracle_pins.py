"""Pins for the FP64 oracle against facts fixed outside it.

Each test checks the oracle against a brute-force definition, exact rational
arithmetic, a closed form, a textbook estimator, calculus (finite
differences), optimality conditions, or a library routine -- never against
a retyped copy of its own formula.  Paper references are to arXiv 2010.16114
(Section 5.3 iteration and likelihood, Section 4.2 soft threshold, Section 4.4
power method, Section 6 Breslow ties and stopping rule).
"""
from fractions import Fraction

import numpy as np
import pytest

import synth


def _rng(seed):
    return np.random.default_rng(seed)


def _tiny(n, ties, seed):
    r = _rng(seed)
    if ties:
        y = r.integers(1, max(2, n // 3), size=n).astype(float)
    else:
        y = r.permutation(n).astype(float) + r.random(n) * 0.5
    delta = (r.random(n) < 0.6).astype(np.uint8)
    eta = r.normal(0, 1.0, n)
    return y, delta, eta


# --- risk sets: brute force O(n^2) and exact rationals ----------------------

@pytest.mark.parametrize("ties", [False, True])
@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
def test_sorted_scans_match_bruteforce(orc, n, ties):
    """Section 5.3 W_j / pi_ij by literal double loops == sorted cumsums."""
    for seed in range(4):
        y, delta, eta = _tiny(n, ties, 100 * n + seed)
        W, u, f = orc.risk(y, delta, eta)
        Wb, ub, fb = orc.risk_bruteforce(y, delta, eta)
        np.testing.assert_allclose(W, Wb, rtol=1e-14, atol=0)
        np.testing.assert_allclose(u, ub, rtol=1e-13, atol=1e-15)
        assert abs(f - fb) <= 1e-13 * max(1.0, abs(fb))


def _exact_risk(y, delta):
    """u and f at eta = 0 in exact rationals, from the risk-set definitions."""
    n = len(y)
    W = [Fraction(sum(1 for j in range(n) if y[j] >= y[i])) for i in range(n)]
    u = [sum((Fraction(1) / W[j] for j in range(n) if y[j] <= y[i] and delta[j]), Fraction(0))
         for i in range(n)]
    return W, u


def test_exact_rational_breslow_example(orc):
    """eta = 0 makes every w_i = 1, so W and u are exact rationals; tie groups
    of sizes 1, 3, 2 with mixed events check the Breslow reading."""
    y = np.array([5.0, 2.0, 2.0, 9.0, 2.0, 5.0, 1.0])
    delta = np.array([1, 1, 0, 0, 1, 0, 1], np.uint8)
    W, u, f = orc.risk(y, delta, np.zeros(7))
    We, ue = _exact_risk(list(y), list(delta))
    np.testing.assert_allclose(W, [float(x) for x in We], rtol=1e-15)
    np.testing.assert_allclose(u, [float(x) for x in ue], rtol=1e-15)
    # hand values: times 1 (1 event, 7 at risk), 2 (2 events, 6 at risk), 5 (1 event, 3 at risk)
    assert W[6] == 7 and W[1] == 6 and W[2] == 6 and W[0] == 3 and W[3] == 1
    np.testing.assert_allclose(u[1], 1 / 7 + 2 / 6, rtol=1e-15)
    np.testing.assert_allclose(u[3], 1 / 7 + 2 / 6 + 1 / 3, rtol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_exact_rationals_random_ties(orc, seed):
    r = _rng(seed)
    n = 25
    y = r.integers(1, 6, size=n).astype(float)
    delta = (r.random(n) < 0.5).astype(np.uint8)
    W, u, f = orc.risk(y, delta, np.zeros(n))
    We, ue = _exact_risk(list(y), list(delta))
    np.testing.assert_allclose(W, [float(x) for x in We], rtol=1e-15)
    np.testing.assert_allclose(u, [float(x) for x in ue], rtol=1e-14)


# --- invariants ---------------------------------------------------------------

@pytest.mark.parametrize("ties", [False, True])
def test_sum_u_equals_sum_delta(orc, ties):
    """1^T P delta = 1^T delta for any beta (each event's pi column sums to 1)."""
    for seed in range(5):
        y, delta, eta = _tiny(500, ties, seed)
        _, u, _ = orc.risk(y, delta, 3 * eta)
        assert abs(u.sum() - delta.sum()) <= 1e-11 * max(1, delta.sum())


@pytest.mark.parametrize("ties", [False, True])
def test_subject_permutation_invariance(orc, ties):
    """Relabelling subjects (including the order inside tie groups) permutes
    W and u and leaves the loss unchanged."""
    y, delta, eta = _tiny(300, ties, 7)
    W, u, f = orc.risk(y, delta, eta)
    perm = _rng(8).permutation(300)
    W2, u2, f2 = orc.risk(y[perm], delta[perm], eta[perm])
    np.testing.assert_allclose(W2, W[perm], rtol=1e-12)
    np.testing.assert_allclose(u2, u[perm], rtol=1e-12, atol=1e-14)
    assert abs(f2 - f) <= 1e-12 * abs(f)


def test_shift_invariance(orc):
    """A common shift of eta cancels in w/W and in the partial likelihood."""
    y, delta, eta = _tiny(200, True, 3)
    _, u, f = orc.risk(y, delta, eta)
    _, u2, f2 = orc.risk(y, delta, eta + 37.25)
    np.testing.assert_allclose(u2, u, rtol=1e-12, atol=1e-14)
    assert abs(f2 - f) <= 1e-12 * abs(f)


def test_overflow_guard(orc):
    """eta of order 1e3 would overflow exp() without the max shift."""
    y, delta, eta = _tiny(100, True, 4)
    _, u, f = orc.risk(y, delta, eta + 900.0)
    _, u0, f0 = orc.risk(y, delta, eta)
    assert np.all(np.isfinite(u)) and np.isfinite(f)
    np.testing.assert_allclose(u, u0, rtol=1e-10, atol=1e-13)


# --- closed forms and textbook estimators ------------------------------------

def test_loss_at_zero_distinct_times(orc):
    """f(0) = (1/n) sum_i delta_i log |R_i| with |R_i| = n - rank_i."""
    n = 400
    y, delta, _ = _tiny(n, False, 11)
    rank = np.argsort(np.argsort(y, kind="stable"), kind="stable")
    expect = np.sum(delta * np.log(n - rank)) / n
    _, _, f = orc.risk(y, delta, np.zeros(n))
    assert abs(f - expect) <= 1e-13 * abs(expect)


def test_loss_at_zero_with_ties(orc):
    """With ties |R(t)| is the number at risk at t (Breslow)."""
    n = 400
    y, delta, _ = _tiny(n, True, 12)
    at_risk = np.array([(y >= t).sum() for t in y])
    expect = np.sum(delta * np.log(at_risk)) / n
    _, _, f = orc.risk(y, delta, np.zeros(n))
    assert abs(f - expect) <= 1e-13 * abs(expect)


@pytest.mark.parametrize("ties", [False, True])
def test_u_at_zero_is_nelson_aalen(orc, ties):
    """At beta = 0, u_i is the Nelson-Aalen cumulative hazard at y_i."""
    y, delta, _ = _tiny(600, ties, 13)
    times = np.unique(y)
    d = np.array([delta[y == t].sum() for t in times], float)
    r = np.array([(y >= t).sum() for t in times], float)
    H = np.cumsum(d / r)
    expect = H[np.searchsorted(times, y)]
    _, u, _ = orc.risk(y, delta, np.zeros(len(y)))
    np.testing.assert_allclose(u, expect, rtol=1e-13)


def test_logrank_score_p1(orc):
    """p = 1, beta = 0: n g = sum over events of (x_i - mean of x over R(y_i)),
    the log-rank score (with Breslow ties)."""
    r = _rng(21)
    n = 300
    y = r.integers(1, 60, n).astype(float)
    delta = (r.random(n) < 0.4).astype(np.uint8)
    x = r.integers(0, 3, n).astype(float)
    _, u, _ = orc.risk(y, delta, np.zeros(n))
    g = orc.grad(x[:, None], None, delta, u)[0]
    score = sum(x[i] - x[y >= y[i]].mean() for i in range(n) if delta[i])
    assert abs(n * g - score) <= 1e-11 * max(1, abs(score))


# --- calculus -------------------------------------------------------------------

@pytest.mark.parametrize("center", [False, True])
def test_gradient_central_differences(orc, center):
    """g = -grad f: central differences of the FP64 loss, h = 1e-5."""
    w = synth.workload("geno_100k_50k", n=400, p=12)
    X = w.dense().astype(float)
    mu = X.mean(0) if center else None
    beta = _rng(5).normal(0, 0.3, w.p)
    eta = orc.eta(X, mu, beta)
    _, u, f = orc.risk(w.y, w.delta, eta)
    g = orc.grad(X, mu, w.delta, u)
    h = 1e-5
    fd = np.zeros(w.p)
    for j in range(w.p):
        e = np.zeros(w.p)
        e[j] = h
        fp = orc.risk(w.y, w.delta, orc.eta(X, mu, beta + e))[2]
        fm = orc.risk(w.y, w.delta, orc.eta(X, mu, beta - e))[2]
        fd[j] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(-fd, g, rtol=1e-7, atol=1e-9 * np.abs(g).max())


def test_centering_leaves_loss_unchanged(orc):
    """X_c beta differs from X beta by a constant, which the loss ignores."""
    w = synth.workload("geno_100k_50k", n=300, p=20)
    X = w.dense().astype(float)
    beta = _rng(6).normal(0, 0.2, w.p)
    f_c = orc.risk(w.y, w.delta, orc.eta(X, X.mean(0), beta))[2]
    f_u = orc.risk(w.y, w.delta, orc.eta(X, None, beta))[2]
    assert abs(f_c - f_u) <= 1e-12 * abs(f_u)


# --- optimisation: KKT, monotone objective, Newton root ------------------------

def test_soft_threshold_cases(orc):
    """Section 4.2: strict inequalities, so |x| == t maps to exactly 0."""
    st = orc.soft_threshold
    assert st(3.0, 1.0) == 2.0 and st(-3.0, 1.0) == -2.0
    assert st(1.0, 1.0) == 0.0 and st(-1.0, 1.0) == 0.0 and st(0.5, 1.0) == 0.0
    assert st(0.0, 0.0) == 0.0 and st(2.5, 0.0) == 2.5


def _small_problem(seed=0, n=150, p=30):
    w = synth.workload("geno_100k_50k", n=n, p=p)
    X = w.dense().astype(float)
    mu = X.mean(0)
    return w, X, mu


def test_ista_kkt_and_monotone(orc):
    """ISTA fixed point <=> KKT: |g_j| <= lambda where beta_j = 0 and
    g_j = lambda sign(beta_j) elsewhere; F_lambda never increases."""
    w, X, mu = _small_problem()
    v0 = synth.normal_vec(95376, 7, w.p)
    L = orc.lipschitz(X, mu, v0, tol=1e-10, maxiter=5000)
    lmax = orc.lambda_max(X, mu, w.y, w.delta)
    lam = 0.3 * lmax
    beta = np.zeros(w.p)
    Ftr = []
    for _ in range(200):
        beta_new, F, g = orc.ista(X, mu, w.y, w.delta, 1.0 / L, lam, 200, beta)
        Ftr.extend(F)
        if np.max(np.abs(beta_new - beta)) < 1e-13:
            beta = beta_new
            break
        beta = beta_new
    Ftr = np.array(Ftr)
    assert np.all(np.diff(Ftr) <= 1e-14 * np.abs(Ftr[1:]))
    eta = orc.eta(X, mu, beta)
    _, u, _ = orc.risk(w.y, w.delta, eta)
    g = orc.grad(X, mu, w.delta, u)
    zero = beta == 0
    assert zero.any() and (~zero).any()
    assert np.all(np.abs(g[zero]) <= lam * (1 + 1e-6))
    np.testing.assert_allclose(g[~zero], lam * np.sign(beta[~zero]), rtol=0, atol=1e-6 * lam)


def test_unpenalised_p1_matches_newton(orc):
    """p = 1, lambda = 0: the ISTA limit is the root of the Cox score,
    found here by Newton's method on score and information written from the
    partial likelihood in numpy."""
    r = _rng(31)
    n = 250
    y = r.integers(1, 40, n).astype(float)
    x = r.normal(0, 1, n)
    delta = (r.random(n) < 0.5).astype(np.uint8)
    b = 0.0
    for _ in range(50):
        e = np.exp(b * x)
        U = I = 0.0
        for i in np.nonzero(delta)[0]:
            R = y >= y[i]
            s0, s1, s2 = e[R].sum(), (e[R] * x[R]).sum(), (e[R] * x[R] ** 2).sum()
            U += x[i] - s1 / s0
            I += s2 / s0 - (s1 / s0) ** 2
        b += U / I
    L = 2 * np.sum((x - x.mean()) ** 2) / n
    beta, F, g = orc.ista(x[:, None], x[None, :].mean(1), y, delta, 1.0 / L, 0.0, 20000)
    assert abs(beta[0] - b) <= 1e-9 * max(1, abs(b))


def test_power_method_matches_svd(orc):
    """Section 4.4 power method vs LAPACK's largest singular value."""
    w, X, mu = _small_problem(n=200, p=40)
    v0 = synth.normal_vec(95376, 7, w.p)
    nrm, it = orc.opnorm2(X, mu, v0, tol=1e-12, maxiter=10000)
    ref = np.linalg.norm(X - mu, 2)
    assert abs(nrm - ref) <= 1e-8 * ref
    nrm6, _ = orc.opnorm2(X, mu, v0)  # the paper's defaults: tol 1e-6, 1000 iterations
    assert abs(nrm6 - ref) <= 1e-5 * ref


# --- the oracle's own rounding ------------------------------------------------------

def test_long_double_twin_agrees(orc):
    """The same source carried in long double agrees to ~1e-13: the FP64
    build's summation order is not a source of error at the test sizes."""
    w, X, mu = _small_problem(n=500, p=25)
    beta = _rng(9).normal(0, 0.3, w.p)
    eta = orc.eta(X, mu, beta)
    eta_ld = orc.eta(X, mu, beta, long_double=True)
    np.testing.assert_allclose(eta, eta_ld, rtol=1e-13, atol=1e-14)
    W, u, f = orc.risk(w.y, w.delta, eta)
    Wl, ul, fl = orc.risk(w.y, w.delta, eta_ld, long_double=True)
    np.testing.assert_allclose(u, ul, rtol=1e-12, atol=1e-14)
    assert abs(f - fl) <= 1e-13 * abs(fl)
    g = orc.grad(X, mu, w.delta, u)
    gl = orc.grad(X, mu, w.delta, ul, long_double=True)
    np.testing.assert_allclose(g, gl, rtol=1e-10, atol=1e-13 * np.abs(gl).max())


# --- Section 6: unpenalised covariates, the lambda path, SNP ranking ---------

def _cox_newton_root(x, y, delta, iters=50):
    """Root of the one-covariate Cox score (Breslow risk sets y_j >= y_i) by
    Newton's method on score and information written from the partial
    likelihood in numpy."""
    b = 0.0
    for _ in range(iters):
        e = np.exp(b * x)
        U = I = 0.0
        for i in np.nonzero(delta)[0]:
            R = y >= y[i]
            s0, s1, s2 = e[R].sum(), (e[R] * x[R]).sum(), (e[R] * x[R] ** 2).sum()
            U += x[i] - s1 / s0
            I += s2 / s0 - (s1 / s0) ** 2
        b += U / I
    return b


def _unpen_problem(q=2, seed=41, n=300, p=25):
    w, X, mu = _small_problem(n=n, p=p)
    r = _rng(seed)
    Z = np.column_stack([(r.random(n) < 0.5).astype(float)] + [r.normal(0, 1, n) for _ in range(q - 1)])
    return w, X, mu, Z


def test_unpen_without_block_is_plain_ista(orc):
    w, X, mu = _small_problem()
    lam, sigma = 0.01, 0.05
    b1, F1, _ = orc.ista(X, mu, w.y, w.delta, sigma, lam, 30)
    b2, g2, F2 = orc.ista_unpen(X, mu, None, w.y, w.delta, sigma, lam, 30)
    assert np.array_equal(b1, b2) and np.array_equal(F1, F2) and len(g2) == 0


def test_unpen_block_alone_reaches_the_cox_mle(orc):
    """With the SNPs held at zero by a penalty above lambda_max, the
    unpenalised coefficient converges to the root of its Cox score."""
    r = _rng(32)
    n = 250
    y = r.integers(1, 40, n).astype(float)
    z = r.normal(0, 1, n) + 3.0
    delta = (r.random(n) < 0.5).astype(np.uint8)
    X = r.integers(0, 3, (n, 4)).astype(float)
    b = _cox_newton_root(z, y, delta)
    L = 2 * np.sum((z - z.mean()) ** 2) / n
    beta, gamma, F = orc.ista_unpen(X, X.mean(0), z, y, delta, 1.0 / L, 1e6, 20000)
    assert np.all(beta == 0)
    assert abs(gamma[0] - b) <= 1e-9 * max(1, abs(b))


def test_unpen_block_shift_invariance(orc):
    """The partial likelihood does not see a shift of a covariate column, so
    the iterates do not either (1'(delta - u) = 0)."""
    w, X, mu, Z = _unpen_problem()
    args = (w.y, w.delta, 0.05, 0.02, 40)
    b1, g1, F1 = orc.ista_unpen(X, mu, Z, *args)
    b2, g2, F2 = orc.ista_unpen(X, mu, Z + np.array([3.0, -7.0]), *args)
    np.testing.assert_allclose(b1, b2, rtol=0, atol=1e-11)
    np.testing.assert_allclose(g1, g2, rtol=0, atol=1e-11)
    np.testing.assert_allclose(F1, F2, rtol=1e-12)


def test_unpen_kkt_and_monotone(orc):
    """At the fixed point the unpenalised block is stationary (Z'(delta-u)/n
    = 0) and the SNPs satisfy the lasso KKT conditions; F never increases."""
    w, X, mu, Z = _unpen_problem()
    XZ = np.column_stack([X - mu, Z - Z.mean(0)])
    L = 2 * np.linalg.norm(XZ, 2) ** 2 / w.n
    lam = 0.3 * orc.lambda_max(X, mu, w.y, w.delta)
    beta, gamma, F = orc.ista_unpen(X, mu, Z, w.y, w.delta, 1.0 / L, lam, 60000)
    assert np.all(np.diff(F) <= 1e-14 * np.abs(F[1:]))
    eta = orc.eta(X, mu, beta) + Z @ gamma
    _, u, _ = orc.risk(w.y, w.delta, eta)
    gz = Z.T @ (w.delta - u) / w.n
    gx = orc.grad(X, mu, w.delta, u)
    assert np.max(np.abs(gz)) <= 1e-9
    zero = beta == 0
    assert zero.any() and (~zero).any()
    assert np.all(np.abs(gx[zero]) <= lam * (1 + 1e-6))
    np.testing.assert_allclose(gx[~zero], lam * np.sign(beta[~zero]), rtol=0, atol=1e-6 * lam)


def test_path_stopping_rule(orc):
    """Section 6 rule |F_t - F_{t-lag}| / |F_t + 1| < tol, tested every lag
    iterations once more than lag values exist: above lambda_max F never
    moves, so the rule fires at the first test after 2 lag iterations; with
    tol = 0 every lambda runs max_iter iterations and equals plain ISTA."""
    w, X, mu = _small_problem()
    lmax = orc.lambda_max(X, mu, w.y, w.delta)
    B, G, it = orc.path(X, mu, None, w.y, w.delta, 0.05, [2 * lmax], tol=1e-5, lag=10, max_iter=500)
    assert it[0] == 20 and np.all(B[0] == 0)
    B, G, it = orc.path(X, mu, None, w.y, w.delta, 0.05, [0.4 * lmax, 0.2 * lmax], tol=0.0, lag=10,
                        max_iter=57)
    assert list(it) == [57, 57]
    for l, lam in enumerate([0.4 * lmax, 0.2 * lmax]):
        b, _, _ = orc.ista(X, mu, w.y, w.delta, 0.05, lam, 57)
        assert np.array_equal(B[l], b)


def test_path_warm_and_cold_reach_one_solution(orc):
    """Warm starts change the route, not the (unique, p < events) minimiser:
    run long enough, both paths agree.  (The stopping rule watches F, which
    flattens to rounding level before slow directions of the parameters, such
    as a binary covariate's, have settled; it is no certificate at 1e-7 in
    beta.)  At the paper's tolerance the warm path needs fewer iterations."""
    w, X, mu, Z = _unpen_problem(p=12)
    XZ = np.column_stack([X - mu, Z - Z.mean(0)])
    sigma = 1.0 / (2 * np.linalg.norm(XZ, 2) ** 2 / w.n)
    lmax = orc.lambda_max(X, mu, w.y, w.delta)
    lams = lmax * np.array([0.8, 0.5, 0.3, 0.15])
    Bc, Gc, _ = orc.path(X, mu, Z, w.y, w.delta, sigma, lams, tol=0.0, lag=10, max_iter=30000)
    Bw, Gw, _ = orc.path(X, mu, Z, w.y, w.delta, sigma, lams, tol=0.0, lag=10, max_iter=30000, warm=True)
    np.testing.assert_allclose(Bw, Bc, rtol=0, atol=1e-9)
    np.testing.assert_allclose(Gw, Gc, rtol=0, atol=1e-9)
    _, _, itc = orc.path(X, mu, Z, w.y, w.delta, sigma, lams, tol=1e-5, lag=10, max_iter=30000)
    _, _, itw = orc.path(X, mu, Z, w.y, w.delta, sigma, lams, tol=1e-5, lag=10, max_iter=30000, warm=True)
    assert itw[1:].sum() < itc[1:].sum() and itw[0] == itc[0]


def test_rank_by_entry_hand_example(orc):
    """Largest lambda with a nonzero coefficient first; ties by |beta| at entry,
    then by index; the order of the lambdas given does not matter."""
    lams = np.array([0.3, 0.2, 0.1])
    B = np.array([[0.0, 0.5, 0.0, 0.0, 0.0, 0.0],
                  [0.1, 0.7, -0.3, 0.0, 0.0, 0.1],
                  [0.2, 0.9, -0.4, 0.0, 0.05, 0.0]])
    order, entry = orc.rank_by_entry(lams, B)
    # SNP 1 joins at 0.3; SNPs 2, 0, 5 at 0.2 (|beta| 0.3, then 0.1 and 0.1 by index);
    # SNP 4 at 0.1; SNP 5 leaves again, which does not move its entry; SNP 3 never joins
    assert list(order) == [1, 2, 0, 5, 4]
    assert list(entry) == [1, 0, 1, -1, 2, 1]
    perm = [2, 0, 1]
    order2, entry2 = orc.rank_by_entry(lams[perm], B[perm])
    assert list(order2) == [1, 2, 0, 5, 4]
    assert [perm[e] if e >= 0 else -1 for e in entry2] == list(entry)


# --- the penalised objective and the centring term, by hand ------------------

def test_objective_hand_example(orc):
    """F = f + lambda ||beta||_1 worked by hand (Section 5.3 likelihood, the l1
    penalty of the problem statement).  Two subjects, y = (1, 2), the first an
    event, the second censored; X = [[1, 0], [0, 0]] uncentred; beta =
    (ln 2, -1).  Then eta = (ln 2, 0), w = (2, 1), the event's risk set holds
    both subjects, W = 3, and f = (1/2)(log 3 - ln 2) = (1/2) ln(3/2); with
    lambda = 1/2 the penalty is (1/2)(ln 2 + 1), so F = (1/2) ln 3 + 1/2.
    A dropped or mis-scaled penalty, a wrong sign in |beta|, or a loss without
    the 1/n all move F away from this value."""
    X = np.array([[1.0, 0.0], [0.0, 0.0]])
    y = np.array([1.0, 2.0])
    d = np.array([1, 0], np.uint8)
    beta = np.array([np.log(2.0), -1.0])
    F = orc.objective(X, None, y, d, beta, 0.5)
    assert abs(F - (0.5 * np.log(3.0) + 0.5)) <= 1e-15
    assert abs(orc.objective(X, None, y, d, beta, 0.0) - 0.5 * np.log(1.5)) <= 1e-15
    # ISTA reports F of the iterate entering each iteration: at t = 0 that is beta0
    _, Ftr, _ = orc.ista(X, None, y, d, 0.1, 0.5, 1, beta)
    assert abs(Ftr[0] - (0.5 * np.log(3.0) + 0.5)) <= 1e-15


def test_centred_eta_hand_example(orc):
    """eta = X_c beta with X_c = X - 1 mu^T, by hand in integers: X = [[1, 2],
    [3, 4]], mu = (2, 3), beta = (1, 10) give eta = (-11, 11).  The loss is
    shift-invariant, so only a direct check sees the centring term."""
    X = np.array([[1.0, 2.0], [3.0, 4.0]])
    eta = orc.eta(X, np.array([2.0, 3.0]), np.array([1.0, 10.0]))
    assert list(eta) == [-11.0, 11.0]
    assert list(orc.eta(X, None, np.array([1.0, 10.0]))) == [21.0, 43.0]


def test_byte_column_products_equal_the_float_ones(orc):
    """eta_u8 / grad_u8 (genotype columns held as bytes) are the same loops as
    eta / grad; on the same codes they agree bit for bit, so every pin of the
    float64 products carries over."""
    r = _rng(5)
    n, m = 257, 19
    Xt = r.integers(0, 3, size=(m, n)).astype(np.uint8)
    X = Xt.T.astype(np.float64)
    mu = X.mean(axis=0)
    beta = r.normal(0, 0.3, m)
    delta = (r.random(n) < 0.4).astype(np.uint8)
    u = r.random(n)
    for mm in (mu, None):
        assert np.array_equal(orc.eta_u8(Xt, mm, beta), orc.eta(X, mm, beta))
        assert np.array_equal(orc.grad_u8(Xt, mm, delta, u), orc.grad(X, mm, delta, u))


# --- Section 5.1 NMF: hand examples, theorems, fixed points ------------------

def test_nmf_objective_hand_example(orc):
    """||X - V W||_F^2 by hand: X = [[1, 2], [3, 4]], V = [[1], [1]], W = [[1, 1]]
    leave the residual [[0, 1], [2, 3]], so f = 0 + 1 + 4 + 9 = 14."""
    assert orc.nmf_objective([[1, 2], [3, 4]], [[1], [1]], [[1, 1]]) == 14.0


def test_nmf_one_iteration_by_hand(orc):
    """1 x 1, x = 6, v = 2^0, w = 2, eps = 0.  Multiplicative: v <- v x w / (v w^2)
    = 12 / 4 = 3, then w <- w v x / (v^2 w) with the new v = 36 / 18 = 2 (so the
    W step sees the new V: with the old one it would give 6).  APG: sigma =
    1/(2 w^4) = 1/32, v <- 1 - (4 - 12)/32 = 1.25; tau = 1/(2 v^4) = 256/1250,
    w <- 2 - tau (v^2 w - v x) = 2 + (256/1250)(35/8) = 2.896."""
    V, W = orc.nmf([[6.0]], [[1.0]], [[2.0]], 1, "mult", 0.0)
    assert V[0, 0] == 3.0 and W[0, 0] == 2.0
    V, W = orc.nmf([[6.0]], [[1.0]], [[2.0]], 1, "apg", 0.0)
    assert V[0, 0] == 1.25 and abs(W[0, 0] - 2.896) <= 1e-15


def _nmf_data(m, n, r, seed, scale=1.0):
    rng = _rng(seed)
    return scale * rng.random((m, n)), rng.random((m, r)), rng.random((r, n))


def test_nmf_multiplicative_is_monotone(orc):
    """Lee and Seung's theorem: the multiplicative updates never increase
    ||X - V W||_F^2 (Section 5.1)."""
    X, V, W = _nmf_data(37, 29, 5, 3)
    f = orc.nmf_objective(X, V, W)
    for _ in range(40):
        V, W = orc.nmf(X, V, W, 1, "mult", 1e-12)
        f1 = orc.nmf_objective(X, V, W)
        assert f1 <= f * (1 + 1e-13)
        f = f1
        assert np.all(V >= 0) and np.all(W >= 0)


def test_nmf_apg_is_monotone_and_nonnegative(orc):
    """APG with the Section 5.1 steps: sigma (V W W^T - X W^T) is sigma/2 times the
    gradient in V, and with ||W W^T||_2 >= 1 the step sigma/2 <= 1/(2 ||W W^T||_2)
    is at most the inverse Lipschitz constant, so f cannot increase (likewise for
    W); the projection keeps both factors nonnegative."""
    X, V, W = _nmf_data(40, 31, 4, 5, scale=3.0)
    V, W = 2 * V, 2 * W
    f = orc.nmf_objective(X, V, W)
    for _ in range(30):
        Vn, Wn = orc.nmf(X, V, W, 1, "apg", 1e-12)
        assert np.linalg.norm(W @ W.T, 2) >= 1 and np.linalg.norm(Vn.T @ Vn, 2) >= 1
        V, W = Vn, Wn
        f1 = orc.nmf_objective(X, V, W)
        assert f1 <= f * (1 + 1e-13)
        f = f1
        assert np.all(V >= 0) and np.all(W >= 0)


def test_nmf_exact_factorization_is_a_fixed_point(orc):
    """X = V0 W0 with positive factors: X W0^T = V0 (W0 W0^T) and V0^T X =
    (V0^T V0) W0, so the multiplicative update leaves both factors unchanged
    (eps = 0) and the APG gradients vanish."""
    rng = _rng(7)
    V0, W0 = rng.random((23, 3)) + 0.1, rng.random((3, 19)) + 0.1
    X = V0 @ W0
    for algo in ("mult", "apg"):
        V, W = orc.nmf(X, V0, W0, 3, algo, 0.0)
        np.testing.assert_allclose(V, V0, rtol=1e-12)
        np.testing.assert_allclose(W, W0, rtol=1e-12)


def test_nmf_zeros_stay_zero(orc):
    """A zero entry of V or W is a fixed point of its multiplicative update."""
    X, V, W = _nmf_data(20, 17, 3, 13)
    V[4, 1] = 0.0
    W[2, 9] = 0.0
    V, W = orc.nmf(X, V, W, 50, "mult", 1e-12)
    assert V[4, 1] == 0.0 and W[2, 9] == 0.0 and np.all(V[np.arange(20) != 4] > 0)


def test_nmf_multiplicative_reaches_kkt(orc):
    """From a strictly positive start on an exactly factorizable X the
    multiplicative updates approach a KKT point of the nonnegative problem:
    grad_V f >= 0 and V .* grad_V f = 0 (same for W) up to a tolerance, with the
    gradients 2 (V W - X) W^T and 2 V^T (V W - X) computed here by numpy."""
    rng = _rng(11)
    V0, W0 = rng.random((30, 3)) + 0.2, rng.random((3, 25)) + 0.2
    X = V0 @ W0
    V, W = orc.nmf(X, rng.random((30, 3)) + 0.1, rng.random((3, 25)) + 0.1, 20000, "mult", 1e-15)
    R = V @ W - X
    gV, gW = 2 * R @ W.T, 2 * V.T @ R
    assert orc.nmf_objective(X, V, W) <= 1e-6 * np.sum(X * X)
    tol = 1e-3 * np.abs(X).max() * max(np.abs(V).max(), np.abs(W).max())
    assert gV.min() >= -tol and gW.min() >= -tol
    assert np.abs(V * gV).max() <= tol * np.abs(V).max() and np.abs(W * gW).max() <= tol * np.abs(W).max()
