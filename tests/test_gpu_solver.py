"""GPU tests of the solver around the iteration: batched path fit with the
lag-10 stopping rule (Section 6), autograd, checkpoint/resume, and device-side
error reporting.  All through the C ABI; expected values from the oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import dense_problem, oracle_loss_grad, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2010_16114_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


@pytest.fixture(scope="module")
def small():
    w, X, Xf, mu = dense_problem("geno_400k_100k_k32", n=2500, p=400)
    v0 = synth.normal_vec(95376, 7, w.p)
    L = oracle.lipschitz(Xf, mu, v0)
    lmax = oracle.lambda_max(Xf, mu, w.y, w.delta)
    return w, X, Xf, mu, L, lmax


def _oracle_path(Xf, mu, y, d, sigma, lam, max_iter, tol, lag=10):
    """The Section 6 rule on oracle iterates, checked every `lag` iterations.
    Returns (beta, iterations, final F, converged, {t: stopping ratio at t})."""
    beta = np.zeros(Xf.shape[1])
    hist = []
    ratios = {}
    t = 0
    while t < max_iter:
        steps = min(lag, max_iter - t)
        beta, F, _ = oracle.ista(Xf, mu, y, d, sigma, lam, steps, beta)
        hist.extend(F)
        t += steps
        if len(hist) > lag:
            ratios[t] = abs(hist[-1] - hist[-1 - lag]) / abs(hist[-1] + 1)
            if ratios[t] < tol:
                return beta, t, hist[-1], True, ratios
    return beta, t, hist[-1], False, ratios


@pytest.mark.parametrize("precision", ["split_e4m3", "split_e2m1"])
def test_path_fit_matches_oracle_rule(pkg, small, precision):
    """Each column stops where the oracle's rule stops, and its beta and F match
    the oracle's there.  The rule is deterministic given F; the counts may differ
    only where the oracle's stopping ratio lies within the F error of tol, which
    the test then asserts before it compares beta at the oracle's count (from a
    fixed-count run): the beta comparison is never skipped."""
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu, L, lmax = small
    lams = np.array([0.6, 0.25, 0.1]) * lmax
    tol, max_iter = 1e-5, 400
    with CoxProblem(X, w.y, w.delta, precision=precision) as prob:
        beta, iters, obj, conv = prob.path_fit(lams, 1.0 / L, max_iter=max_iter, tol=tol)
        B = beta.cpu().numpy().astype(np.float64)
        for c, lam in enumerate(lams):
            b_o, t_o, F_o, conv_o, ratios = _oracle_path(Xf, mu, w.y, w.delta, 1.0 / L, lam, max_iter, tol)
            t_g = int(iters[c])
            if t_g == t_o:
                assert rel_l2(B[c], b_o) <= 1e-4, (c, rel_l2(B[c], b_o))
                assert abs(obj[c] - F_o) <= 1e-6 * abs(F_o)
                continue
            # a near-tie: the F values the rule compares differ by at most the
            # objective's error (loss 1e-7 relative, as the loss gate), so the ratio
            # moves by at most ~2e-7 |F| / |F + 1| around tol
            t_star = min(t_g, t_o)
            slack = 4e-7 * max(1.0, abs(F_o)) / abs(F_o + 1)
            assert t_star in ratios and abs(ratios[t_star] - tol) <= slack, (c, t_g, t_o, ratios.get(t_star))
            b_fix, it_fix, _, _ = prob.path_fit([lam], 1.0 / L, max_iter=t_o, tol=0.0)
            assert int(it_fix[0]) == t_o
            assert rel_l2(b_fix.cpu().numpy()[0].astype(np.float64), b_o) <= 1e-4


@pytest.mark.parametrize("precision", ["split_e4m3", "split_e2m1"])
def test_batched_columns_equal_solo_runs(pkg, small, precision):
    """A frozen column stops changing, so each column of a batched path fit is
    bit-identical to fitting that penalty alone."""
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu, L, lmax = small
    lams = np.array([0.6, 0.25, 0.1]) * lmax
    with CoxProblem(X, w.y, w.delta, precision=precision) as prob:
        beta, iters, obj, _ = prob.path_fit(lams, 1.0 / L, max_iter=200, tol=1e-5)
        for c, lam in enumerate(lams):
            b1, it1, ob1, _ = prob.path_fit([lam], 1.0 / L, max_iter=200, tol=1e-5)
            assert it1[0] == iters[c]
            assert torch.equal(b1[0], beta[c])
            assert ob1[0] == obj[c]


@pytest.mark.parametrize("precision", ["split_e4m3", "split_e2m1"])
def test_checkpoint_resume_bit_identical(pkg, small, precision):
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu, L, lmax = small
    lams = np.array([0.3, 0.05]) * lmax
    with CoxProblem(X, w.y, w.delta, precision=precision) as prob:
        full, it_full, ob_full, _ = prob.path_fit(lams, 1.0 / L, max_iter=80, tol=0.0)
        part, it_part, _, _ = prob.path_fit(lams, 1.0 / L, max_iter=40, tol=0.0)
        assert list(it_part) == [40, 40]
        blob = prob.get_state()
    with CoxProblem(X, w.y, w.delta, precision=precision) as prob2:
        prob2.set_state(blob)
        beta = prob2.zeros(2)
        res, it_res, ob_res, _ = prob2.path_fit(lams, 1.0 / L, max_iter=80, tol=0.0, beta=beta, warm=2)
        assert list(it_res) == [80, 80]
        assert torch.equal(res, full)
        assert np.array_equal(ob_res, ob_full)


def test_autograd_matches_fd_and_oracle(pkg):
    """geno_200k_10k recipe (scaled): backward of CoxNLL at 64 seeded coordinates vs
    central differences (h = 1e-3) of the FP64 oracle loss, and vs the oracle
    gradient overall."""
    from paper_2010_16114_gb300.autograd import cox_nll
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu = dense_problem("geno_200k_10k", n=20000, p=600)
    r = np.random.default_rng(2)
    b0 = np.zeros(w.p)
    nz = r.choice(w.p, 40, replace=False)
    b0[nz] = r.normal(0, 0.1, 40)
    with CoxProblem(X, w.y, w.delta) as prob:
        beta = torch.tensor(b0[None], dtype=torch.float32, device="cuda", requires_grad=True)
        f = cox_nll(beta, prob)
        f.sum().backward()
        g = beta.grad.cpu().numpy()[0].astype(np.float64)
        bf = beta.detach().cpu().numpy()[0].astype(np.float64)
    f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, bf)
    assert abs(float(f[0]) - f_o) <= 1e-7 * abs(f_o)
    assert rel_l2(g, g_o) <= 1e-5
    coords = synth.Workload(synth.WORKLOADS["geno_200k_10k"].scaled(n=20000, p=600)).uniform_vec(11, 64)
    coords = np.unique((coords * w.p).astype(int))
    h = 1e-3
    gmax = np.abs(g_o).max()
    for j in coords:
        e = np.zeros(w.p)
        e[j] = h
        fp = oracle.risk(w.y, w.delta, oracle.eta(Xf, mu, bf + e))[2]
        fm = oracle.risk(w.y, w.delta, oracle.eta(Xf, mu, bf - e))[2]
        fd = (fp - fm) / (2 * h)
        assert abs(g[j] - fd) <= max(1e-4 * abs(fd), 1e-4 * gmax), (j, g[j], fd)


def test_nonfinite_is_reported(pkg):
    from paper_2010_16114_gb300._lib import COX_ERR_NONFINITE, CoxError
    from paper_2010_16114_gb300.cox import CoxProblem
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=600, p=200)
    with CoxProblem(X, w.y, w.delta) as prob:
        beta = torch.full((1, w.p), 3e37, dtype=torch.float32, device="cuda")
        beta[0, ::2] = -3e37
        with pytest.raises(CoxError) as ei:
            prob.loss_grad(beta)
        assert ei.value.code == COX_ERR_NONFINITE
        ok = torch.zeros((1, w.p), dtype=torch.float32, device="cuda")
        loss, _ = prob.loss_grad(ok)  # the handle stays usable
        assert np.isfinite(loss[0])
