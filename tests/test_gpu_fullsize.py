"""Parity at the genotype workloads' full sizes, in the launch configuration
the benchmark uses (genotypes generated on the device, 2-bit packed, 256-chunk
accumulation windows; for the 16- and 32-penalty workloads the autotuner's
shapes, as bench.py runs them).

Inputs the two sides share are fixed on the host, never read back from the
GPU: the step sigma = 1 / L_bound with L_bound = (sqrt n + sqrt p)^2 / n, the
Marchenko-Pastur edge of 2 ||X_c||_2^2 / n for near-independent genotype
columns of variance at most 1/2 (so sigma <= 1/L and the iteration is a
descent); the penalties are fractions of the oracle's max |g_j(0)| (over all
columns where the oracle streams X, over 2048 seeded columns elsewhere).

* geno_100k_50k (n=100,000, p=50,000, k=1): 50 whole iterations on both
  sides, the oracle streaming X (bytes per code) in parallel column blocks:
  beta after 50 iterations element by element (relative L2 <= 1e-4, the same
  support outside a 1e-6 threshold margin), g(0) in full, the loss there.
* geno_200k_10k (n=200,000, p=10,000, k=1): two whole iterations and the
  autograd backward at full size.
* geno_400k_100k_k32 (50 iterations, 32 penalties) and geno_400k_500k_k16
  (3 iterations, 16 penalties; in both operand forms of the tensor-core
  products, e4m3 and e2m1): the oracle cannot run whole iterations at
  these sizes, so the checks sit at the nonzero beta the GPU reached.  At it
  the oracle computes eta at 64 sampled subjects for every column (the first
  product over all p SNPs), and, for up to 4 columns whose support it can
  regenerate, eta over all subjects, the loss, the gradient at 64 sampled SNPs
  plus support SNPs, and the next iterate there.  At beta = 0: g_j(0) at 64
  sampled SNPs, the first iterate there and the closed form of the loss,
  f(0) = (1/n) sum_i delta_i log |R_i|.  geno_400k_500k_k16 also checks eta
  for a dense random beta (every one of the 3,907 K chunks contributes).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = max(1, min(32, os.cpu_count() or 1))


def _device_problem(name, **kw):
    import paper_2010_16114_gb300 as P
    from paper_2010_16114_gb300.cox import CoxProblem
    P.build()
    synth.build_device()
    w = synth.workload(name)
    n, p = w.n, w.p
    thr = torch.from_numpy(w.thr.view(np.int32).copy()).cuda()
    packed = torch.empty((n, (p + 3) // 4), dtype=torch.uint8, device="cuda")
    w.packed_rows_device(packed.data_ptr(), torch.cuda.current_stream().cuda_stream, thr.data_ptr())
    torch.cuda.synchronize()
    prob = CoxProblem(packed, w.y, w.delta, p=p, **kw)
    del packed
    torch.cuda.empty_cache()
    return w, prob


def _step(n, p):
    """1 / L_bound: the edge (1 + sqrt(p/n))^2 of the spectrum of X_c^T X_c / n
    for independent columns, times 2 x the largest genotype variance 1/2."""
    return n / (np.sqrt(n) + np.sqrt(p)) ** 2


def _loss_at_zero(w):
    order = np.argsort(w.y, kind="stable")
    ys = w.y[order]
    # |R_i| = number with y >= y_i: n minus the first rank of y_i's tie group
    first = np.searchsorted(ys, w.y, side="left")
    return float(np.sum(w.delta * np.log(w.n - first)) / w.n)


def _par_grad(Xt, mu, delta, u, block=512):
    """oracle.grad_u8 over the columns (rows of Xt), in parallel column blocks:
    each column's sum is the oracle's own, so the result is the whole call's."""
    from concurrent.futures import ThreadPoolExecutor
    m = Xt.shape[0]
    g = np.zeros(m)

    def run(j0):
        j1 = min(m, j0 + block)
        g[j0:j1] = oracle.grad_u8(Xt[j0:j1], mu[j0:j1], delta, u)

    with ThreadPoolExecutor(THREADS) as ex:
        list(ex.map(run, range(0, m, block)))
    return g


def _cols_mu(w, idx):
    Xt = w.cols_u8(idx, threads=THREADS)
    return Xt, Xt.mean(axis=1, dtype=np.float64)


def _ranks(y):
    order = np.argsort(y, kind="stable")
    rank = np.empty(len(y), np.int64)
    rank[order] = np.arange(len(y))
    return rank


# --------------------------------------------------------------- geno_100k_50k
def test_geno_100k_50k_fifty_iterations():
    """n = 100,000 x p = 50,000, lambda = 0.5 lambda_max: 50 iterations on the GPU
    against the oracle's 50 iterates (Section 5.3 iteration, run as the oracle's
    ISTA: eta over the support, the risk-set sums, the gradient over every
    column, the soft-threshold step)."""
    w, prob = _device_problem("geno_100k_50k")
    try:
        n, p = w.n, w.p
        Xt, mu = _cols_mu(w, np.arange(p))  # 5 GB of codes, one byte each
        sigma = _step(n, p)
        _, u0, f0 = oracle.risk(w.y, w.delta, np.zeros(n))
        g0 = _par_grad(Xt, mu, w.delta, u0)
        lmax = float(np.abs(g0).max())
        lam = 0.5 * lmax
        # beta = 0: loss, gradient, lambda_max
        beta = prob.zeros(1)
        loss, grad = prob.loss_grad(beta)
        assert abs(loss[0] - f0) <= 1e-12 * abs(f0)
        assert rel_l2(grad.cpu().numpy()[0].astype(np.float64), -g0) <= 1e-5
        assert abs(prob.lambda_max() - lmax) <= 1e-5 * lmax
        # 50 iterations
        iters = 50
        for _ in range(iters):
            prob.prox_step(beta, [lam], sigma)
        prob.sync()
        Bg = beta.cpu().numpy()[0].astype(np.float64)
        b_o = np.zeros(p)
        for t in range(iters):
            S = np.nonzero(b_o)[0]
            eta = oracle.eta_u8(Xt[S], mu[S], b_o[S]) if len(S) else np.zeros(n)
            _, u, f = oracle.risk(w.y, w.delta, eta)
            g = g0 if t == 0 else _par_grad(Xt, mu, w.delta, u)
            z = b_o + sigma * g
            b_o = oracle.prox(b_o, g, sigma, lam)
        assert np.count_nonzero(b_o) > 0
        amb = np.abs(np.abs(z) - sigma * lam) <= 1e-6
        assert np.all(((Bg != 0) == (b_o != 0)) | amb)
        assert rel_l2(Bg, b_o) <= 1e-4, rel_l2(Bg, b_o)
        # loss and gradient at the GPU's 50th iterate
        S = np.nonzero(Bg)[0]
        eta = oracle.eta_u8(Xt[S], mu[S], Bg[S])
        _, u, f = oracle.risk(w.y, w.delta, eta)
        g = _par_grad(Xt, mu, w.delta, u)
        loss, grad = prob.loss_grad(beta)
        assert abs(loss[0] - f) <= 1e-7 * abs(f)
        assert rel_l2(grad.cpu().numpy()[0].astype(np.float64), -g) <= 1e-5
    finally:
        prob.close()


# ------------------------------------------------- geno_400k_100k_k32, geno_400k_500k_k16
def _lambda_anchor(w, idx, u0):
    """max_j |g_j(0)| over the sampled columns idx (the oracle's): a lower bound
    of lambda_max from which the penalty grid is laid out."""
    Xs, mus = _cols_mu(w, idx)
    return float(np.abs(_par_grad(Xs, mus, w.delta, u0)).max())


def _check_eta_rows(w, prob, beta, rows, rank, gate=1e-4):
    """eta = X_c beta at sampled subjects, up to the common shift (the loss and
    gradient do not see one): the GPU's centred eta against the oracle's X beta
    over all p SNPs at those subjects, each centred over the sample."""
    B = beta.detach().cpu().numpy().astype(np.float64)
    eg = prob.eta(beta).cpu().numpy()[:, rank[rows]]
    Xr = np.ascontiguousarray(w.rows_u8(rows).T)  # p x 64: the "columns" are SNPs
    for c in range(B.shape[0]):
        eo = oracle.eta_u8(Xr, None, B[c])
        dg, do = eg[c] - eg[c].mean(), eo - eo.mean()
        if np.linalg.norm(do) == 0:
            assert np.all(np.abs(dg) <= 1e-12)
            continue
        assert rel_l2(dg, do) <= gate, (c, rel_l2(dg, do))


def _check_at_gpu_beta(w, prob, beta, lams, sigma, rank, max_support=4000, ncols=4):
    """Loss, gradient and next iterate at the GPU's beta for up to `ncols`
    columns whose support the oracle can regenerate in full."""
    B = beta.cpu().numpy().astype(np.float64)
    k = B.shape[0]
    sizes = np.count_nonzero(B, axis=1)
    cand = [c for c in np.argsort(-sizes) if 1 <= sizes[c] <= max_support][:ncols]
    assert cand, f"no column with 1..{max_support} nonzeros: supports {sizes.tolist()}"
    loss, grad = prob.loss_grad(beta)
    G = grad.cpu().numpy().astype(np.float64)
    nxt = beta.clone()
    prob.prox_step(nxt, lams, sigma)
    Bn = nxt.cpu().numpy().astype(np.float64)
    samp = np.unique((w.uniform_vec(17, 64) * w.p).astype(np.int64))
    for c in cand:
        S = np.nonzero(B[c])[0]
        XS, muS = _cols_mu(w, S)
        eta = oracle.eta_u8(XS, muS, B[c, S])
        _, u, f = oracle.risk(w.y, w.delta, eta)
        J = np.unique(np.concatenate([samp, S[:64]]))
        XJ, muJ = _cols_mu(w, J)
        g = _par_grad(XJ, muJ, w.delta, u)
        assert abs(loss[c] - f) <= 1e-7 * abs(f), (c, loss[c], f)
        assert rel_l2(G[c, J], -g) <= 1e-5, (c, rel_l2(G[c, J], -g))
        z = B[c, J] + sigma * g
        b1 = oracle.prox(B[c, J], g, sigma, lams[c])
        # the gradient bar bounds every |dz_j| by 1e-5 sigma ||g_J||; the soft
        # threshold is 1-Lipschitz; beta is stored in FP32
        dz = 1e-5 * sigma * np.linalg.norm(g) + 2.0 ** -22 * np.abs(B[c]).max()
        amb = np.abs(np.abs(z) - sigma * lams[c]) <= max(1e-6, dz)
        assert np.all(((Bn[c, J] != 0) == (b1 != 0)) | amb), c
        assert np.all(np.abs(Bn[c, J] - b1) <= dz + 1e-6 * np.abs(b1)), (c, np.abs(Bn[c, J] - b1).max(), dz)
    return cand


@pytest.mark.parametrize("name,iters,precision", [("geno_400k_100k_k32", 50, "split_e4m3"),
                                                   ("geno_400k_500k_k16", 3, "split_e4m3"),
                                                   ("geno_400k_500k_k16", 3, "split_e2m1")])
def test_full_size_sampled(name, iters, precision):
    w, prob = _device_problem(name, precision=precision)
    try:
        r = w.r
        # the launch configuration bench.py times: the autotuner's shapes for k columns
        tune = prob.autotune(r.k, reps=1)
        want = 3 if precision == "split_e4m3" else 1  # plannable shapes of the k-column class
        assert tune["x_b"]["candidates"] >= want and tune["xt_v"]["candidates"] >= want
        n, p = w.n, w.p
        sigma = _step(n, p)
        rank = _ranks(w.y)
        _, u0, _ = oracle.risk(w.y, w.delta, np.zeros(n))
        # beta = 0: the loss in closed form, g_j(0) at 64 sampled SNPs, lambda_max
        idx = np.unique((w.uniform_vec(13, 64) * p).astype(np.int64))
        Xi, mui = _cols_mu(w, idx)
        g0 = _par_grad(Xi, mui, w.delta, u0)
        beta = prob.zeros(r.k)
        loss, grad = prob.loss_grad(beta)
        assert np.allclose(loss, _loss_at_zero(w), rtol=1e-12, atol=0)
        assert rel_l2(grad.cpu().numpy()[0, idx].astype(np.float64), -g0) <= 1e-5
        lmax = prob.lambda_max()
        assert np.abs(g0).max() <= lmax * (1 + 1e-5)
        anchor = _lambda_anchor(w, np.unique((w.uniform_vec(19, 2048) * p).astype(np.int64)), u0)
        assert anchor <= lmax * (1 + 1e-5)
        lams = anchor * r.lambda_fracs()
        # the first iterate at the sampled SNPs
        prob.prox_step(beta, lams, sigma)
        prob.sync()
        B1 = beta.cpu().numpy()[:, idx].astype(np.float64)
        z = sigma * g0
        dz = 1e-5 * np.linalg.norm(z)
        for c, lam in enumerate(lams):
            b1 = np.array([oracle.soft_threshold(zj, sigma * lam) for zj in z])
            amb = np.abs(np.abs(z) - sigma * lam) <= max(1e-6, dz)
            assert np.all(((B1[c] != 0) == (b1 != 0)) | amb)
            nz = b1 != 0
            if nz.any():
                np.testing.assert_allclose(B1[c][nz], b1[nz], rtol=1e-4, atol=dz)
        # the remaining iterations, then the checks at the GPU's nonzero beta
        for _ in range(iters - 1):
            prob.prox_step(beta, lams, sigma)
        prob.sync()
        assert np.count_nonzero(beta.cpu().numpy()) > 0
        rows = np.unique((w.uniform_vec(23, 64) * n).astype(np.int64))
        _check_eta_rows(w, prob, beta, rows, rank)
        _check_at_gpu_beta(w, prob, beta, lams, sigma, rank)
        if name == "geno_400k_500k_k16":
            # a dense beta: every K chunk of the first product contributes
            rng = np.random.default_rng(7)
            dense = torch.tensor(rng.normal(0, 0.01, (r.k, p)), dtype=torch.float32, device="cuda")
            _check_eta_rows(w, prob, dense, rows, rank)
    finally:
        prob.close()


# --------------------------------------------------------------- geno_200k_10k
def _streamed_grad(w, beta, blocks):
    """Oracle gradient and loss at beta, X streamed in column blocks."""
    n, p = w.n, w.p
    nzc = np.nonzero(beta)[0]
    if len(nzc):
        Xs, mus = _cols_mu(w, nzc)
        eta = oracle.eta_u8(Xs, mus, beta[nzc])
    else:
        eta = np.zeros(n)
    _, u, f = oracle.risk(w.y, w.delta, eta)
    g = np.zeros(p)
    for blk in blocks:
        Xb, mub = _cols_mu(w, blk)
        g[blk] = _par_grad(Xb, mub, w.delta, u)
    return g, f, u, eta


def test_geno_200k_10k_two_full_iterations():
    """n = 200,000 x p = 10,000 at full size: two iterations from beta = 0 at lambda =
    0.5 lambda_max, the oracle streaming X in blocks of 2500 columns."""
    w, prob = _device_problem("geno_200k_10k")
    try:
        n, p = w.n, w.p
        blocks = [np.arange(j, min(j + 2500, p)) for j in range(0, p, 2500)]
        g0, f0, _, _ = _streamed_grad(w, np.zeros(p), blocks)
        lmax = float(np.abs(g0).max())
        assert abs(prob.lambda_max() - lmax) <= 1e-5 * lmax
        lam = 0.5 * lmax
        step = _step(n, p)
        beta = prob.zeros(1)
        loss, grad = prob.loss_grad(beta)
        assert abs(loss[0] - f0) <= 1e-12 * abs(f0)
        assert rel_l2(grad.cpu().numpy()[0], -g0) <= 1e-5
        b_o = np.zeros(p)
        g_o = g0
        for it in range(2):
            prob.prox_step(beta, [lam], step)
            prob.sync()
            z = b_o + step * g_o
            b_o = oracle.prox(b_o, g_o, step, lam)
            Bg = beta.cpu().numpy()[0].astype(np.float64)
            amb = np.abs(np.abs(z) - step * lam) <= 1e-6
            assert np.all(((Bg != 0) == (b_o != 0)) | amb), it
            assert rel_l2(Bg, b_o) <= 1e-4, (it, rel_l2(Bg, b_o))
            g_o, _, _, _ = _streamed_grad(w, b_o, blocks)
    finally:
        prob.close()


def test_geno_200k_10k_autograd_full_size():
    """n = 200,000 x p = 10,000 at full size: the backward of CoxNLL
    (the library's gradient) at 64 seeded coordinates against central
    differences (h = 1e-3) of the FP64 oracle loss, and against the oracle
    gradient over all columns (streamed in blocks of 2500)."""
    from paper_2010_16114_gb300.autograd import cox_nll
    w, prob = _device_problem("geno_200k_10k")
    try:
        n, p = w.n, w.p
        r = np.random.default_rng(2)
        b0 = np.zeros(p)
        nz = r.choice(p, 40, replace=False)
        b0[nz] = r.normal(0, 0.1, 40)
        beta = torch.tensor(b0[None], dtype=torch.float32, device="cuda", requires_grad=True)
        f = cox_nll(beta, prob)
        f.sum().backward()
        g = beta.grad.cpu().numpy()[0].astype(np.float64)
        bf = beta.detach().cpu().numpy()[0].astype(np.float64)
        blocks = [np.arange(j, min(j + 2500, p)) for j in range(0, p, 2500)]
        g_o, f0, _, eta0 = _streamed_grad(w, bf, blocks)
        g_o = -g_o
        assert abs(float(f.detach()[0]) - f0) <= 1e-7 * abs(f0)
        assert rel_l2(g, g_o) <= 1e-5
        coords = np.unique((w.uniform_vec(11, 64) * p).astype(np.int64))
        h, gmax = 1e-3, np.abs(g_o).max()
        Xc, muc = _cols_mu(w, coords)
        for t, j in enumerate(coords):
            xc = Xc[t].astype(np.float64) - muc[t]
            fp = oracle.risk(w.y, w.delta, eta0 + h * xc)[2]
            fm = oracle.risk(w.y, w.delta, eta0 - h * xc)[2]
            fd = (fp - fm) / (2 * h)
            assert abs(g[j] - fd) <= max(1e-4 * abs(fd), 1e-4 * gmax), (j, g[j], fd)
    finally:
        prob.close()
