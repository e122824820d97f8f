"""Parity at the genotype workloads' full sizes, in the launch configuration
the benchmark uses (genotypes generated on the device, 2-bit packed, default
tiles).

* geno_200k_10k (n=200,000, p=10,000, k=1): the oracle runs two whole iterations,
  streaming X in column blocks; beta after each iteration and the gradient at
  beta = 0 are compared element by element.
* geno_100k_50k, geno_400k_100k_k32, geno_400k_500k_k16 (up to n=400,000 x
  p=500,000): sampled outputs the oracle
  computes one by one -- g_j(0) and the first iterate beta_j(1) of every
  penalty at 64 seeded columns j -- and the closed form of the loss at
  beta = 0, f(0) = (1/n) sum_i delta_i log |R_i|.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _loss_at_zero(w):
    order = np.argsort(w.y, kind="stable")
    ys = w.y[order]
    # |R_i| = number with y >= y_i: n minus the first rank of y_i's tie group
    first = np.searchsorted(ys, w.y, side="left")
    return float(np.sum(w.delta * np.log(w.n - first)) / w.n)


def _grad0_cols(w, idx):
    """g(0) at columns idx from the oracle: u(0) does not depend on X."""
    _, u0, _ = oracle.risk(w.y, w.delta, np.zeros(w.n))
    Xc = w.cols(idx)
    return oracle.grad(Xc, Xc.mean(axis=0), w.delta, u0)


@pytest.mark.parametrize("name", ["geno_100k_50k", "geno_400k_100k_k32", "geno_400k_500k_k16"])
def test_sampled_first_iteration_full_size(name):
    w, prob = _device_problem(name)
    try:
        r = w.r
        lmax = prob.lambda_max()
        lams = lmax * r.lambda_fracs()
        L = prob.lipschitz(tol=1e-3, maxiter=20)
        step = 1.0 / L
        beta = prob.zeros(r.k)
        loss, grad = prob.loss_grad(beta)
        assert np.allclose(loss, _loss_at_zero(w), rtol=1e-12, atol=0)
        prob.prox_step(beta, lams, step)
        prob.sync()
        idx = np.unique((w.uniform_vec(13, 64) * w.p).astype(np.int64))
        g0 = _grad0_cols(w, idx)
        G = grad.cpu().numpy()[0, idx].astype(np.float64)
        assert rel_l2(G, -g0) <= 1e-5
        # lambda_max is max_j |g_j(0)|: no sampled column may exceed it
        assert np.abs(g0).max() <= lmax * (1 + 1e-5)
        B = beta.cpu().numpy()[:, idx].astype(np.float64)
        z = step * g0
        # the gradient bar bounds every |dz_j| by 1e-5 ||z||_2, and the soft
        # threshold is 1-Lipschitz, so |dbeta_j| <= 1e-5 ||z||_2 as well
        dz = 1e-5 * np.linalg.norm(z)
        for c, lam in enumerate(lams):
            b1 = np.array([oracle.soft_threshold(zj, step * lam) for zj in z])
            amb = np.abs(np.abs(z) - step * lam) <= max(1e-6, dz)
            assert np.all(((B[c] != 0) == (b1 != 0)) | amb)
            nz = b1 != 0
            if nz.any():
                np.testing.assert_allclose(B[c][nz], b1[nz], rtol=1e-4, atol=dz)
    finally:
        prob.close()


def test_geno_200k_10k_two_full_iterations():
    """n = 200,000 x p = 10,000 at full size: two iterations from beta = 0 at lambda =
    0.5 lambda_max, the oracle streaming X in blocks of 500 columns."""
    w, prob = _device_problem("geno_200k_10k")
    try:
        n, p = w.n, w.p
        blocks = [np.arange(j, min(j + 500, p)) for j in range(0, p, 500)]
        # oracle gradient at beta, streaming X
        def oracle_grad(beta):
            nzc = np.nonzero(beta)[0]
            if len(nzc):
                Xs = w.cols(nzc)
                eta = oracle.eta(Xs, Xs.mean(axis=0), beta[nzc])
            else:
                eta = np.zeros(n)
            _, u, f = oracle.risk(w.y, w.delta, eta)
            g = np.zeros(p)
            for blk in blocks:
                Xb = w.cols(blk)
                g[blk] = oracle.grad(Xb, Xb.mean(axis=0), w.delta, u)
            return g, f

        g0, f0 = oracle_grad(np.zeros(p))
        lmax = float(np.abs(g0).max())
        assert abs(prob.lambda_max() - lmax) <= 1e-5 * lmax
        lam = 0.5 * lmax
        L = prob.lipschitz(tol=1e-4, maxiter=100)
        step = 1.0 / L
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
            g_o, _ = oracle_grad(b_o)
    finally:
        prob.close()


def test_geno_200k_10k_autograd_full_size():
    """n = 200,000 x p = 10,000 at full size: the backward of CoxNLL
    (the library's gradient) at 64 seeded coordinates against central
    differences (h = 1e-3) of the FP64 oracle loss, and against the oracle
    gradient over all columns (streamed in blocks of 500)."""
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
        nzc = np.nonzero(bf)[0]
        Xs = w.cols(nzc)
        eta0 = oracle.eta(Xs, Xs.mean(axis=0), bf[nzc])
        _, u0, f0 = oracle.risk(w.y, w.delta, eta0)
        assert abs(float(f.detach()[0]) - f0) <= 1e-7 * abs(f0)
        g_o = np.zeros(p)
        for j0 in range(0, p, 500):
            blk = np.arange(j0, min(j0 + 500, p))
            Xb = w.cols(blk)
            g_o[blk] = -oracle.grad(Xb, Xb.mean(axis=0), w.delta, u0)
        assert rel_l2(g, g_o) <= 1e-5
        coords = np.unique((w.uniform_vec(11, 64) * p).astype(np.int64))
        h, gmax = 1e-3, np.abs(g_o).max()
        for j in coords:
            xj = w.cols(np.array([j]))[:, 0]
            xc = xj - xj.mean()
            fp = oracle.risk(w.y, w.delta, eta0 + h * xc)[2]
            fm = oracle.risk(w.y, w.delta, eta0 - h * xc)[2]
            fd = (fp - fm) / (2 * h)
            assert abs(g[j] - fd) <= max(1e-4 * abs(fd), 1e-4 * gmax), (j, g[j], fd)
    finally:
        prob.close()
