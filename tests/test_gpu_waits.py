"""Device-side waits give up and report instead of hanging.

Every mbarrier wait in the tensor-core product has a cycle limit; when it
runs out the kernel raises a flag, waits (with its own fixed limit) for its
copies and MMAs in flight, frees its Tensor Memory and returns.  A handle
created with a wait limit of zero makes the first wait that is not already
satisfied run out, so the call reports COX_ERR_TIMEOUT; the device stays
usable afterwards.  No fault, trap or endless loop is involved."""
import numpy as np
import pytest

from helpers import dense_problem, oracle_loss_grad, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_zero_wait_limit_reports_timeout():
    import paper_2010_16114_gb300 as P
    from paper_2010_16114_gb300._lib import COX_ERR_TIMEOUT, CoxError
    from paper_2010_16114_gb300.cox import CoxProblem
    P.build()
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=8192, p=4096)
    beta = torch.zeros((2, w.p), dtype=torch.float32, device="cuda")
    beta[:, ::7] = 0.01
    codes = []
    # the per-tile issue mode: one issuer per row tile
    with CoxProblem(X, w.y, w.delta, wait_limit_s=0.0, tile_m=2, chunks=2, issue=1) as prob:
        for _ in range(3):
            try:
                prob.loss_grad(beta)
                codes.append(0)
            except CoxError as e:
                codes.append(e.code)
    assert COX_ERR_TIMEOUT in codes
    # a normal handle on the same device still computes the right answer
    with CoxProblem(X, w.y, w.delta) as prob:
        loss, grad = prob.loss_grad(beta)
        f_o, g_o = oracle_loss_grad(Xf, mu, w.y, w.delta, beta[0].cpu().numpy().astype(np.float64))
        assert rel_l2(grad.cpu().numpy()[0], g_o) <= 1e-5
