"""The column-sharded iteration's host logic on CPU: two gloo ranks, each a
shard of the SNP columns (Section 5.3 with X split by columns, one all-reduce
of eta per iteration), driven by ShardedCox.  The shards' arithmetic is the
FP64 oracle's (a stand-in object with the library's call names), so the
sharded iterates must equal the oracle's unsharded ISTA up to the order in
which the two shards' parts of eta are added."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from helpers import dense_problem


class OracleShard:
    """A column shard with the library's call names, computed by the oracle."""

    def __init__(self, Xg, mug, y, delta):
        self.Xg, self.mug, self.y, self.delta = Xg, mug, y, delta
        self.f = self.l1 = None

    def eta(self, beta):
        B = beta.numpy()
        return torch.tensor(np.stack([oracle.eta(self.Xg, self.mug, b) for b in B]))

    def prox_step_eta(self, beta, eta, lambdas, step):
        lam = np.broadcast_to(np.asarray(lambdas, dtype=np.float64), (beta.shape[0],))
        f, l1 = [], []
        for c in range(beta.shape[0]):
            _, u, fc = oracle.risk(self.y, self.delta, eta[c].numpy())
            g = oracle.grad(self.Xg, self.mug, self.delta, u)
            b = beta[c].numpy()
            f.append(fc)
            l1.append(float(np.abs(b).sum()))
            beta[c] = torch.from_numpy(oracle.prox(b, g, step, lam[c]))
        self.f, self.l1 = np.array(f), np.array(l1)
        return beta

    def last_loss_l1(self, k):
        return self.f, self.l1


def _rank(rank, world, port, outdir, cols, iters, sigma, lams):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2010_16114_gb300.shard import ShardedCox
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=700, p=90)
    c = cols[rank]
    sh = ShardedCox(OracleShard(Xf[:, c], mu[c], w.y, w.delta))
    beta = torch.zeros((len(lams), len(c)), dtype=torch.float64)
    F = []
    for _ in range(iters):
        sh.step(beta, lams, sigma)
        F.append(sh.objective(lams))
    np.save(os.path.join(outdir, f"beta{rank}.npy"), beta.numpy())
    np.save(os.path.join(outdir, f"F{rank}.npy"), np.array(F))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_iterates_equal_the_unsharded_oracle(orc):
    w, X, Xf, mu = dense_problem("geno_100k_50k", n=700, p=90)
    cols = [np.arange(0, 37), np.arange(37, 90)]
    lmax = oracle.lambda_max(Xf, mu, w.y, w.delta)
    lams = np.array([0.5, 0.2]) * lmax
    sigma, iters = 0.5, 6
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(2, _free_port(), d, cols, iters, sigma, lams), nprocs=2, join=True,
                           start_method="spawn")
        B = np.concatenate([np.load(os.path.join(d, "beta0.npy")), np.load(os.path.join(d, "beta1.npy"))], axis=1)
        F0, F1 = np.load(os.path.join(d, "F0.npy")), np.load(os.path.join(d, "F1.npy"))
    assert np.array_equal(F0, F1)  # every rank sees the same objective
    for c, lam in enumerate(lams):
        b_o, F_o, _ = oracle.ista(Xf, mu, w.y, w.delta, sigma, lam, iters)
        assert np.count_nonzero(b_o) > 0
        np.testing.assert_allclose(B[c], b_o, rtol=1e-10, atol=1e-13)
        np.testing.assert_allclose(F0[:, c], F_o, rtol=1e-12)
