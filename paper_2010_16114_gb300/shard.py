"""Column-sharded proximal-gradient iteration (arXiv 2010.16114, Section 5.3,
with X split by SNP columns over devices, the layout of the paper's
distributed matrices, and one all-reduce after the product X beta).

Each rank holds a handle on its own columns X_g (same subjects, times and
events on every rank) and its coefficients B_g.  One iteration:

  1. eta_g = (X_g)_c B_g on each rank (cox_eta, k x n doubles, sorted order);
  2. a sum all-reduce of eta over the ranks (NCCL on device tensors, or a
     host-side backend such as gloo on host copies);
  3. on every rank the risk-set scans on the summed eta (the same on each),
     then its own X_g^T V and the soft-threshold step (cox_prox_step_eta).

The penalised objective needs ||B||_1 over all ranks: ``objective`` sums the
ranks' parts.  Host plumbing only: every step of the arithmetic runs in the
handles' CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


class ShardedCox:
    """One rank's part of a column-sharded fit.  ``problem`` is this rank's
    ``CoxProblem`` (or any object with the same ``eta``, ``prox_step_eta`` and
    ``last_loss_l1`` calls); ``group`` a torch.distributed process group (None:
    the default group)."""

    def __init__(self, problem, group=None):
        self.problem = problem
        self.group = group

    def _device_collective(self) -> bool:
        return dist.get_backend(self.group) == "nccl"

    def allreduce(self, t: torch.Tensor) -> torch.Tensor:
        """Sum over the ranks, in place."""
        if t.is_cuda and not self._device_collective():
            h = t.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.SUM, group=self.group)
            t.copy_(h)
        else:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def eta(self, beta: torch.Tensor) -> torch.Tensor:
        """eta = X_c B summed over the ranks, (k, n) float64."""
        eta = self.problem.eta(beta)
        return self.allreduce(eta)

    def step(self, beta: torch.Tensor, lambdas, step: float) -> torch.Tensor:
        """One iteration in place on this rank's coefficients."""
        self.problem.prox_step_eta(beta, self.eta(beta), lambdas, step)
        return beta

    def objective(self, lambdas) -> np.ndarray:
        """F = f + lambda ||B||_1 of the iterate that entered the last step,
        ||B||_1 summed over the ranks."""
        lam = np.atleast_1d(np.asarray(lambdas, dtype=np.float64))
        f, l1 = self.problem.last_loss_l1(len(lam))
        t = torch.tensor(np.asarray(l1, dtype=np.float64))
        if self._device_collective():
            t = t.cuda()
        self.allreduce(t)
        return np.asarray(f) + lam * t.cpu().numpy()
