"""Shared helpers for the parity tests: oracle runs on synth inputs."""
from __future__ import annotations

import numpy as np

import oracle
import synth


def dense_problem(name: str, n: int | None = None, p: int | None = None):
    """(workload, X float64 (n, p), mu or None) for workload recipe `name` at given sizes."""
    w = synth.workload(name, **({} if n is None and p is None else {"n": n, "p": p}))
    X = w.dense()
    Xf = X.astype(np.float64)
    mu = Xf.mean(axis=0) if w.r.center else None
    return w, X, Xf, mu


def oracle_loss_grad(Xf, mu, y, delta, beta):
    """f(beta) and grad f = -g from the oracle."""
    eta = oracle.eta(Xf, mu, beta)
    _, u, f = oracle.risk(y, delta, eta)
    g = oracle.grad(Xf, mu, delta, u)
    return f, -g


def oracle_iterates(Xf, mu, y, delta, sigma, lam, iters, beta0=None):
    beta, F, g = oracle.ista(Xf, mu, y, delta, sigma, lam, iters, beta0)
    return beta, F


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(a - b)
    nb = np.linalg.norm(b)
    return d / nb if nb > 0 else d


def support_matches(beta_gpu, beta_orc, z_orc, thr, margin=1e-6):
    """Identical support except where the oracle's pre-threshold value lies
    within `margin` of the threshold."""
    amb = np.abs(np.abs(z_orc) - thr) <= margin
    s_g = beta_gpu != 0
    s_o = beta_orc != 0
    return bool(np.all((s_g == s_o) | amb))
