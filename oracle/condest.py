"""Estimate of the spectral condition number of an SPD matrix (FP64).

ORACLE / TEST INFRASTRUCTURE ONLY.

The solution error after GMRES stops at a relative residual ``rtol`` obeys
``||x - x*|| / ||x*|| <= kappa(A) ||b - A x|| / ||b||`` (the paper solves ``A x = b`` with
``A`` SPD, Section 1, to a residual tolerance, Section 3).  This module estimates
``kappa(A) = lambda_max / lambda_min`` so a test can state that bound beside the measured
error:

* ``lambda_max`` is estimated by the Lanczos process (with full reorthogonalisation) on
  ``A``: the largest Ritz value of the tridiagonal matrix approaches it from below (the
  largest Gershgorin row sum ``max_i sum_j |a_ij|`` bounds it from above);
* ``1 / lambda_min = lambda_max(A^{-1})`` is estimated by the same process on ``A^{-1}``,
  applied through an exact solve.
"""
from __future__ import annotations

import numpy as np


def gershgorin_max(A) -> float:
    """Largest Gershgorin bound ``max_i sum_j |a_ij|`` (>= lambda_max for symmetric A)."""
    return float(np.abs(A).sum(axis=1).max())


def lanczos_max(op, n: int, iters: int, seed: int = 0) -> float:
    """Largest Ritz value of ``iters`` Lanczos steps on the symmetric operator ``op``
    (a function of an n-vector), started from a seeded random vector."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.standard_normal(n)
    q /= np.linalg.norm(q)
    Q = [q]
    alpha, beta = [], []
    for j in range(min(iters, n)):
        w = op(Q[j])
        a = float(Q[j] @ w)
        alpha.append(a)
        for v in Q:                      # full reorthogonalisation, twice
            w = w - (v @ w) * v
        for v in Q:
            w = w - (v @ w) * v
        b = float(np.linalg.norm(w))
        if b <= 1e-14 * abs(a) or j == min(iters, n) - 1:
            break
        beta.append(b)
        Q.append(w / b)
    T = np.diag(alpha) + np.diag(beta[:len(alpha) - 1], 1) + np.diag(beta[:len(alpha) - 1], -1)
    return float(np.linalg.eigvalsh(T)[-1])


def kappa_estimate(A, solve, iters: int = 30, seed: int = 0) -> float:
    """``kappa(A)`` ~ the Lanczos estimates of ``lambda_max(A)`` and ``lambda_max(A^{-1})``
    multiplied; ``solve(v)`` must return ``A^{-1} v``."""
    n = A.shape[0]
    return lanczos_max(lambda v: A @ v, n, iters, seed) * lanczos_max(solve, n, iters, seed + 1)
