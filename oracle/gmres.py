"""Right-preconditioned restarted GMRES(m) in FP64.

ORACLE / TEST INFRASTRUCTURE ONLY.

The paper uses the (approximate) multifrontal solve as a preconditioner of GMRES
(Sections 1 and 3; Saad & Schultz's method) and stops at a relative residual
tolerance with an iteration cap of 4000 (results table caption).  This oracle:
``x0 = 0``; Arnoldi with modified Gram-Schmidt on ``A M^{-1}``; Givens rotations for the
Hessenberg least-squares problem; at the end of each cycle (or when the rotated
residual estimate reaches the tolerance) ``x += M^{-1} V y`` and the TRUE relative
residual ``||b - A x|| / ||b||`` decides convergence.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, precond, b: np.ndarray, rtol: float = 1e-10, restart: int = 30,
          max_iters: int = 4000, x0: np.ndarray | None = None):
    """Returns ``(x, info)`` with ``info = {"iters", "relres", "converged", "history"}``."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros(n), {"iters": 0, "relres": 0.0, "converged": True, "history": []}
    iters = 0
    history = []
    r = b - matvec(x)
    relres = float(np.linalg.norm(r)) / bnorm
    while relres > rtol and iters < max_iters:
        beta = float(np.linalg.norm(r))
        V = np.zeros((n, restart + 1))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[:, 0] = r / beta
        j = 0
        while j < restart and iters < max_iters:
            w = matvec(precond(V[:, j]))
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = float(np.dot(V[:, i], w))
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                          # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            iters += 1
            history.append(abs(g[j]) / bnorm)
            if abs(g[j]) / bnorm <= rtol:
                break
        y = np.zeros(j)
        for i in range(j - 1, -1, -1):                  # back substitution R y = g
            y[i] = (g[i] - H[i, i + 1:j] @ y[i + 1:j]) / H[i, i]
        x = x + precond(V[:, :j] @ y)
        r = b - matvec(x)
        relres = float(np.linalg.norm(r)) / bnorm
    return x, {"iters": iters, "relres": relres, "converged": relres <= rtol, "history": history}
