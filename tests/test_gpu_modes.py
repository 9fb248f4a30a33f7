"""The solver's other modes of use: the direct mode (the factorization applied once, then
iterative refinement, no Krylov method) and the accuracy sweep over the compression
tolerance (iterations fall and ranks grow as the tolerance tightens)."""
import numpy as np
import pytest

from fixtures import lognormal_coefficients, q1_square, rhs_uniform
from oracle import dense_mf

pytestmark = pytest.mark.gpu

try:
    import paper_1410_2697_gb300 as hm
except ImportError:
    import torch
    if torch.cuda.is_available():
        raise
    pytest.skip("CUDA library not built on this CPU-only machine", allow_module_level=True)


def small_ctx(precision, leaf=16):
    o = hm.hm_default_opts()
    o.precision = precision
    o.n_c = leaf
    o.hodlr_leaf = leaf
    return hm.hm_create(o)


def test_direct_mode_at_tol0_is_the_exact_solve():
    P = q1_square(48, lognormal_coefficients(48 * 48, sigma=1.0, mu=0.0, seed=41))
    ctx = small_ctx(hm.HM_PREC_FP64)
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
    fi = hm.hm_factor(s, P.values, 0.0)
    assert fi["n_hodlr"] > 0
    b = rhs_uniform(P.n, 2, 42)
    x = np.zeros_like(b)
    info = hm.hm_direct_solve(s, 2, b, 0, x)
    assert info["iters"] == 1 and info["relres"] <= 1e-11
    for c in range(2):
        xs = dense_mf.direct_solve(P.rowptr, P.colidx, P.values, P.coords, b[:, c])
        assert np.linalg.norm(x[:, c] - xs) / np.linalg.norm(xs) <= 1e-9
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


def test_direct_mode_refinement_contracts():
    P = q1_square(96, lognormal_coefficients(96 * 96, sigma=1.0, mu=0.0, seed=43))
    ctx = small_ctx(hm.HM_PREC_MIXED)
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
    hm.hm_factor(s, P.values, 1e-6)
    b = rhs_uniform(P.n, 3, 44)
    A = P.scipy()
    prev = np.inf
    for refine in (0, 1, 2, 4):
        x = np.zeros_like(b)
        info = hm.hm_direct_solve(s, 3, b, refine, x)
        host = max(np.linalg.norm(b[:, c] - A @ x[:, c]) / np.linalg.norm(b[:, c]) for c in range(3))
        assert abs(host - info["relres"]) <= 1e-3 * host + 1e-15  # the device's FP64 residual
        assert info["relres"] < prev
        prev = info["relres"]
    assert prev <= 1e-9
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


def test_accuracy_sweep():
    P = q1_square(128, lognormal_coefficients(128 * 128, sigma=1.0, mu=0.0, seed=45))
    b = rhs_uniform(P.n, 1, 46)
    A = P.scipy()
    its, ranks = [], []
    for tol in (1e-1, 1e-2, 1e-3, 1e-4, 1e-6):
        ctx = small_ctx(hm.HM_PREC_MIXED, leaf=32)
        s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
        fi = hm.hm_factor(s, P.values, tol)
        x = np.zeros_like(b)
        info = hm.hm_solve(s, 1, b, 1e-10, 4000, x)
        assert info["converged"] == 1
        assert np.linalg.norm(b[:, 0] - A @ x[:, 0]) / np.linalg.norm(b[:, 0]) <= 1e-10
        its.append(info["iters"])
        ranks.append(fi["max_rank"])
        hm.hm_destroy(s)
        hm.hm_ctx_destroy(ctx)
    assert all(a >= b_ for a, b_ in zip(its, its[1:])), its      # tighter tolerance, fewer iterations
    assert all(a <= b_ for a, b_ in zip(ranks, ranks[1:])), ranks  # and larger ranks
    assert its[0] > its[-1]
