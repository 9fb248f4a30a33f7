"""The autotuner: every tunable launch site timed in each variant on a real system; the
context keeps the choices, and solutions stay the same (the variants compute the same
quantities) on the tuned system and on a new analysis of the same shapes."""
import numpy as np
import pytest

from fixtures import lognormal_coefficients, q1_square, rhs_uniform

pytestmark = pytest.mark.gpu

try:
    import paper_1410_2697_gb300 as hm
except ImportError:
    import torch
    if torch.cuda.is_available():
        raise
    pytest.skip("CUDA library not built on this CPU-only machine", allow_module_level=True)


@pytest.mark.parametrize("precision", ["HM_PREC_MIXED", "HM_PREC_FP64"])
def test_autotune_keeps_solutions(precision):
    m = 192
    P = q1_square(m, lognormal_coefficients(m * m, sigma=1.0, mu=0.0, seed=11))
    o = hm.hm_default_opts()
    o.precision = getattr(hm, precision)
    o.n_c = 32
    o.hodlr_leaf = 32
    ctx = hm.hm_create(o)
    b = rhs_uniform(P.n, 4, 12)
    A = P.scipy()

    def solve(s):
        x = np.zeros_like(b)
        info = hm.hm_solve(s, 4, b, 1e-10, 2000, x)
        assert info["converged"] == 1
        for c in range(4):
            assert np.linalg.norm(b[:, c] - A @ x[:, c]) / np.linalg.norm(b[:, c]) <= 1e-10
        return x

    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
    hm.hm_factor(s, P.values, 1e-4)
    x0 = solve(s)
    nsites = hm.hm_autotune(s, P.values, 1e-4, 4, reps=1)
    assert nsites > 10  # GEMM batches, panel QRs and dense apply levels of every tree level
    x1 = solve(s)
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) <= 1e-8
    hm.hm_destroy(s)
    # a new analysis on the tuned context takes the stored choices
    s2 = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
    hm.hm_factor(s2, P.values, 1e-4)
    x2 = solve(s2)
    assert np.linalg.norm(x2 - x0) / np.linalg.norm(x0) <= 1e-8
    hm.hm_destroy(s2)
    hm.hm_ctx_destroy(ctx)


def test_autotune_refuses_while_profiling():
    P = q1_square(32)
    ctx = hm.hm_create(hm.hm_default_opts())
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
    hm.hm_factor(s, P.values, 1e-6)
    hm.hm_profile_enable(ctx, True)
    with pytest.raises(hm.HmError) as e:
        hm.hm_autotune(s, P.values, 1e-6, 1)
    assert e.value.status == hm.abi.HM_ERR_STATE
    hm.hm_profile_enable(ctx, False)
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


@pytest.mark.parametrize("precision", ["HM_PREC_MIXED", "HM_PREC_FP64"])
def test_every_forced_variant_solves(precision):
    """Each launch variant, forced on every site, gives the same solution (the GEMM
    variants add in the same order; QR and apply variants differ in rounding only)."""
    m = 160
    P = q1_square(m, lognormal_coefficients(m * m, sigma=1.0, mu=0.0, seed=13))
    o = hm.hm_default_opts()
    o.precision = getattr(hm, precision)
    o.n_c = 32
    o.hodlr_leaf = 32
    ctx = hm.hm_create(o)
    b = rhs_uniform(P.n, 2, 14)
    A = P.scipy()
    xs = []
    for v in (0, 1, 2, 3, 4):
        hm.hm_tune_force(ctx, v)
        s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
        hm.hm_factor(s, P.values, 1e-4)
        x = np.zeros_like(b)
        info = hm.hm_solve(s, 2, b, 1e-10, 2000, x)
        assert info["converged"] == 1, v
        for c in range(2):
            assert np.linalg.norm(b[:, c] - A @ x[:, c]) / np.linalg.norm(b[:, c]) <= 1e-10, v
        xs.append(x)
        hm.hm_destroy(s)
    for v in (1, 2, 3, 4):
        assert np.linalg.norm(xs[v] - xs[0]) / np.linalg.norm(xs[0]) <= 1e-8, v
    with pytest.raises(hm.HmError):
        hm.hm_tune_force(ctx, 7)
    hm.hm_ctx_destroy(ctx)


def test_hodlr_apply_variants_agree():
    """The HODLR fronts' cluster apply with 512 threads per CTA (variant 4) computes every
    row and every column sum in the same order as with 256 (variant 0): on two identical
    factorizations (both under variant 0) the applies agree to FP32 rounding."""
    m = 160
    P = q1_square(m, lognormal_coefficients(m * m, sigma=1.0, mu=0.0, seed=17))
    o = hm.hm_default_opts()
    o.precision = hm.HM_PREC_MIXED
    o.n_c = 32
    o.hodlr_leaf = 32
    ctx = hm.hm_create(o)
    r = rhs_uniform(P.n, 3, 18)
    zs = []
    for v in (0, 4):
        hm.hm_tune_force(ctx, 0)
        s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
        info = hm.hm_factor(s, P.values, 1e-4)
        assert info["n_hodlr"] > 0
        hm.hm_tune_force(ctx, v)  # the apply plan and its launches are made after this
        z = np.zeros_like(r)
        hm.hm_precond_apply(s, 3, r, z)
        zs.append(z)
        hm.hm_destroy(s)
    hm.hm_tune_force(ctx, -1)
    assert np.linalg.norm(zs[1] - zs[0]) / np.linalg.norm(zs[0]) <= 1e-6
    hm.hm_ctx_destroy(ctx)
