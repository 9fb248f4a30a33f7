"""Edge cases and error behaviour through the C ABI: the smallest systems, the largest
right-hand-side block, zero right-hand sides, refactorization with new values,
indefinite matrices, calls out of order and invalid arguments."""
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


def ctx(precision=None, **kw):
    o = hm.hm_default_opts()
    if precision is not None:
        o.precision = precision
    for k, v in kw.items():
        setattr(o, k, v)
    return hm.hm_create(o)


@pytest.mark.parametrize("m", [2, 3, 5])
@pytest.mark.parametrize("precision", ["HM_PREC_FP64", "HM_PREC_MIXED"])
def test_smallest_systems(m, precision):
    """One unknown (m = 2), then a few: the solve is the exact inverse."""
    P = q1_square(m, lognormal_coefficients(m * m, 1.0, seed=90 + m))
    c = ctx(getattr(hm, precision))
    s = hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 2, P.coords)
    hm.hm_factor(s, P.values, 1e-6)
    b = rhs_uniform(P.n, 3, 91)
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 3, b, 1e-10, 100, x)
    assert info["converged"] == 1
    np.testing.assert_allclose(x, np.linalg.solve(P.scipy().toarray(), b), rtol=1e-9, atol=1e-12)
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(c)


def test_largest_rhs_block_and_zero_columns():
    """64 right-hand sides (the limit) in one call equal the same columns solved alone;
    a zero right-hand side gives x = 0 at once; 65 is refused."""
    P = q1_square(48, lognormal_coefficients(48 * 48, 1.0, seed=92))
    c = ctx(hm.HM_PREC_MIXED, n_c=16, hodlr_leaf=16)
    s = hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 2, P.coords)
    hm.hm_factor(s, P.values, 1e-4)
    b = rhs_uniform(P.n, 64, 93)
    b[:, 5] = 0.0
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 64, b, 1e-10, 2000, x)
    assert info["converged"] == 1
    assert np.all(x[:, 5] == 0.0)
    A = P.scipy()
    for col in (0, 31, 63):
        x1 = np.zeros((P.n, 1))
        hm.hm_solve(s, 1, np.ascontiguousarray(b[:, col:col + 1]), 1e-10, 2000, x1)
        assert np.linalg.norm(b[:, col] - A @ x[:, col]) <= 1e-10 * np.linalg.norm(b[:, col])
        assert np.linalg.norm(x1[:, 0] - x[:, col]) <= 1e-8 * np.linalg.norm(x1[:, 0])
    with pytest.raises(hm.HmError) as e:
        hm.hm_solve(s, 65, np.zeros((P.n, 65)), 1e-10, 10, np.zeros((P.n, 65)))
    assert e.value.status == hm.abi.HM_ERR_INVALID_ARG
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(c)


def test_refactorization_with_new_values():
    """One analysis, two factorizations with different coefficients: each solve answers
    its own matrix."""
    m = 40
    P1 = q1_square(m, lognormal_coefficients(m * m, 1.0, seed=94))
    P2 = q1_square(m, lognormal_coefficients(m * m, 1.0, seed=95))
    c = ctx(hm.HM_PREC_MIXED, n_c=16, hodlr_leaf=16)
    s = hm.hm_analyze(c, P1.n, P1.rowptr, P1.colidx, 2, P1.coords)
    b = rhs_uniform(P1.n, 1, 96)
    for P in (P1, P2, P1):
        hm.hm_factor(s, P.values, 1e-4)
        x = np.zeros_like(b)
        assert hm.hm_solve(s, 1, b, 1e-10, 2000, x)["converged"] == 1
        assert np.linalg.norm(b[:, 0] - P.scipy() @ x[:, 0]) <= 1e-10 * np.linalg.norm(b[:, 0])
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(c)


@pytest.mark.parametrize("n_c", [64, 8])
def test_indefinite_matrix_is_reported(n_c):
    """-A is negative definite: the factorization reports HM_ERR_NOT_SPD (dense fronts)
    or a breakdown of the HODLR leaves, and raises nothing on the device."""
    P = q1_square(24)
    c = ctx(hm.HM_PREC_FP64, n_c=n_c, hodlr_leaf=8)
    s = hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 2, P.coords)
    with pytest.raises(hm.HmError) as e:
        hm.hm_factor(s, -P.values, 1e-6)
    assert e.value.status in (hm.abi.HM_ERR_NOT_SPD, hm.abi.HM_ERR_BREAKDOWN)
    # the context stays usable: the true matrix factors and solves afterwards
    hm.hm_factor(s, P.values, 1e-6)
    b = rhs_uniform(P.n, 1, 97)
    x = np.zeros_like(b)
    assert hm.hm_solve(s, 1, b, 1e-10, 200, x)["converged"] == 1
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(c)


def test_calls_out_of_order_and_bad_inputs():
    P = q1_square(16)
    c = ctx()
    s = hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 2, P.coords)
    b = rhs_uniform(P.n, 1, 98)
    with pytest.raises(hm.HmError) as e:
        hm.hm_solve(s, 1, b, 1e-10, 10, np.zeros_like(b))
    assert e.value.status == hm.abi.HM_ERR_STATE
    hm.hm_destroy(s)
    coords = P.coords.copy()
    coords[0] = coords[1]  # two unknowns on one lattice point: the grid is not full
    with pytest.raises(hm.HmError) as e:
        hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 2, coords)
    assert e.value.status == hm.abi.HM_ERR_INVALID_ARG
    with pytest.raises(hm.HmError) as e:
        hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 4, P.coords)  # dim must be 2 or 3
    assert e.value.status == hm.abi.HM_ERR_INVALID_ARG
    hm.hm_ctx_destroy(c)


@pytest.mark.parametrize("precision", ["HM_PREC_FP64", "HM_PREC_MIXED"])
def test_iteration_cap_reports_no_convergence(precision):
    """A cap of 2 GMRES iterations on a problem that needs more: HM_ERR_NO_CONVERGENCE,
    info reports the cap and a residual above rtol, x holds the last iterate (its residual
    is the reported one, and below that of x0 = 0); the system stays usable."""
    P = q1_square(48, lognormal_coefficients(48 * 48, 1.0, seed=95))
    c = ctx(getattr(hm, precision), nd_leaf=16, hodlr_leaf=16, n_c=16, samples=8)
    s = hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 2, P.coords)
    hm.hm_factor(s, P.values, 1e-1)
    b = rhs_uniform(P.n, 2, 96)
    x = np.zeros_like(b)
    with pytest.raises(hm.HmError) as e:
        hm.hm_solve(s, 2, b, 1e-12, 2, x)
    assert e.value.status == hm.abi.HM_ERR_NO_CONVERGENCE
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 2, b, 1e-12, 2, x, raise_on_no_convergence=False)
    assert info["converged"] == 0 and info["iters"] == 2 and info["relres"] > 1e-12
    A = P.scipy()
    rr = max(np.linalg.norm(b[:, k] - A @ x[:, k]) / np.linalg.norm(b[:, k]) for k in range(2))
    assert abs(rr - info["relres"]) <= 1e-6 * rr and rr < 1.0
    info = hm.hm_solve(s, 2, b, 1e-10, 4000, x)  # the same system converges without the cap
    assert info["converged"] == 1
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(c)


def test_tensor_core_wait_that_runs_out_reports_timeout():
    """The BF16 mode's tensor-core GEMM waits on its MMAs through bounded mbarrier polls.
    The fault injection option adds one more wait per tile, on a barrier that nothing
    arrives on, limited to 16 polls: it runs out right after the tile's last MMA commit
    (no fault, no hang: the kernel then drains the MMAs it issued, with the default
    limit, before it frees its tensor memory), and the factorization reports
    HM_ERR_DEVICE_TIMEOUT.  A new context without the injection on the same device then
    factors and solves."""
    from fixtures import hex_cube
    P = hex_cube(20, lognormal_coefficients(20 ** 3, 0.5, seed=97))
    c = ctx(hm.HM_PREC_MIXED_BF16, wait_limit=16, inject_wait_timeout=1)
    s = hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 3, P.coords)
    with pytest.raises(hm.HmError) as e:
        hm.hm_factor(s, P.values, 1e-4)
    assert e.value.status == hm.abi.HM_ERR_DEVICE_TIMEOUT
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(c)
    c = ctx(hm.HM_PREC_MIXED_BF16)
    s = hm.hm_analyze(c, P.n, P.rowptr, P.colidx, 3, P.coords)
    hm.hm_factor(s, P.values, 1e-4)
    b = rhs_uniform(P.n, 1, 98)
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 1, b, 1e-10, 4000, x)
    assert info["converged"] == 1
    assert np.linalg.norm(b[:, 0] - P.scipy() @ x[:, 0]) / np.linalg.norm(b[:, 0]) <= 1e-10
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(c)
