"""3D linear elasticity (three displacement components per node) through the C ABI:
nested dissection over whole nodes (dofs_per_node = 3) bit-exact against the oracle,
solutions against the oracle's direct solve, and the full-size 40^3 workload."""
import numpy as np
import pytest

from fixtures import hex_elasticity, lognormal_coefficients, rhs_uniform, workload
from oracle import dense_mf, nd, symbolic

pytestmark = pytest.mark.gpu

try:
    import paper_1410_2697_gb300 as hm
except ImportError:
    import torch
    if torch.cuda.is_available():
        raise
    pytest.skip("CUDA library not built on this CPU-only machine", allow_module_level=True)


def ctx_for(precision, leaf=64, n_c=64, hodlr_leaf=64):
    o = hm.hm_default_opts()
    o.precision = precision
    o.dofs_per_node = 3
    o.nd_leaf = leaf
    o.n_c = n_c
    o.hodlr_leaf = hodlr_leaf
    return hm.hm_create(o)


def check_ordering(s, P, leaf):
    et = nd.nested_dissection(P.coords, leaf, 3)
    sym = symbolic.symbolic(P.rowptr, P.colidx, et)
    perm, first, parent, level = hm.hm_get_ordering(s)
    assert np.array_equal(perm, et.perm) and np.array_equal(first, et.first)
    assert np.array_equal(parent, et.parent) and np.array_equal(level, et.level)
    nupd, off, lst, rel = hm.hm_get_symbolic(s)
    for q in range(et.nfronts):
        assert np.array_equal(lst[off[q]:off[q] + nupd[q]], sym.If[q]), q
        if et.parent[q] >= 0:
            assert np.array_equal(rel[off[q]:off[q] + nupd[q]], sym.relmap[q]), q


@pytest.mark.parametrize("m,leaf", [(7, 24), (10, 64)])
def test_elasticity_ordering_bit_exact(m, leaf):
    P = hex_elasticity(m, lognormal_coefficients(m ** 3, 0.5, seed=60 + m))
    ctx = ctx_for(hm.HM_PREC_MIXED, leaf=leaf)
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 3, P.coords)
    check_ordering(s, P, leaf)
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


@pytest.mark.parametrize("precision", ["HM_PREC_FP64", "HM_PREC_MIXED"])
def test_elasticity_solution_matches_oracle(precision):
    m = 10
    P = hex_elasticity(m, lognormal_coefficients(m ** 3, 0.5, seed=71))
    ctx = ctx_for(getattr(hm, precision), leaf=64, n_c=24, hodlr_leaf=24)
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 3, P.coords)
    fi = hm.hm_factor(s, P.values, 1e-4)
    assert fi["n_hodlr"] > 0
    b = rhs_uniform(P.n, 2, 72)
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 2, b, 1e-10, 2000, x)
    assert info["converged"] == 1
    for c in range(2):
        xs = dense_mf.direct_solve(P.rowptr, P.colidx, P.values, P.coords, b[:, c], leaf_size=64,
                                   dofs_per_node=3)
        assert np.linalg.norm(x[:, c] - xs) / np.linalg.norm(xs) <= 1e-8
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


def test_dofs_per_node_needs_shared_coordinates():
    P = hex_elasticity(5)
    coords = P.coords.copy()
    coords[4, 0] += 1  # the second component of node 1 moved to another lattice point
    ctx = ctx_for(hm.HM_PREC_MIXED)
    with pytest.raises(hm.HmError) as e:
        hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 3, coords)
    assert e.value.status == hm.abi.HM_ERR_INVALID_ARG
    hm.hm_ctx_destroy(ctx)


def test_elasticity_40_full_size():
    """The bench workload (178k unknowns): ordering and front sets bit-exact, true FP64
    residual of the bench's solve at rtol."""
    P, prm = workload("elasticity_hex_40^3")
    ctx = ctx_for(hm.HM_PREC_MIXED)
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 3, P.coords)
    check_ordering(s, P, 64)
    hm.hm_factor(s, P.values, prm["tol"])
    b = rhs_uniform(P.n, 1, prm["rhs_seed"])
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 1, b, 1e-10, 4000, x)
    assert info["converged"] == 1
    assert np.linalg.norm(b[:, 0] - P.scipy() @ x[:, 0]) / np.linalg.norm(b[:, 0]) <= 1e-10
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)
