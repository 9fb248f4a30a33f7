"""Batched independent meshes (a block-diagonal A analysed as a forest): the CUDA path
against per-mesh oracle runs.  Ordering and tree are integer work (bit-exact with the
per-mesh nested dissection, blocks concatenated); GMRES must converge on every
(mesh, right-hand side) pair separately, and each mesh's solution must match the direct
solve of that mesh alone."""
import numpy as np
import pytest

from fixtures import block_diagonal, p1_jittered, q1_square, rhs_uniform
from oracle import dense_mf, nd

pytestmark = pytest.mark.gpu

try:
    import paper_1410_2697_gb300 as hm
except ImportError:  # the library is built on the GPU machine; a CPU-only machine skips
    import torch
    if torch.cuda.is_available():
        raise
    pytest.skip("CUDA library not built on this CPU-only machine", allow_module_level=True)


def small_batch():
    meshes = [p1_jittered(nc, seed=5 + i) for i, nc in enumerate([9, 14, 21, 6, 12, 17])]
    meshes.append(q1_square(13))
    return block_diagonal(meshes), meshes


def analyze(prob, block_ptr, precision, **kw):
    o = hm.hm_default_opts()
    o.precision = precision
    o.nd_leaf = kw.get("nd_leaf", 16)
    o.hodlr_leaf = kw.get("hodlr_leaf", 16)
    o.n_c = kw.get("n_c", 16)
    o.samples = kw.get("samples", 24)
    ctx = hm.hm_create(o)
    s = hm.hm_analyze_batch(ctx, prob.n, prob.rowptr, prob.colidx, prob.dim, prob.coords, block_ptr)
    return ctx, s


def test_forest_ordering_is_per_mesh_nested_dissection():
    (prob, bp), meshes = small_batch()
    ctx, s = analyze(prob, bp, 1)
    perm, first, parent, level = hm.hm_get_ordering(s)
    ref_perm, ref_first, ref_parent, ref_level = [], [], [], []
    off = 0
    for b, m in enumerate(meshes):
        et = nd.nested_dissection(m.coords, 16)
        ref_perm.append(et.perm + bp[b])
        ref_first.append(np.asarray(et.first[:-1]) + bp[b])
        ref_parent.append(np.where(et.parent >= 0, et.parent + off, -1))
        ref_level.append(et.level)
        off += et.nfronts
    assert np.array_equal(perm, np.concatenate(ref_perm))
    assert np.array_equal(first[:-1], np.concatenate(ref_first)) and first[-1] == prob.n
    assert np.array_equal(parent, np.concatenate(ref_parent))
    assert np.array_equal(level, np.concatenate(ref_level))
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_gmres_converges_per_mesh(prec):
    (prob, bp), meshes = small_batch()
    # right-hand sides of very different sizes per mesh: each must meet its own rtol
    b = rhs_uniform(prob.n, 2, 11)
    for k in range(len(meshes)):
        b[bp[k]:bp[k + 1]] *= 10.0 ** (3 * (k % 3) - 3)
    ctx, s = analyze(prob, bp, prec)
    hm.hm_factor(s, prob.values, 1e-6 if prec == 0 else 1e-4)
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 2, b, 1e-10, 500, x)
    assert info["converged"] == 1
    for k, m in enumerate(meshes):
        A = m.scipy()
        sl = slice(bp[k], bp[k + 1])
        for c in range(2):
            rel = np.linalg.norm(b[sl, c] - A @ x[sl, c]) / np.linalg.norm(b[sl, c])
            assert rel <= 1e-10, (k, c, rel)
        xs = np.stack([dense_mf.direct_solve(m.rowptr, m.colidx, m.values, m.coords, b[sl, c])
                       for c in range(2)], 1)
        err = np.linalg.norm(x[sl] - xs) / np.linalg.norm(xs)
        assert err <= 1e-8, (k, err)
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


def test_batch_rejects_couplings_between_blocks():
    (prob, bp), _ = small_batch()
    bad = bp.copy()
    bad[1] += 1  # moves one unknown (and its couplings) across a block boundary
    o = hm.hm_default_opts()
    ctx = hm.hm_create(o)
    with pytest.raises(hm.HmError):
        hm.hm_analyze_batch(ctx, prob.n, prob.rowptr, prob.colidx, prob.dim, prob.coords, bad)
    hm.hm_ctx_destroy(ctx)
