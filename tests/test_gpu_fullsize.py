"""Parity at the benchmark configurations' full sizes, in the launch configuration that
bench.py times, on outputs the oracle can produce at that size: the whole ordering,
tree and frontal index sets (bit-exact), sampled dense-front update matrices (each
recomputed by the oracle from the assembled front alone), and, for the solutions,
properties that hold at any size (every right-hand side's true FP64 residual, computed
on the host, at or below rtol; per-mesh residuals for the batch; direct solves of the
batch's smallest meshes)."""
import numpy as np
import pytest

from fixtures import p1_batch, rhs_uniform, workload
from oracle import dense_mf, nd, symbolic

pytestmark = pytest.mark.gpu

try:
    import paper_1410_2697_gb300 as hm
except ImportError:  # the library is built on the GPU machine; a CPU-only machine skips
    import torch
    if torch.cuda.is_available():
        raise
    pytest.skip("CUDA library not built on this CPU-only machine", allow_module_level=True)

RTOL = 1e-10


def bench_ctx(precision, keep_fronts=0):
    o = hm.hm_default_opts()  # nd_leaf 64, hodlr_leaf 64, n_c 64, samples 48: bench.py's
    o.precision = precision
    o.keep_fronts = keep_fronts  # 1: every front's update stays readable (hm_get_update)
    return hm.hm_create(o)


def check_ordering(s, et, sym):
    perm, first, parent, level = hm.hm_get_ordering(s)
    assert np.array_equal(perm, et.perm)
    assert np.array_equal(first, et.first)
    assert np.array_equal(parent, et.parent)
    assert np.array_equal(level, et.level)
    nupd, off, lst, rel = hm.hm_get_symbolic(s)
    for q in range(et.nfronts):
        assert nupd[q] == len(sym.If[q]), q
        assert np.array_equal(lst[off[q]:off[q] + nupd[q]], sym.If[q]), q
        if et.parent[q] >= 0:
            assert np.array_equal(rel[off[q]:off[q] + nupd[q]], sym.relmap[q]), q


@pytest.fixture(scope="module")
def q1024():
    P, prm = workload("q1_lognormal_1024x1024")
    et = nd.nested_dissection(P.coords, 64)
    sym = symbolic.symbolic(P.rowptr, P.colidx, et)
    return P, prm, et, sym


def test_q1024_ordering_and_symbolic_bit_exact(q1024):
    P, _, et, sym = q1024
    ctx = bench_ctx(hm.HM_PREC_MIXED)
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
    check_ordering(s, et, sym)
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


def test_q1024_sampled_leaf_updates_and_bench_solve(q1024):
    P, prm, et, sym = q1024
    ctx = bench_ctx(hm.HM_PREC_MIXED, keep_fronts=1)
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 2, P.coords)
    hm.hm_factor(s, P.values, prm["tol"])
    # leaves: U = F_ff - F_fp F_pp^{-1} F_pf of the assembled front alone (FP32 factor)
    Ap = dense_mf.permuted_matrix(P.rowptr, P.colidx, P.values, et)
    has_child = np.zeros(et.nfronts, bool)
    has_child[et.parent[et.parent >= 0]] = True
    leaves = np.flatnonzero(~has_child)
    for q in leaves[np.linspace(0, len(leaves) - 1, 24).astype(int)]:
        F = dense_mf.assemble_fbar(Ap, et, sym, int(q))
        npv = int(et.first[q + 1] - et.first[q])
        ref = F[npv:, npv:] - F[npv:, :npv] @ np.linalg.solve(F[:npv, :npv], F[:npv, npv:])
        U = hm.hm_get_update(s, int(q), len(sym.If[q]))
        err = np.abs(np.tril(U) - np.tril(ref)).max() / np.abs(ref).max()
        assert err <= 2e-4, (q, err)
    # the bench's solve: 16 right-hand sides to rtol, true residuals on the host
    b = rhs_uniform(P.n, prm["nrhs"], prm["rhs_seed"])
    x = np.zeros_like(b)
    info = hm.hm_solve(s, prm["nrhs"], b, RTOL, 4000, x)
    assert info["converged"] == 1
    A = P.scipy()
    for c in range(prm["nrhs"]):
        assert np.linalg.norm(b[:, c] - A @ x[:, c]) / np.linalg.norm(b[:, c]) <= RTOL, c
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


def test_hex64_bf16_ordering_and_solve():
    P, prm = workload("hex_lognormal_64^3")
    et = nd.nested_dissection(P.coords, 64)
    sym = symbolic.symbolic(P.rowptr, P.colidx, et)
    ctx = bench_ctx(hm.HM_PREC_MIXED_BF16)
    s = hm.hm_analyze(ctx, P.n, P.rowptr, P.colidx, 3, P.coords)
    check_ordering(s, et, sym)
    hm.hm_factor(s, P.values, prm["tol"])
    b = rhs_uniform(P.n, 1, prm["rhs_seed"])
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 1, b, RTOL, 4000, x)
    assert info["converged"] == 1
    assert np.linalg.norm(b[:, 0] - P.scipy() @ x[:, 0]) / np.linalg.norm(b[:, 0]) <= RTOL
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)


def test_p1_batch256_per_mesh_ordering_and_solutions():
    P, bp, meshes = p1_batch(256, 5)
    ctx = bench_ctx(hm.HM_PREC_MIXED)
    s = hm.hm_analyze_batch(ctx, P.n, P.rowptr, P.colidx, 2, P.coords, bp)
    perm, first, parent, level = hm.hm_get_ordering(s)
    node = 0
    for k, m in enumerate(meshes):  # each mesh's block is its own nested dissection
        et = nd.nested_dissection(m.coords, 64)
        nfk = et.nfronts
        assert np.array_equal(perm[bp[k]:bp[k + 1]], et.perm + bp[k]), k
        assert np.array_equal(first[node:node + nfk], et.first[:-1] + bp[k]), k
        assert np.array_equal(parent[node:node + nfk], np.where(et.parent >= 0, et.parent + node, -1)), k
        assert np.array_equal(level[node:node + nfk], et.level), k
        node += nfk
    hm.hm_factor(s, P.values, 1e-4)
    b = rhs_uniform(P.n, 1, 6)
    x = np.zeros_like(b)
    info = hm.hm_solve(s, 1, b, RTOL, 4000, x)
    assert info["converged"] == 1
    r = b[:, 0] - P.scipy() @ x[:, 0]
    for k in range(len(meshes)):
        sl = slice(bp[k], bp[k + 1])
        assert np.linalg.norm(r[sl]) / np.linalg.norm(b[sl, 0]) <= RTOL, k
    for k in np.argsort([m.n for m in meshes])[:3]:  # direct solves of the smallest meshes
        m, sl = meshes[k], slice(bp[k], bp[k + 1])
        xs = dense_mf.direct_solve(m.rowptr, m.colidx, m.values, m.coords, b[sl, 0])
        assert np.linalg.norm(x[sl, 0] - xs) / np.linalg.norm(xs) <= 1e-8, k
    hm.hm_destroy(s)
    hm.hm_ctx_destroy(ctx)
