"""Oracle computations for the full-size parity tests, run in spawned worker processes.

Test infrastructure: these functions call only ``fixtures`` (the seeded inputs) and
``oracle`` (the FP64 CPU restatement of the method); nothing here imports the CUDA
package.  The full-size tests start a ``spawn`` process pool on them before their GPU
solves, so the oracle's minutes of host work overlap the GPU work.
"""
from __future__ import annotations

import numpy as np

from fixtures import p1_batch_sizes, p1_jittered, rhs_uniform, workload
from oracle import condest, dense_mf, hodlr, hodlr_mf, nd, symbolic


def direct_with_kappa(name: str, nrhs: int, kappa_iters: int = 20, **kw):
    """The exact solution ``x*`` (conventional multifrontal direct solve, Eqs. update,
    upward, downward, plus two steps of FP64 refinement) of the named workload's seeded
    right-hand sides, and the Lanczos estimate of ``kappa(A)`` (through the same
    factor).  Returns ``(x*, kappa)`` in the original numbering."""
    P, prm = workload(name, **kw)
    dpn = 3 if name.startswith("elasticity") else 1
    b = rhs_uniform(P.n, nrhs, prm["rhs_seed"])
    et = nd.nested_dissection(P.coords, 64, dpn)
    sym = symbolic.symbolic(P.rowptr, P.colidx, et)
    Ap = dense_mf.permuted_matrix(P.rowptr, P.colidx, P.values, et)
    fronts, _ = dense_mf.factor(Ap, et, sym)
    bn = b[et.perm]
    x = dense_mf.solve(fronts, et, sym, bn)
    for _ in range(2):
        x = x + dense_mf.solve(fronts, et, sym, bn - Ap @ x)
    out = np.empty_like(x)
    out[et.perm] = x
    kappa = condest.kappa_estimate(Ap, lambda v: dense_mf.solve(fronts, et, sym, v), kappa_iters)
    return out, kappa


def batch_direct(indices, count: int = 256, seed: int = 5, rhs_seed: int = 6, kappa_iters: int = 12):
    """``x*`` and the kappa estimate of meshes ``indices`` of the P1 batch, for the
    batch's seeded right-hand side (one column over all meshes' unknowns)."""
    sizes = p1_batch_sizes(count, seed)
    nk = (sizes.astype(np.int64) - 1) ** 2
    bp = np.concatenate([[0], np.cumsum(nk)])
    b = rhs_uniform(int(bp[-1]), 1, rhs_seed)[:, 0]
    out = []
    for k in indices:
        m = p1_jittered(int(sizes[k]), seed=seed + int(k))
        bk = b[bp[k]:bp[k + 1]]
        et = nd.nested_dissection(m.coords, 64)
        sym = symbolic.symbolic(m.rowptr, m.colidx, et)
        Ap = dense_mf.permuted_matrix(m.rowptr, m.colidx, m.values, et)
        fronts, _ = dense_mf.factor(Ap, et, sym)
        bn = bk[et.perm]
        x = dense_mf.solve(fronts, et, sym, bn)
        for _ in range(2):
            x = x + dense_mf.solve(fronts, et, sym, bn - Ap @ x)
        xs = np.empty_like(x)
        xs[et.perm] = x
        kappa = condest.kappa_estimate(Ap, lambda v: dense_mf.solve(fronts, et, sym, v), kappa_iters)
        out.append((int(k), xs, kappa))
    return out


def hodlr_blocks(name: str, max_level: int, tol: float, samples: int, seed: int = 0x5EED, **kw):
    """The oracle's HODLR-MF factorization (Section 4.2.1) with the range finder and the
    GPU's sketch (same Philox stream, width ``samples``) on the named workload.  For
    every HODLR front at tree depth <= ``max_level``: ``{key: (B, U, V)}`` with ``B`` the
    exact block of the oracle's own assembled front ``F_p`` (built from the oracle's own
    children's updates) and ``B ~ U V^T`` its compressed form; key ``(-1, 0)`` is the
    coupling block ``F_fp ~ W V^T``, key ``(level, node)`` an off-diagonal block of the
    pivot block's HODLR tree.  Also returns ``nupd`` per front."""
    P, _ = workload(name, **kw)
    et = nd.nested_dissection(P.coords, 64)
    sym = symbolic.symbolic(P.rowptr, P.colidx, et)
    Ap = dense_mf.permuted_matrix(P.rowptr, P.colidx, P.values, et)
    prm = hodlr_mf.Params(tol=tol, n_c=64, leaf=64, compressor="rrf", samples=samples, seed=seed)
    fr, tr = hodlr_mf.factor(Ap, et, sym, prm, keep=True)
    out = {}
    for q in range(et.nfronts):
        f = fr[q]
        if et.level[q] > max_level or f.kind != "hodlr":
            continue
        F, npv = tr["F"][q], f.npiv
        blocks = {}
        if f.W.shape[0]:
            blocks[(-1, 0)] = (F[npv:, :npv].copy(), f.W, f.V)
        for node in hodlr.iter_nodes(f.H):
            if node.children:
                a, b = node.children
                blocks[(node.level, node.index)] = (F[a.lo:a.hi, b.lo:b.hi].copy(), node.U, node.V)
        out[q] = (len(sym.If[q]), npv, blocks)
    return out
