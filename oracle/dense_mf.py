"""Conventional multifrontal factorization and solve (exact direct solve, FP64).

ORACLE / TEST INFRASTRUCTURE ONLY.

Follows Section 4.1 of the paper:

* ``F_bar_p`` (Eq. fbar): the submatrix of ``A`` on ``I_p U I_p^f`` (rows/columns
  ordered ``I_p`` then ``I_p^f``) with its ``I_p^f x I_p^f`` block set to zero;
* ``F_p = F_bar_p (+) U_{c_1} (+) ...`` (extend-add of the children's updates);
* ``F_p`` split into ``F_pp, F_pf, F_fp, F_ff``; Eq. (update):
  ``U_p = F_ff - F_fp F_pp^{-1} F_pf``;
* solve: upward pass (Eq. upward) ``b_f <- b_f - F_fp F_pp^{-1} b_p`` from leaves to the
  root, then downward pass (Eq. downward) ``x_p = F_pp^{-1}(b_p - F_pf x_f)`` from the
  root to the leaves, ``b_p`` being the value left by the upward pass.

``F_pp^{-1}`` is applied through a Cholesky factorization (LAPACK ``potrf``); every
front's matrices are kept densely.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .nd import ETree
from .symbolic import Symbolic


def permuted_matrix(rowptr, colidx, values, et: ETree) -> sp.csr_matrix:
    """``P A P^T`` in the new numbering (new index i is original index perm[i])."""
    n = et.perm.shape[0]
    A = sp.csr_matrix((values, colidx, rowptr), shape=(n, n))
    return A[et.perm][:, et.perm].tocsr()


def front_indices(et: ETree, sym: Symbolic, p: int) -> np.ndarray:
    b, e = int(et.first[p]), int(et.first[p + 1])
    return np.concatenate([np.arange(b, e), sym.If[p]]).astype(np.int64)


def assemble_fbar(Ap: sp.csr_matrix, et: ETree, sym: Symbolic, p: int) -> np.ndarray:
    """Eq. (fbar): dense ``F_bar_p`` with a zero ``I_p^f x I_p^f`` block."""
    idx = front_indices(et, sym, p)
    F = Ap[idx][:, idx].toarray()
    npv = int(et.first[p + 1] - et.first[p])
    F[npv:, npv:] = 0.0
    return F


def extend_add(F: np.ndarray, U_c: np.ndarray, relmap_c: np.ndarray) -> None:
    """``F <- F (+) U_c``: add the child's update at the rows/columns ``relmap_c``."""
    F[np.ix_(relmap_c, relmap_c)] += U_c


@dataclass
class DenseFront:
    npiv: int
    cho: tuple          # scipy cho_factor of F_pp
    Ffp: np.ndarray     # (nf, npiv)


def factor(Ap: sp.csr_matrix, et: ETree, sym: Symbolic, keep_fronts: bool = False):
    """Conventional multifrontal factorization; returns per-node ``DenseFront``s (and,
    if asked, the assembled fronts ``F_p`` and updates ``U_p``)."""
    nf = et.nfronts
    fronts: list = [None] * nf
    updates: list = [None] * nf
    assembled: list = [None] * nf if keep_fronts else None
    for p in range(nf):
        F = assemble_fbar(Ap, et, sym, p)
        for c in sym.children[p]:
            extend_add(F, updates[c], sym.relmap[c])
            if not keep_fronts:
                updates[c] = None
        if keep_fronts:
            assembled[p] = F.copy()
        npv = int(et.first[p + 1] - et.first[p])
        Fpp, Ffp, Fff = F[:npv, :npv], F[npv:, :npv], F[npv:, npv:]
        cho = sla.cho_factor(Fpp, lower=True)
        updates[p] = Fff - Ffp @ sla.cho_solve(cho, Ffp.T)      # Eq. (update)
        fronts[p] = DenseFront(npv, cho, Ffp.copy())
    return fronts, (assembled, updates) if keep_fronts else None


def solve(fronts, et: ETree, sym: Symbolic, b_new: np.ndarray) -> np.ndarray:
    """Eqs. (upward)/(downward) on a vector or column block in the new numbering."""
    bu = np.array(b_new, dtype=np.float64, copy=True)
    nf = et.nfronts
    for p in range(nf):                                   # upward: leaves -> root
        b, e = int(et.first[p]), int(et.first[p + 1])
        fr = fronts[p]
        bu[sym.If[p]] -= fr.Ffp @ sla.cho_solve(fr.cho, bu[b:e])
    x = np.zeros_like(bu)
    for p in range(nf - 1, -1, -1):                       # downward: root -> leaves
        b, e = int(et.first[p]), int(et.first[p + 1])
        fr = fronts[p]
        x[b:e] = sla.cho_solve(fr.cho, bu[b:e] - fr.Ffp.T @ x[sym.If[p]])
    return x


def direct_solve(rowptr, colidx, values, coords, b, leaf_size: int = 64, refine: int = 2,
                 dofs_per_node: int = 1):
    """Exact ``x* = A^{-1} b`` (original numbering) by the conventional multifrontal
    method plus ``refine`` steps of FP64 iterative refinement."""
    from .nd import nested_dissection
    from .symbolic import symbolic
    et = nested_dissection(coords, leaf_size, dofs_per_node)
    sym = symbolic(rowptr, colidx, et)
    Ap = permuted_matrix(rowptr, colidx, values, et)
    fronts, _ = factor(Ap, et, sym)
    bn = np.asarray(b)[et.perm]
    x = solve(fronts, et, sym, bn)
    for _ in range(refine):
        x = x + solve(fronts, et, sym, bn - Ap @ x)
    out = np.empty_like(x)
    out[et.perm] = x
    return out
