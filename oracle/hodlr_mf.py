"""HODLR-accelerated multifrontal factorization and solve (FP64 oracle).

ORACLE / TEST INFRASTRUCTURE ONLY.

Section 4.2 of the paper, taken step by step:

* every front ``F_p`` is assembled from ``F_bar_p`` and the children's updates
  (Eqs. HODLR_EA / HODLR_EA_Expand); this oracle forms the sum densely (each child
  update ``U_c = F_ff,c - W_c T_c W_c^T`` expanded), which is allowed for a reference;
* fronts whose pivot block has at most ``n_c`` unknowns stay dense (the paper's
  dense-to-HODLR threshold ``n_c``, table caption of the results table) and follow the
  conventional steps of ``dense_mf``;
* larger fronts: ``F_pp`` becomes a HODLR matrix (recursive halving, ``leaf``), each
  off-diagonal block and the coupling block ``F_fp ~ W V^T`` are compressed at ``tol``;
  ``F_pp^HODLR`` is factored by recursive Woodbury; the update keeps the low-rank form
  ``U_p = F_ff - W_p V_p^T`` with ``V_p^T = T W^T``, ``T = V^T (F_pp^HODLR)^{-1} V``
  (Eq. update_HODLR_Parent, whose inverse is read as ``F_pp``'s, consistent with
  Eq. update);
* ``compress_ff=True`` additionally replaces ``F_ff`` by its HODLR approximation before
  the update is formed (the paper's ``F_ff^HODLR``); the default keeps ``F_ff`` dense,
  as the GPU design does;
* solve (Section 4.2.2): the conventional upward/downward passes with ``F_pp^{-1}``
  replaced by the HODLR solve and ``F_fp``, ``F_pf`` by the low-rank products:
  upward ``b_f <- b_f - W V^T (F_pp^HODLR)^{-1} b_p``, downward
  ``x_p = (F_pp^HODLR)^{-1} (b_p - V W^T x_f)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import bdlr, hodlr
from .dense_mf import assemble_fbar, extend_add, front_indices
from .nd import ETree
from .philox import block_id, sketch
from .symbolic import Symbolic


@dataclass
class Params:
    tol: float = 1e-6
    n_c: int = 64
    leaf: int = 64
    compressor: str = "svd"        # "svd" | "rrf" | "bdlr"
    bdlr_depth: int = 1            # BDLR graph-distance depth
    samples: int = 64              # RRF sketch width k (capped by the block's size)
    seed: int = 0x5EED             # RRF sketch seed
    compress_ff: bool = False
    level_samples: dict | None = None  # sketch width per front level (tree depth); default samples
    adaptive: bool = False         # grow the width of a level whose blocks hit it (see factor)
    max_samples: int = 96          # largest width the adaptive rule may reach (64 for FP64 parity)


@dataclass
class Front:
    npiv: int
    kind: str                       # "dense" | "hodlr"
    cho: tuple | None = None        # dense: Cholesky of F_pp
    Ffp: np.ndarray | None = None   # dense: F_fp
    H: hodlr.HNode | None = None    # hodlr: factored F_pp^HODLR
    W: np.ndarray | None = None     # hodlr: F_fp ~ W V^T
    V: np.ndarray | None = None


def _compressor(prm: Params, front: int, kind: int, graph=None, npv: int = 0, samples: int | None = None):
    width = prm.samples if samples is None else samples

    def comp(B, level, index, lo=None, mid=None, hi=None):
        if prm.compressor == "svd":
            return hodlr.truncated_svd(B, prm.tol)
        if prm.compressor == "bdlr":
            # rows / columns of B as positions in the front: pivot-block nodes [lo, mid) x
            # [mid, hi); the coupling block F_fp has the update rows and the pivot columns
            off = npv if kind == 2 else 0  # F_ff nodes sit after the pivot positions
            X = np.arange(off + lo, off + mid) if kind != 1 else np.arange(npv, npv + B.shape[0])
            Y = np.arange(off + mid, off + hi) if kind != 1 else np.arange(0, npv)
            cap = min(width, B.shape[0], B.shape[1])
            I, J = bdlr.select(graph, X, Y, prm.bdlr_depth, cap)
            return bdlr.compress(B, I, J, prm.tol)
        k = min(width, B.shape[0], B.shape[1])
        Om = sketch(B.shape[1], k, block_id(front, kind, level, index), prm.seed)
        return hodlr.randomized_range_finder(B, prm.tol, Om)
    return comp


def factor(Ap: sp.csr_matrix, et: ETree, sym: Symbolic, prm: Params, keep: bool = False):
    """HODLR-MF factorization.  With ``prm.adaptive`` the tolerance rule of Section 2.2
    decides the ranks: a block whose rank reached its sketch width was cut by the width,
    not by tol, so the width of every front level (tree depth) holding such a block is
    doubled (up to ``max_samples`` and the level's largest block dimension) and the
    factorization is repeated, at most four times; the widths used are returned in
    ``trace["widths"]`` when ``keep`` is set, and always in ``factor.last_widths``."""
    widths = dict(prm.level_samples or {})
    for _ in range(5):
        fronts, trace = _factor_once(Ap, et, sym, prm, widths, keep)
        if not prm.adaptive:
            break
        capped, room = _capped_levels(fronts, et, prm, widths)
        grow = False
        for lv in sorted(capped):
            w = widths.get(lv, prm.samples)
            if w < min(prm.max_samples, room[lv]):
                widths[lv] = min(2 * w, prm.max_samples, room[lv])
                grow = True
        if not grow:
            break
    factor.last_widths = dict(widths)
    if keep:
        trace["widths"] = dict(widths)
    return fronts, trace


def _capped_levels(fronts, et: ETree, prm: Params, widths: dict):
    """Front levels holding a block whose rank equals its sketch width while the block
    is larger than that width; and, per level, the largest block dimension."""
    capped, room = set(), {}
    for p, fr in enumerate(fronts):
        if fr.kind != "hodlr":
            continue
        lv = int(et.level[p])
        w = widths.get(lv, prm.samples)
        blocks = [(fr.W.shape[1], fr.W.shape[0], fr.V.shape[0])] if fr.W.shape[0] else []
        for node in hodlr.iter_nodes(fr.H):
            if node.children:
                a, b = node.children
                blocks.append((node.U.shape[1], a.hi - a.lo, b.hi - b.lo))
        for r, m, n in blocks:
            room[lv] = max(room.get(lv, 0), min(m, n))
            if r >= min(w, m, n) and min(w, m, n) < min(m, n):
                capped.add(lv)
    return capped, room


def _factor_once(Ap: sp.csr_matrix, et: ETree, sym: Symbolic, prm: Params, widths: dict, keep: bool):
    nf = et.nfronts
    fronts: list = [None] * nf
    updates: list = [None] * nf
    trace = {"F": [None] * nf, "U": [None] * nf} if keep else None
    for p in range(nf):
        F = assemble_fbar(Ap, et, sym, p)
        for c in sym.children[p]:
            extend_add(F, updates[c], sym.relmap[c])
            if not keep:
                updates[c] = None
        if keep:
            trace["F"][p] = F.copy()
        npv = int(et.first[p + 1] - et.first[p])
        Fpp, Ffp, Fff = F[:npv, :npv], F[npv:, :npv], F[npv:, npv:]
        if npv <= prm.n_c:
            cho = sla.cho_factor(Fpp, lower=True)
            updates[p] = Fff - Ffp @ sla.cho_solve(cho, Ffp.T)
            fronts[p] = Front(npv, "dense", cho=cho, Ffp=Ffp.copy())
        else:
            graph = bdlr.front_graph(Ap, front_indices(et, sym, p)) if prm.compressor == "bdlr" else None
            w = widths.get(int(et.level[p]), prm.samples)
            H = hodlr.build(Fpp, prm.leaf, prm.tol, _compressor(prm, p, 0, graph, npv, w))
            hodlr.factor(H)
            W, V = _compressor(prm, p, 1, graph, npv, w)(Ffp, 0, 0) if Ffp.shape[0] else \
                (np.zeros((0, 0)), np.zeros((npv, 0)))
            if prm.compress_ff and Fff.shape[0]:
                Fff = hodlr.to_dense(hodlr.build(Fff, prm.leaf, prm.tol, _compressor(prm, p, 2, graph, npv, w)))
            T = V.T @ hodlr.solve(H, V)
            updates[p] = Fff - W @ T @ W.T
            fronts[p] = Front(npv, "hodlr", H=H, W=W, V=V)
        if keep:
            trace["U"][p] = updates[p]
    return fronts, trace


def _pivot_solve(fr: Front, X: np.ndarray) -> np.ndarray:
    if fr.kind == "dense":
        return sla.cho_solve(fr.cho, X)
    return hodlr.solve(fr.H, X)


def apply(fronts, et: ETree, sym: Symbolic, r_new: np.ndarray) -> np.ndarray:
    """Preconditioner ``M^{-1} r`` (new numbering; vector or column block)."""
    bu = np.array(r_new, dtype=np.float64, copy=True)
    nf = et.nfronts
    for p in range(nf):                                            # upward pass
        b, e = int(et.first[p]), int(et.first[p + 1])
        fr = fronts[p]
        y = _pivot_solve(fr, bu[b:e])
        if fr.kind == "dense":
            bu[sym.If[p]] -= fr.Ffp @ y
        else:
            bu[sym.If[p]] -= fr.W @ (fr.V.T @ y)
    x = np.zeros_like(bu)
    for p in range(nf - 1, -1, -1):                                # downward pass
        b, e = int(et.first[p]), int(et.first[p + 1])
        fr = fronts[p]
        xf = x[sym.If[p]]
        if fr.kind == "dense":
            x[b:e] = _pivot_solve(fr, bu[b:e] - fr.Ffp.T @ xf)
        else:
            x[b:e] = _pivot_solve(fr, bu[b:e] - fr.V @ (fr.W.T @ xf))
    return x


def ranks(fronts) -> dict:
    """Per front: ranks of the pivot block's off-diagonal blocks and of ``F_fp``."""
    out = {}
    for p, fr in enumerate(fronts):
        if fr.kind == "hodlr":
            out[p] = {"fp": int(fr.W.shape[1]),
                      "pp": [(nd.level, nd.index, nd.rank) for nd in hodlr.iter_nodes(fr.H) if nd.children]}
    return out
