"""Boundary distance low-rank approximation (BDLR), Section 2.2 and Eq. (Bhat).

ORACLE / TEST INFRASTRUCTURE ONLY.

For an off-diagonal block ``B = K[X, Y]`` of a frontal matrix (X, Y disjoint sets of
the front's local positions), the interaction graph is the graph of ``A`` restricted to
the front's unknowns ``I_p U I_p^f`` (Section 4.2.1).  The reading taken here:

* rows ``I``: the positions of X whose graph distance to the set Y is at most ``depth``,
  columns ``J``: the positions of Y within ``depth`` of X; each list ordered by distance,
  then by position, and cut to at most ``cap`` entries;
* ``B^ = B(I, J)`` is factored by Gaussian elimination with complete pivoting
  (``P B^ Q = L U``); the pivot of step s is the entry of largest magnitude among the
  rows and columns not yet pivoted, ties going to the lower (row, column) in the order
  of I and J; the rank r is the number of leading pivots with ``|u_ss| >= eps |u_11|``;
* ``C~ = B(:, J_q[:r]) U_r^{-1}``, ``R~ = L_r^{-1} B(I_p[:r], :)`` and ``B ~ C~ R~``,
  returned as ``(U, V) = (C~, R~^T)``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def front_graph(Ap: sp.csr_matrix, idx: np.ndarray) -> sp.csr_matrix:
    """Structural pattern of ``A`` among the front's unknowns (local positions), no self
    loops: stored entries count as edges even where their value is zero (the trilinear
    hex stores exact zeros for edge-adjacent nodes)."""
    G = Ap[idx][:, idx].tocsr()
    G = sp.csr_matrix((np.ones(G.data.shape[0], np.int8), G.indices, G.indptr), shape=G.shape)
    G.setdiag(0)
    G.eliminate_zeros()
    return G


def distances(G: sp.csr_matrix, sources: np.ndarray, depth: int) -> np.ndarray:
    """Breadth-first distance of every vertex to the source set, up to ``depth``
    (``depth + 1`` stands for farther or unreachable)."""
    n = G.shape[0]
    d = np.full(n, depth + 1, dtype=np.int64)
    d[sources] = 0
    frontier = np.asarray(sources, dtype=np.int64)
    for level in range(1, depth + 1):
        nb = np.unique(G[frontier].indices) if frontier.size else np.zeros(0, np.int64)
        new = nb[d[nb] > depth]
        d[new] = level
        frontier = new
    return d


def select(G: sp.csr_matrix, X: np.ndarray, Y: np.ndarray, depth: int, cap: int):
    """Positions (relative to X and to Y) of the rows I and columns J of the block."""
    dY = distances(G, Y, depth)
    dX = distances(G, X, depth)

    def pick(d_other, S):
        dist = d_other[S]
        order = np.lexsort((np.arange(S.shape[0]), dist))
        order = order[dist[order] <= depth]
        return order[:cap]

    return pick(dY, X), pick(dX, Y)


def complete_pivoting_lu(Bh: np.ndarray, eps: float):
    """Rank-revealing LU with complete pivoting: (pr, pc, L_r, U_r) with r = len(pr)."""
    M = np.array(Bh, dtype=np.float64, copy=True)
    nI, nJ = M.shape
    rows_used = np.zeros(nI, bool)
    cols_used = np.zeros(nJ, bool)
    pr, pc = [], []
    u11 = 0.0
    for s in range(min(nI, nJ)):
        A = np.abs(M)
        A[rows_used, :] = -1.0
        A[:, cols_used] = -1.0
        flat = int(np.argmax(A))           # first maximum in row-major order
        i, j = divmod(flat, nJ)
        v = A[i, j]
        if s == 0:
            u11 = v
        if v <= 0.0 or (s > 0 and eps > 0.0 and v < eps * u11):
            break
        pr.append(i)
        pc.append(j)
        piv = M[i, j]
        act_r = ~rows_used
        act_r[i] = False
        act_c = ~cols_used
        act_c[j] = False
        l = M[act_r, j] / piv
        M[np.ix_(act_r, act_c)] -= np.outer(l, M[i, act_c])
        M[act_r, j] = l
        rows_used[i] = True
        cols_used[j] = True
    r = len(pr)
    S = M[np.ix_(pr, pc)] if r else np.zeros((0, 0))
    L = np.tril(S, -1) + np.eye(r)
    U = np.triu(S)
    return np.array(pr, int), np.array(pc, int), L, U


def compress(B: np.ndarray, I: np.ndarray, J: np.ndarray, eps: float):
    """``(U, V)`` with ``B ~ U V^T`` from the rows I and columns J (Eq. Bhat)."""
    if I.size == 0 or J.size == 0:
        return np.zeros((B.shape[0], 0)), np.zeros((B.shape[1], 0))
    pr, pc, L, U = complete_pivoting_lu(B[np.ix_(I, J)], eps)
    if pr.size == 0:
        return np.zeros((B.shape[0], 0)), np.zeros((B.shape[1], 0))
    C = B[:, J[pc]]
    R = B[I[pr], :]
    Ct = sla.solve_triangular(U.T, C.T, lower=True).T          # C U_r^{-1}
    Rt = sla.solve_triangular(L, R, lower=True, unit_diagonal=True)  # L_r^{-1} R
    return Ct, Rt.T
