"""HODLR matrices: compression, recursive Woodbury factorization, solve (FP64).

ORACLE / TEST INFRASTRUCTURE ONLY.

* Structure (Section 2.1, Eq. HODLR2): a matrix is split into a 2x2 block matrix whose
  diagonal blocks are HODLR matrices themselves and whose off-diagonal blocks are low
  rank, ``K_12 = U V^T``.  The partition of an index range of size ``n`` halves it
  (``floor(n/2)`` first) down to a uniform depth ``L = ceil(log2(n / leaf))`` so every
  leaf has at most ``leaf`` rows.  Symmetric storage: ``K_21 = K_12^T = V U^T``.
* Compression of an off-diagonal block ``B`` to rank ``r`` at tolerance ``tol``:
  ``truncated_svd`` keeps the singular values ``sigma_i > tol * sigma_1(B)`` (the
  relative rule of Section 2.2, ``|u_{r+1,r+1} / u_11| < eps``, read for singular
  values); ``randomized_range_finder`` is the randomized alternative the paper cites
  (Section 2.2): ``Y = B Omega``, ``Q = orth(Y)``, SVD of ``Q^T B`` truncated by the
  same rule.  Both return ``U = U_r Sigma_r`` and ``V = V_r``.
* Factorization (the paper factors ``F_pp^HODLR`` "using an HODLR solver", Section
  4.2.1): recursive Woodbury.  With ``D = diag(K_1, K_2)``, ``Z = diag(U, V)`` and
  ``S = [[0, I], [I, 0]]``, ``K = D + Z S Z^T`` and
  ``K^{-1} = D^{-1} - D^{-1} Z (S + Z^T D^{-1} Z)^{-1} Z^T D^{-1}``  (``S^{-1} = S``).
  The small core ``C = S + Z^T D^{-1} Z`` is symmetric indefinite: LU with partial
  pivoting.  Leaves: Cholesky.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


def hodlr_depth(n: int, leaf: int) -> int:
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    return L


def truncated_svd(B: np.ndarray, tol: float):
    """Rank-revealing truncation by the SVD: ``B ~ U V^T``, ``sigma_i > tol sigma_1``."""
    m, n = B.shape
    if m == 0 or n == 0:
        return np.zeros((m, 0)), np.zeros((n, 0))
    Us, s, Vh = np.linalg.svd(B, full_matrices=False)
    if s[0] == 0.0:
        return np.zeros((m, 0)), np.zeros((n, 0))
    r = int(np.count_nonzero(s > tol * s[0]))
    return Us[:, :r] * s[:r], Vh[:r, :].T.copy()


def randomized_range_finder(B: np.ndarray, tol: float, Omega: np.ndarray):
    """Randomized compression with a given sketch ``Omega`` (n x k):
    ``Y = B Omega``; ``Q`` = orthonormal basis of range(Y) (QR); ``Q^T B = Uh S Vh``;
    keep ``S_i > tol S_1``; ``U = Q Uh_r S_r``, ``V = Vh_r^T``."""
    m, n = B.shape
    if m == 0 or n == 0 or Omega.shape[1] == 0:
        return np.zeros((m, 0)), np.zeros((n, 0))
    Y = B @ Omega
    Q, _ = np.linalg.qr(Y)
    Bt = Q.T @ B
    Uh, s, Vh = np.linalg.svd(Bt, full_matrices=False)
    if s[0] == 0.0:
        return np.zeros((m, 0)), np.zeros((n, 0))
    r = int(np.count_nonzero(s > tol * s[0]))
    return Q @ (Uh[:, :r] * s[:r]), Vh[:r, :].T.copy()


@dataclass
class HNode:
    lo: int
    hi: int                       # rows [lo, hi) of the HODLR matrix
    level: int
    index: int                    # position among the nodes of its level
    children: list = field(default_factory=list)
    K: np.ndarray | None = None   # dense leaf block
    U: np.ndarray | None = None   # K_12 = U V^T, U rows of child 0
    V: np.ndarray | None = None   # V rows of child 1
    # factorization
    cho: tuple | None = None
    Zhat: np.ndarray | None = None
    core: tuple | None = None

    @property
    def rank(self) -> int:
        return 0 if self.U is None else int(self.U.shape[1])


def build(K: np.ndarray, leaf: int, tol: float, compressor=None) -> HNode:
    """HODLR representation of the dense symmetric matrix ``K``.

    ``compressor(B, level, index, lo=, mid=, hi=)`` returns ``(U, V)`` for the upper
    off-diagonal block ``K[lo:mid, mid:hi]`` of the node at (level, index); the default
    is ``truncated_svd(B, tol)``."""
    n = K.shape[0]
    L = hodlr_depth(n, leaf)
    if compressor is None:
        compressor = lambda B, level, index, **kw: truncated_svd(B, tol)  # noqa: E731

    def rec(lo, hi, level, index):
        node = HNode(lo, hi, level, index)
        if level == L:
            node.K = K[lo:hi, lo:hi].copy()
            return node
        mid = lo + (hi - lo) // 2
        node.children = [rec(lo, mid, level + 1, 2 * index), rec(mid, hi, level + 1, 2 * index + 1)]
        node.U, node.V = compressor(K[lo:mid, mid:hi], level, index, lo=lo, mid=mid, hi=hi)
        return node

    return rec(0, n, 0, 0)


def to_dense(node: HNode) -> np.ndarray:
    """The matrix the HODLR representation stands for (symmetric storage)."""
    if not node.children:
        return node.K.copy()
    a, b = node.children
    out = np.zeros((node.hi - node.lo, node.hi - node.lo))
    na = a.hi - a.lo
    out[:na, :na] = to_dense(a)
    out[na:, na:] = to_dense(b)
    B = node.U @ node.V.T
    out[:na, na:] = B
    out[na:, :na] = B.T
    return out


def factor(node: HNode) -> None:
    """Recursive Woodbury factorization (in place)."""
    if not node.children:
        node.cho = sla.cho_factor(node.K, lower=True)
        return
    a, b = node.children
    factor(a)
    factor(b)
    r = node.rank
    if r == 0:
        return
    na = a.hi - a.lo
    n = node.hi - node.lo
    Z = np.zeros((n, 2 * r))
    Z[:na, :r] = node.U
    Z[na:, r:] = node.V
    Zhat = np.vstack([solve(a, Z[:na]), solve(b, Z[na:])])      # D^{-1} Z
    S = np.zeros((2 * r, 2 * r))
    S[:r, r:] = np.eye(r)
    S[r:, :r] = np.eye(r)
    node.Zhat = Zhat
    node.core = sla.lu_factor(S + Z.T @ Zhat)


def solve(node: HNode, X: np.ndarray) -> np.ndarray:
    """``K^{-1} X`` by the recursive Woodbury formula."""
    if not node.children:
        return sla.cho_solve(node.cho, X)
    a, b = node.children
    na = a.hi - a.lo
    Y = np.concatenate([solve(a, X[:na]), solve(b, X[na:])], axis=0)   # D^{-1} X
    if node.rank == 0:
        return Y
    r = node.rank
    ZtY = np.concatenate([node.U.T @ Y[:na], node.V.T @ Y[na:]], axis=0)  # Z^T D^{-1} X
    return Y - node.Zhat @ sla.lu_solve(node.core, ZtY)


def iter_nodes(node: HNode):
    yield node
    for c in node.children:
        yield from iter_nodes(c)
