"""Geometric nested dissection and the elimination tree it induces.

ORACLE / TEST INFRASTRUCTURE ONLY.

Section 4.1.1 of the paper: unknowns are eliminated in the order imposed by the
elimination tree; each tree node owns a set of unknowns ``I_p`` that cannot be
eliminated before those of its children.  The paper does not fix the ordering; this
oracle uses the following rule (shared, as a specification, with the CUDA path):

* a box is a set of interior lattice points ``[lo_d, hi_d]`` (inclusive) per axis;
* a box is a leaf if it holds at most ``leaf_size`` points or its longest extent is
  below 3;
* otherwise it is split along its longest axis (ties go to the lowest axis, x < y < z)
  by the one-point-thick plane ``mid = (lo + hi) // 2``; the lower half, then the
  upper half, are ordered recursively, then the separator plane;
* the points of a leaf box and of a separator are ordered lexicographically with x
  fastest;
* tree nodes are numbered in postorder (lower subtree, upper subtree, separator), a
  separator's children are the roots of its two half-boxes, ``parent[root] = -1``.

Every lattice point of the bounding box must be an unknown (full grids).

Vector problems (``dofs_per_node`` b > 1, e.g. 3D elasticity): unknown ``b k + d`` is
component d of node k, and all b components share the node's lattice point.  The rule
above is applied to the nodes (leaf test: at most ``leaf_size // b`` nodes), and every
node is then expanded into its b unknowns, consecutive in the new numbering, so that
separators hold whole nodes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ETree:
    perm: np.ndarray      # int32 (n,): new index -> original index
    iperm: np.ndarray     # int32 (n,): original index -> new index
    first: np.ndarray     # int32 (nf+1,): node p owns new indices [first[p], first[p+1])
    parent: np.ndarray    # int32 (nf,): postorder parent, -1 at the root
    level: np.ndarray     # int32 (nf,): depth (root 0)

    @property
    def nfronts(self) -> int:
        return int(self.parent.shape[0])

    def children(self, p: int) -> list[int]:
        return [int(c) for c in np.nonzero(self.parent == p)[0]]


def _box_points(lo, hi, lattice_to_old, ext):
    """Original indices of the box's points in lexicographic order, x fastest."""
    axes = [np.arange(l, h + 1) for l, h in zip(lo, hi)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
    coords = [g.reshape(-1) for g in grids[::-1]]   # back to (x, y, z)
    lin = np.zeros_like(coords[0])
    stride = 1
    for d in range(len(ext)):
        lin = lin + coords[d] * stride
        stride *= ext[d]
    return lattice_to_old[lin]


def nested_dissection(coords: np.ndarray, leaf_size: int = 64, dofs_per_node: int = 1) -> ETree:
    """Postorder separator tree and permutation for unknowns at lattice ``coords``."""
    if dofs_per_node > 1:
        b = dofs_per_node
        coords = np.asarray(coords, dtype=np.int64)
        if coords.shape[0] % b or np.any(coords.reshape(-1, b, coords.shape[1]) != coords[::b, None, :]):
            raise ValueError("nested_dissection: the b unknowns of a node must be consecutive and share coords")
        et = nested_dissection(coords[::b], max(1, leaf_size // b))
        d = np.arange(b, dtype=np.int32)
        perm = (b * et.perm[:, None] + d[None, :]).reshape(-1).astype(np.int32)
        iperm = np.empty_like(perm)
        iperm[perm] = np.arange(perm.shape[0], dtype=np.int32)
        return ETree(perm, iperm, (b * et.first).astype(np.int32), et.parent, et.level)
    coords = np.asarray(coords, dtype=np.int64)
    n, dim = coords.shape
    lo0 = coords.min(axis=0)
    ext = tuple(int(v) for v in (coords.max(axis=0) - lo0 + 1))
    rel = coords - lo0
    lin = np.zeros(n, dtype=np.int64)
    stride = 1
    for d in range(dim):
        lin += rel[:, d] * stride
        stride *= ext[d]
    if stride != n or np.unique(lin).shape[0] != n:
        raise ValueError("nested_dissection: unknowns must fill their bounding lattice box")
    lattice_to_old = np.empty(n, dtype=np.int64)
    lattice_to_old[lin] = np.arange(n)

    perm_parts: list[np.ndarray] = []
    sizes: list[int] = []
    parents: list[int] = []
    levels: list[int] = []

    def visit(lo, hi, depth):
        """Order the box; return the postorder id of its root node."""
        extents = [h - l + 1 for l, h in zip(lo, hi)]
        count = int(np.prod(extents))
        longest = max(extents)
        if count <= leaf_size or longest < 3:
            perm_parts.append(_box_points(lo, hi, lattice_to_old, ext))
            sizes.append(count)
            parents.append(-1)
            levels.append(depth)
            return len(sizes) - 1
        axis = extents.index(longest)  # first maximum = lowest axis on ties
        mid = (lo[axis] + hi[axis]) // 2
        lo_l, hi_l = list(lo), list(hi)
        hi_l[axis] = mid - 1
        lo_r, hi_r = list(lo), list(hi)
        lo_r[axis] = mid + 1
        left = visit(lo_l, hi_l, depth + 1)
        right = visit(lo_r, hi_r, depth + 1)
        lo_s, hi_s = list(lo), list(hi)
        lo_s[axis] = mid
        hi_s[axis] = mid
        perm_parts.append(_box_points(lo_s, hi_s, lattice_to_old, ext))
        sizes.append(int(np.prod([h - l + 1 for l, h in zip(lo_s, hi_s)])))
        parents.append(-1)
        levels.append(depth)
        me = len(sizes) - 1
        parents[left] = me
        parents[right] = me
        return me

    visit([0] * dim, [e - 1 for e in ext], 0)
    perm = np.concatenate(perm_parts).astype(np.int32)
    iperm = np.empty(n, dtype=np.int32)
    iperm[perm] = np.arange(n, dtype=np.int32)
    first = np.zeros(len(sizes) + 1, dtype=np.int32)
    first[1:] = np.cumsum(sizes)
    return ETree(perm, iperm, first, np.asarray(parents, dtype=np.int32),
                 np.asarray(levels, dtype=np.int32))
