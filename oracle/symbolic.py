"""Symbolic multifrontal structure: coupling sets, frontal index sets, relative maps.

ORACLE / TEST INFRASTRUCTURE ONLY.

Section 4.1.1 of the paper:

* ``I_p`` -- the unknowns of tree node ``p`` (a contiguous range in the new order);
* ``S_p`` (Eq. couplingSet) -- unknowns ``j`` numbered after the last unknown of ``I_p``
  that are adjacent in the graph of ``A`` to some unknown of ``I_p``; adjacency is the
  structural pattern of the CSR matrix;
* ``I_p^f = S_p U (U_k I^U_{c_k}) minus I_p``, with ``I^U_c`` the index set of child
  ``c``'s update matrix, i.e. ``I^U_c = I_c^f``; sets are kept sorted ascending in the
  new numbering;
* the extend-add (the paper's circled plus) places entry ``t`` of a child's update at
  position ``relmap[t]`` of the parent's front, whose rows/columns are ``I_p`` followed
  by ``I_p^f``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .nd import ETree


@dataclass
class Symbolic:
    If: list            # per node: int32 array, sorted new indices of I_p^f
    relmap: list        # per node: int32 array, positions of I_p^f inside parent front
    children: list      # per node: list of child ids (ascending)

    def front_size(self, et: ETree, p: int) -> tuple[int, int]:
        return int(et.first[p + 1] - et.first[p]), int(self.If[p].shape[0])


def symbolic(rowptr: np.ndarray, colidx: np.ndarray, et: ETree) -> Symbolic:
    nf = et.nfronts
    children: list[list[int]] = [[] for _ in range(nf)]
    for c in range(nf):
        if et.parent[c] >= 0:
            children[int(et.parent[c])].append(c)
    If: list = [None] * nf
    for p in range(nf):  # postorder: children before parents
        b, e = int(et.first[p]), int(et.first[p + 1])
        old_rows = et.perm[b:e]
        nbrs = np.concatenate([colidx[rowptr[r]:rowptr[r + 1]] for r in old_rows]) if e > b \
            else np.zeros(0, np.int32)
        nbrs_new = et.iperm[nbrs]
        S_p = np.unique(nbrs_new[nbrs_new > e - 1])          # Eq. couplingSet
        parts = [S_p] + [If[c] for c in children[p]]
        union = np.unique(np.concatenate(parts)) if parts else np.zeros(0, np.int32)
        If[p] = union[(union < b) | (union >= e)].astype(np.int32)  # minus I_p
    relmap: list = [None] * nf
    for c in range(nf):
        p = int(et.parent[c])
        if p < 0:
            relmap[c] = np.zeros(0, np.int32)
            continue
        b, e = int(et.first[p]), int(et.first[p + 1])
        front = np.concatenate([np.arange(b, e, dtype=np.int64), If[p].astype(np.int64)])
        pos = {int(v): k for k, v in enumerate(front)}
        relmap[c] = np.asarray([pos[int(v)] for v in If[c]], dtype=np.int32)
    return Symbolic(If, relmap, children)
