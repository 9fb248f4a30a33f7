"""Philox4x32-10 counter-based generator and the sketch matrix drawn from it.

ORACLE / TEST INFRASTRUCTURE ONLY.

Philox4x32-10 is implemented from its published definition (Salmon, Moraes, Dror,
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
``(hi0, lo0) = mulhilo(M0, c0); (hi1, lo1) = mulhilo(M1, c2);
c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)`` with the key advanced by the Weyl
constants between rounds.  The randomized range finder of the method (the paper's
alternative to BDLR, Section 2.2) draws its sketch ``Omega`` from this generator; the
CUDA path implements the same published definition independently, so both sides see
bit-identical sketches.

Sketch entry convention: for a block with 64-bit id ``blk`` and seed ``seed``, entry
``Omega[i, c]`` uses counter ``(i, c, blk_lo, blk_hi)`` and key ``(seed_lo, seed_hi)``;
with ``w`` the output word 0, its value is ``((w >> 8) - 2^23) / 2^23``: uniform on a grid
of 2^24 points in [-1, 1), exactly representable in FP32 and FP64 (no rounding, so both
sides see identical sketches).  A continuous-like distribution keeps square sketches
invertible with overwhelming probability (a +-1 sketch is singular with noticeable
probability at small sizes).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10. All inputs uint32-compatible arrays (broadcast)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint32) for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0, k1 = k0.copy(), k1.copy()
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = (k0 + W0).astype(np.uint32)
                k1 = (k1 + W1).astype(np.uint32)
            p0 = M0 * c0.astype(np.uint64)
            p1 = M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def block_id(front: int, kind: int, level: int, node: int) -> int:
    """64-bit id of one compressed block: ``kind`` 0 = off-diagonal block of the pivot
    block's HODLR tree at (level, node), 1 = the front's F_fp block."""
    return (int(front) << 24) | (int(kind) << 20) | (int(level) << 16) | int(node)


def sketch(rows: int, cols: int, blk: int, seed: int) -> np.ndarray:
    """``rows x cols`` sketch matrix from Philox4x32-10 (convention above)."""
    i = np.arange(rows, dtype=np.uint32)[:, None]
    c = np.arange(cols, dtype=np.uint32)[None, :]
    blo = np.uint32(blk & 0xFFFFFFFF)
    bhi = np.uint32((blk >> 32) & 0xFFFFFFFF)
    slo = np.uint32(seed & 0xFFFFFFFF)
    shi = np.uint32((seed >> 32) & 0xFFFFFFFF)
    w0, _, _, _ = philox4x32_10(i, c, blo, bhi, slo, shi)
    return ((w0 >> np.uint32(8)).astype(np.float64) - 8388608.0) / 8388608.0
