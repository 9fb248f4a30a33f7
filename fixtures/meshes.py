"""Finite-element problem generators (inputs only).

The paper solves ``A x = b`` with ``A`` a symmetric positive definite finite-element
stiffness matrix of an elliptic PDE (Section 1).  Its own matrices (cylinder head,
FETI-DP) are not available, so these generators build synthetic stand-ins with the
same structure: scalar diffusion ``-div(k grad u) = f`` on structured 2D/3D grids and
on jittered unstructured triangle meshes, Dirichlet boundary nodes eliminated.

Conventions shared by every generator
-------------------------------------
* Unknowns are the interior lattice nodes, numbered lexicographically x-fastest.
* ``coords`` are the integer lattice coordinates of each unknown (0-based over the
  interior), int32, shape ``(n, dim)``; the unstructured P1 meshes still live on a
  logical ``(i, j)`` lattice (nodes are jittered, connectivity is not).
* CSR: ``rowptr`` int64 ``(n+1,)``, ``colidx`` int32 sorted per row, ``values`` FP64.
  The pattern is the element-connectivity pattern (entries that cancel to an exact
  zero, e.g. face neighbours of the trilinear hex, are kept as structural entries).
* Random numbers come from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    name: str
    n: int
    dim: int
    rowptr: np.ndarray  # int64 (n+1,)
    colidx: np.ndarray  # int32 (nnz,)
    values: np.ndarray  # float64 (nnz,)
    coords: np.ndarray  # int32 (n, dim) interior lattice coordinates
    extents: tuple  # interior lattice extents per axis
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.values, self.colidx, self.rowptr), shape=(self.n, self.n))


def lognormal_coefficients(n_elems: int, sigma: float, mu: float = 0.0, seed: int | None = None,
                           rng: np.random.Generator | None = None) -> np.ndarray:
    """Piecewise-constant coefficient ``k_e = exp(mu + sigma z_e)``, z_e ~ N(0,1) i.i.d.,
    one per element in lexicographic element order."""
    if rng is None:
        rng = np.random.Generator(np.random.PCG64(seed))
    if sigma == 0.0:
        return np.full(n_elems, np.exp(mu))
    return np.exp(mu + sigma * rng.standard_normal(n_elems))


def rhs_uniform(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Right-hand sides with i.i.d. U[-1, 1] entries, column-major ``(n, nrhs)``.

    Column k is the k-th length-n draw from the seeded stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    return np.asfortranarray(b.T)


def _assemble(n_nodes_total: int, conn: np.ndarray, ke: np.ndarray, interior_index: np.ndarray,
              n: int):
    """Sum element matrices ``ke[e]`` (E, a, a) over connectivity ``conn`` (E, a) and keep
    interior rows/columns (Dirichlet nodes eliminated)."""
    E, a = conn.shape
    rows = np.repeat(conn, a, axis=1).reshape(-1)
    cols = np.tile(conn, (1, a)).reshape(-1)
    vals = ke.reshape(-1)
    ri = interior_index[rows]
    ci = interior_index[cols]
    keep = (ri >= 0) & (ci >= 0)
    m = sp.coo_matrix((vals[keep], (ri[keep], ci[keep])), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return (m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64))


# Q1 bilinear element on a square, nodes counter-clockwise from the lower-left corner.
_Q1_KE = np.array([[4, -1, -2, -1],
                   [-1, 4, -1, -2],
                   [-2, -1, 4, -1],
                   [-1, -2, -1, 4]], dtype=np.float64) / 6.0


def q1_square(m: int, coef: np.ndarray | None = None, name: str | None = None) -> Problem:
    """2D Q1 bilinear diffusion on the unit square with ``m x m`` elements (h = 1/m).

    Interior unknowns ``(m-1)^2``; the element matrix of a square element is
    h-independent: ``k/6 [[4,-1,-2,-1],[-1,4,-1,-2],[-2,-1,4,-1],[-1,-2,-1,4]]``."""
    if coef is None:
        coef = np.ones(m * m)
    coef = np.asarray(coef, dtype=np.float64)
    assert coef.shape == (m * m,)
    nn = m + 1
    ex, ey = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    ex = ex.reshape(-1)
    ey = ey.reshape(-1)  # element e = ex + m*ey (x-fastest)
    node = lambda i, j: i + nn * j  # noqa: E731
    conn = np.stack([node(ex, ey), node(ex + 1, ey), node(ex + 1, ey + 1), node(ex, ey + 1)], axis=1)
    ke = coef[:, None, None] * _Q1_KE[None, :, :]
    gi, gj = np.meshgrid(np.arange(nn), np.arange(nn), indexing="xy")
    gi = gi.reshape(-1)
    gj = gj.reshape(-1)
    interior = (gi > 0) & (gi < m) & (gj > 0) & (gj < m)
    n = (m - 1) ** 2
    interior_index = np.full(nn * nn, -1, dtype=np.int64)
    interior_index[interior] = (gi[interior] - 1) + (m - 1) * (gj[interior] - 1)
    rowptr, colidx, values = _assemble(nn * nn, conn, ke, interior_index, n)
    ii, jj = np.meshgrid(np.arange(m - 1), np.arange(m - 1), indexing="xy")
    coords = np.stack([ii.reshape(-1), jj.reshape(-1)], axis=1).astype(np.int32)
    return Problem(name or f"q1_square_{m}", n, 2, rowptr, colidx, values, coords,
                   (m - 1, m - 1), {"m": m, "h": 1.0 / m})


def _hex_ke() -> np.ndarray:
    """Trilinear hex Laplacian element matrix for a unit-coefficient cube of side 1,
    local node a = dx + 2 dy + 4 dz:  4/12 on the diagonal, 0 for edge neighbours,
    -1/12 for face and body diagonals."""
    M = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            d = bin(a ^ b).count("1")
            M[a, b] = {0: 4.0, 1: 0.0, 2: -1.0, 3: -1.0}[d]
    return M / 12.0


def hex_cube(m: int, coef: np.ndarray | None = None, name: str | None = None) -> Problem:
    """3D trilinear-hex diffusion on the unit cube with ``m^3`` elements (h = 1/m);
    element matrix ``k h/12 M``.  Interior unknowns ``(m-1)^3``."""
    if coef is None:
        coef = np.ones(m ** 3)
    coef = np.asarray(coef, dtype=np.float64)
    assert coef.shape == (m ** 3,)
    h = 1.0 / m
    nn = m + 1
    ez, ey, ex = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ex = ex.reshape(-1)
    ey = ey.reshape(-1)
    ez = ez.reshape(-1)  # element e = ex + m*ey + m*m*ez
    node = lambda i, j, k: i + nn * (j + nn * k)  # noqa: E731
    conn = np.stack([node(ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1)) for a in range(8)],
                    axis=1)
    ke = (coef * h)[:, None, None] * _hex_ke()[None, :, :]
    gk, gj, gi = np.meshgrid(np.arange(nn), np.arange(nn), np.arange(nn), indexing="ij")
    gi = gi.reshape(-1)
    gj = gj.reshape(-1)
    gk = gk.reshape(-1)
    interior = (gi > 0) & (gi < m) & (gj > 0) & (gj < m) & (gk > 0) & (gk < m)
    n = (m - 1) ** 3
    interior_index = np.full(nn ** 3, -1, dtype=np.int64)
    interior_index[interior] = (gi[interior] - 1) + (m - 1) * ((gj[interior] - 1) + (m - 1) * (gk[interior] - 1))
    rowptr, colidx, values = _assemble(nn ** 3, conn, ke, interior_index, n)
    kk, jj, ii = np.meshgrid(np.arange(m - 1), np.arange(m - 1), np.arange(m - 1), indexing="ij")
    coords = np.stack([ii.reshape(-1), jj.reshape(-1), kk.reshape(-1)], axis=1).astype(np.int32)
    return Problem(name or f"hex_cube_{m}", n, 3, rowptr, colidx, values, coords,
                   (m - 1, m - 1, m - 1), {"m": m, "h": h})


def _hex_elasticity_ke(nu: float) -> np.ndarray:
    """24 x 24 stiffness of isotropic linear elasticity (Young's modulus 1, Poisson ratio
    nu) on a trilinear cube element of side 1, by 2 x 2 x 2 Gauss quadrature (exact for
    this element); local node a = dx + 2 dy + 4 dz, unknown 3 a + c for component c.
    For side h it scales by h."""
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2.0 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    g = 1.0 / np.sqrt(3.0)
    K = np.zeros((24, 24))
    sa = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1] for a in range(8)], float)
    for xi in (-g, g):
        for eta in (-g, g):
            for zeta in (-g, g):
                p = np.array([xi, eta, zeta])
                # dN_a/dx on the unit cube (x = (xi + 1) / 2): 2 * dN_a/dxi
                dN = np.empty((8, 3))
                for a in range(8):
                    f = 1.0 + sa[a] * p
                    dN[a, 0] = sa[a, 0] * f[1] * f[2] / 8.0 * 2.0
                    dN[a, 1] = sa[a, 1] * f[0] * f[2] / 8.0 * 2.0
                    dN[a, 2] = sa[a, 2] * f[0] * f[1] / 8.0 * 2.0
                B = np.zeros((6, 24))
                for a in range(8):
                    dx, dy, dz = dN[a]
                    c = 3 * a
                    B[0, c] = dx
                    B[1, c + 1] = dy
                    B[2, c + 2] = dz
                    B[3, c], B[3, c + 1] = dy, dx
                    B[4, c + 1], B[4, c + 2] = dz, dy
                    B[5, c], B[5, c + 2] = dz, dx
                K += B.T @ D @ B * (1.0 / 8.0)  # Gauss weight 1, Jacobian (1/2)^3
    return K


def hex_elasticity(m: int, young: np.ndarray | None = None, nu: float = 0.3, name: str | None = None,
                   dirichlet: bool = True) -> Problem:
    """3D linear elasticity (3 displacement components per node) on the unit cube with
    ``m^3`` trilinear hex elements, Young's modulus ``young[e]`` per element, Poisson
    ratio ``nu``.  Every boundary node is clamped (eliminated): ``3 (m-1)^3`` unknowns,
    unknown ``3 k + c`` = component c of interior node k (nodes lexicographic, x fastest);
    all three components carry their node's lattice coordinates (``meta['dofs_per_node']``
    = 3).  ``dirichlet=False`` keeps every node (the singular operator, for patch tests)."""
    if young is None:
        young = np.ones(m ** 3)
    young = np.asarray(young, dtype=np.float64)
    assert young.shape == (m ** 3,)
    h = 1.0 / m
    nn = m + 1
    ez, ey, ex = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ex, ey, ez = ex.reshape(-1), ey.reshape(-1), ez.reshape(-1)
    node = lambda i, j, k: i + nn * (j + nn * k)  # noqa: E731
    nconn = np.stack([node(ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1)) for a in range(8)], axis=1)
    conn = (3 * nconn[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)
    ke = (young * h)[:, None, None] * _hex_elasticity_ke(nu)[None, :, :]
    gk, gj, gi = np.meshgrid(np.arange(nn), np.arange(nn), np.arange(nn), indexing="ij")
    gi, gj, gk = gi.reshape(-1), gj.reshape(-1), gk.reshape(-1)
    if dirichlet:
        keep = (gi > 0) & (gi < m) & (gj > 0) & (gj < m) & (gk > 0) & (gk < m)
        lo, ext = 1, m - 1
    else:
        keep = np.ones(nn ** 3, dtype=bool)
        lo, ext = 0, nn
    node_index = np.full(nn ** 3, -1, dtype=np.int64)
    node_index[keep] = (gi[keep] - lo) + ext * ((gj[keep] - lo) + ext * (gk[keep] - lo))
    nodes = ext ** 3
    dof_index = np.where(node_index[:, None] >= 0, 3 * node_index[:, None] + np.arange(3)[None, :], -1).reshape(-1)
    rowptr, colidx, values = _assemble(3 * nn ** 3, conn, ke, dof_index, 3 * nodes)
    kk, jj, ii = np.meshgrid(np.arange(ext), np.arange(ext), np.arange(ext), indexing="ij")
    ncoords = np.stack([ii.reshape(-1), jj.reshape(-1), kk.reshape(-1)], axis=1).astype(np.int32)
    coords = np.repeat(ncoords, 3, axis=0)
    return Problem(name or f"hex_elasticity_{m}", 3 * nodes, 3, rowptr, colidx, values, coords,
                   (ext, ext, ext), {"m": m, "h": h, "nu": nu, "dofs_per_node": 3})


def p1_jittered(n_cells: int, seed: int, sigma: float = 1.0, jitter: float = 0.3,
                name: str | None = None) -> Problem:
    """Unstructured 2D P1 triangle mesh: an ``n x n`` cell grid on the unit square,
    interior nodes jittered by U[-jitter h, jitter h] per coordinate, each cell split
    along a random diagonal, lognormal coefficient (sigma) per triangle.

    Element matrix ``k * area * G G^T`` with G the gradients of the barycentric
    functions.  Draw order from one seeded stream: jitter (x then y for every node,
    node-major), diagonal choices (one per cell), coefficients (one per triangle)."""
    n = n_cells
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    nn = n + 1
    gi, gj = np.meshgrid(np.arange(nn), np.arange(nn), indexing="xy")
    gi = gi.reshape(-1)
    gj = gj.reshape(-1)
    jit = rng.uniform(-jitter * h, jitter * h, size=(nn * nn, 2))
    interior = (gi > 0) & (gi < n) & (gj > 0) & (gj < n)
    x = gi * h + np.where(interior, jit[:, 0], 0.0)
    y = gj * h + np.where(interior, jit[:, 1], 0.0)
    diag = rng.integers(0, 2, size=n * n)  # 0: lower-left to upper-right, 1: other
    ex, ey = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    ex = ex.reshape(-1)
    ey = ey.reshape(-1)
    node = lambda i, j: i + nn * j  # noqa: E731
    n00, n10, n11, n01 = node(ex, ey), node(ex + 1, ey), node(ex + 1, ey + 1), node(ex, ey + 1)
    t1 = np.where(diag[:, None] == 0, np.stack([n00, n10, n11], 1), np.stack([n00, n10, n01], 1))
    t2 = np.where(diag[:, None] == 0, np.stack([n00, n11, n01], 1), np.stack([n10, n11, n01], 1))
    tri = np.stack([t1, t2], axis=1).reshape(-1, 3)  # triangle 2e, 2e+1 of cell e
    coef = lognormal_coefficients(tri.shape[0], sigma, rng=rng)
    px, py = x[tri], y[tri]
    d11 = px[:, 1] - px[:, 0]
    d12 = px[:, 2] - px[:, 0]
    d21 = py[:, 1] - py[:, 0]
    d22 = py[:, 2] - py[:, 0]
    det = d11 * d22 - d12 * d21
    area = 0.5 * np.abs(det)
    # grad(lambda_1), grad(lambda_2) are the rows of inv([[d11, d12], [d21, d22]])
    g1 = np.stack([d22, -d12], 1) / det[:, None]
    g2 = np.stack([-d21, d11], 1) / det[:, None]
    g0 = -(g1 + g2)
    G = np.stack([g0, g1, g2], axis=1)  # (T, 3, 2)
    ke = (coef * area)[:, None, None] * np.einsum("tad,tbd->tab", G, G)
    nint = (n - 1) ** 2
    interior_index = np.full(nn * nn, -1, dtype=np.int64)
    interior_index[interior] = (gi[interior] - 1) + (n - 1) * (gj[interior] - 1)
    rowptr, colidx, values = _assemble(nn * nn, tri, ke, interior_index, nint)
    ii, jj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="xy")
    coords = np.stack([ii.reshape(-1), jj.reshape(-1)], axis=1).astype(np.int32)
    return Problem(name or f"p1_jittered_{n}_s{seed}", nint, 2, rowptr, colidx, values, coords,
                   (n - 1, n - 1), {"n_cells": n, "h": h, "min_det": float(det.min())})


# ---------------------------------------------------------------------------------------
# Named workloads (sizes, distributions and seeds of the benchmark configurations)
# ---------------------------------------------------------------------------------------

def _cfg_poisson64():
    p = q1_square(64, name="q1_poisson_64x64")
    return p, {"tol": 1e-6, "leaf": 64, "n_c": 64, "restart": 30, "rtol": 1e-10, "rhs_seed": 0,
               "nrhs": 1}


def _cfg_lognormal1024(m: int = 1024):
    coef = lognormal_coefficients(m * m, sigma=1.0, mu=0.0, seed=1)
    p = q1_square(m, coef, name=f"q1_lognormal_{m}x{m}")
    return p, {"tol": 1e-4, "leaf": 64, "n_c": 64, "restart": 30, "rtol": 1e-10, "rhs_seed": 2,
               "nrhs": 16}


def _cfg_hex64(m: int = 64):
    coef = lognormal_coefficients(m ** 3, sigma=0.5, mu=0.0, seed=3)
    p = hex_cube(m, coef, name=f"hex_lognormal_{m}^3")
    return p, {"tol": 1e-4, "leaf": 64, "n_c": 64, "restart": 30, "rtol": 1e-10, "rhs_seed": 4,
               "nrhs": 1}


def _cfg_elasticity40(m: int = 40):
    young = lognormal_coefficients(m ** 3, sigma=0.5, mu=0.0, seed=51)
    p = hex_elasticity(m, young, nu=0.3, name=f"elasticity_hex_{m}^3")
    return p, {"tol": 1e-4, "leaf": 64, "n_c": 64, "restart": 30, "rtol": 1e-10, "rhs_seed": 52,
               "nrhs": 1}


WORKLOADS = {
    "q1_poisson_64x64": _cfg_poisson64,
    "q1_lognormal_1024x1024": _cfg_lognormal1024,
    "hex_lognormal_64^3": _cfg_hex64,
    "elasticity_hex_40^3": _cfg_elasticity40,
}


def workload(name: str, **kw):
    """Return ``(Problem, params)`` for a named workload; ``kw`` may shrink sizes
    (e.g. ``m=128``) for tests."""
    return WORKLOADS[name](**kw)


def p1_batch_sizes(count: int = 256, seed: int = 5) -> np.ndarray:
    """Cell counts ``n ~ U{32..256}`` for the batch of unstructured meshes; mesh i then
    uses seed ``seed + i`` for its own geometry and coefficients."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(32, 257, size=count)


def block_diagonal(problems: list) -> tuple:
    """Independent meshes as one block-diagonal problem: ``(Problem, block_ptr)`` with
    mesh b's unknowns at ``[block_ptr[b], block_ptr[b+1])`` (each keeps its own lattice
    coordinates)."""
    block_ptr = np.zeros(len(problems) + 1, dtype=np.int32)
    for b, p in enumerate(problems):
        block_ptr[b + 1] = block_ptr[b] + p.n
    rowptr = [np.zeros(1, dtype=np.int64)]
    colidx, values, coords = [], [], []
    nnz = 0
    for b, p in enumerate(problems):
        rowptr.append(p.rowptr[1:] + nnz)
        colidx.append(p.colidx + block_ptr[b])
        values.append(p.values)
        coords.append(p.coords)
        nnz += p.nnz
    dims = {p.dim for p in problems}
    assert len(dims) == 1
    prob = Problem(f"batch_{len(problems)}", int(block_ptr[-1]), dims.pop(), np.concatenate(rowptr),
                   np.concatenate(colidx).astype(np.int32), np.concatenate(values),
                   np.ascontiguousarray(np.concatenate(coords)), (), {"blocks": len(problems)})
    return prob, block_ptr


def p1_batch(count: int = 256, seed: int = 5) -> tuple:
    """The batch of unstructured P1 meshes: mesh i has ``n ~ U{32..256}`` cells per side
    (from ``p1_batch_sizes``), geometry and coefficients from seed ``seed + i``.  Returns
    ``(Problem, block_ptr, meshes)``."""
    sizes = p1_batch_sizes(count, seed)
    meshes = [p1_jittered(int(nc), seed=seed + i) for i, nc in enumerate(sizes)]
    prob, block_ptr = block_diagonal(meshes)
    return prob, block_ptr, meshes
