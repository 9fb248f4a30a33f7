"""Pins of the oracle against facts fixed by mathematics, not by the oracle itself.

Each test names what it pins and why a plausible slip in the oracle would fail it.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spl

from fixtures import hex_cube, hex_elasticity, p1_jittered, q1_square, rhs_uniform, lognormal_coefficients
from oracle import dense_mf, gmres, hodlr, hodlr_mf, nd, symbolic
from oracle.philox import philox4x32_10, sketch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- fixtures
@pytest.mark.parametrize("m", [5, 6, 9])
def test_q1_closed_form_eigenvalues(m):
    """Constant-coefficient Q1 stiffness: lambda_jk = 2/3 (4 - c_j - c_k - 2 c_j c_k),
    c_j = cos(j pi h) -- a wrong element matrix or a dropped entry moves them."""
    p = q1_square(m)
    h = 1.0 / m
    c = np.cos(np.arange(1, m) * np.pi * h)
    lam = (2.0 / 3.0) * (4 - c[:, None] - c[None, :] - 2 * c[:, None] * c[None, :])
    ev = np.linalg.eigvalsh(p.scipy().toarray())
    np.testing.assert_allclose(np.sort(ev), np.sort(lam.ravel()), atol=1e-13)
    assert p.nnz == (3 * (m - 1) - 2) ** 2


@pytest.mark.parametrize("m", [4, 6])
def test_hex_closed_form_eigenvalues(m):
    """Trilinear hex: lambda = 2h/9 [(1-c_j)(2+c_k)(2+c_l) + perms]."""
    p = hex_cube(m)
    h = 1.0 / m
    c = np.cos(np.arange(1, m) * np.pi * h)
    cj, ck, cl = c[:, None, None], c[None, :, None], c[None, None, :]
    lam = (2 * h / 9) * ((1 - cj) * (2 + ck) * (2 + cl) + (2 + cj) * (1 - ck) * (2 + cl)
                         + (2 + cj) * (2 + ck) * (1 - cl))
    ev = np.linalg.eigvalsh(p.scipy().toarray())
    np.testing.assert_allclose(np.sort(ev), np.sort(lam.ravel()), atol=1e-13)
    assert p.nnz == (3 * (m - 1) - 2) ** 3


def test_elasticity_element_closed_forms():
    """Trilinear-hex elasticity element: (i) nu = 0 diagonal entry = 2/9 on the unit cube
    (E times the x-part of the hex Laplacian diagonal, 1/9, plus mu = 1/2 times its y and
    z parts, 2/9); (ii) the null space is exactly the 6 rigid-body motions; (iii) scaling
    with Young's modulus and side h."""
    from fixtures.meshes import _hex_elasticity_ke
    K0 = _hex_elasticity_ke(0.0)
    assert abs(K0[0, 0] - 2.0 / 9.0) < 1e-14
    K = _hex_elasticity_ke(0.3)
    assert np.abs(K - K.T).max() < 1e-15
    x = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    modes = []
    for c in range(3):  # translations
        u = np.zeros((8, 3)); u[:, c] = 1.0; modes.append(u.reshape(-1))
    for w in np.eye(3):  # infinitesimal rotations u = w x x
        modes.append(np.cross(w, x).reshape(-1))
    R = np.array(modes).T
    assert np.abs(K @ R).max() < 1e-14
    ev = np.linalg.eigvalsh(K)
    assert np.all(np.abs(ev[:6]) < 1e-14) and ev[6] > 1e-2
    p1, p2 = hex_elasticity(3), hex_elasticity(3, 2.5 * np.ones(27))
    np.testing.assert_allclose(p2.values, 2.5 * p1.values, rtol=1e-13, atol=1e-15)


def test_elasticity_patch_test():
    """Constant strain is exact: with uniform moduli the full (unclamped) operator
    applied to an affine displacement field vanishes at every interior node; a quadratic
    field does not (so the check sees the assembly)."""
    m = 5
    p = hex_elasticity(m, 1.7 * np.ones(m ** 3), nu=0.27, dirichlet=False)
    nodes = p.coords[::3].astype(float) / m
    G = np.array([[0.3, -1.1, 0.2], [0.5, 0.1, -0.4], [-0.7, 0.9, 0.6]])
    u = (nodes @ G.T + np.array([0.1, -0.2, 0.3])).reshape(-1)
    r = (p.scipy() @ u).reshape(-1, 3)
    inner = np.all((p.coords[::3] > 0) & (p.coords[::3] < m), axis=1)
    assert np.abs(r[inner]).max() < 1e-12 * np.abs(p.values).max()
    q = (nodes ** 2 @ G.T).reshape(-1)
    assert np.abs((p.scipy() @ q).reshape(-1, 3)[inner]).max() > 1e-3


def test_p1_mesh_spd_and_consistent():
    """P1 element matrices annihilate constants: interior rows away from the boundary
    sum to zero; the reduced matrix is symmetric positive definite."""
    p = p1_jittered(12, seed=5)
    A = p.scipy()
    assert abs(A - A.T).max() < 1e-14
    assert np.linalg.eigvalsh(A.toarray()).min() > 0
    ii, jj = p.coords[:, 0], p.coords[:, 1]
    deep = (ii > 0) & (ii < p.extents[0] - 1) & (jj > 0) & (jj < p.extents[1] - 1)
    rs = np.asarray(A.sum(axis=1)).ravel()
    assert np.abs(rs[deep]).max() < 1e-12
    assert np.abs(rs[~deep]).min() > 0  # boundary-adjacent rows keep a positive sum


def test_lognormal_and_rhs_are_seeded():
    a = lognormal_coefficients(100, 1.0, seed=1)
    b = lognormal_coefficients(100, 1.0, seed=1)
    assert np.array_equal(a, b) and np.all(a > 0)
    r = rhs_uniform(50, 3, 2)
    assert r.shape == (50, 3) and r.flags.f_contiguous and np.abs(r).max() <= 1


# ----------------------------------------------------------------------------- philox
def test_philox_known_answer_vectors():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_sketch_is_uniform_grid_and_keyed():
    a = sketch(200, 50, 7, 11)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert np.all(a * 8388608.0 == np.round(a * 8388608.0))           # 24-bit grid
    assert np.array_equal(a, a.astype(np.float32).astype(np.float64))  # exact in FP32
    assert abs(a.mean()) < 0.05 and abs(a.var() - 1.0 / 3.0) < 0.02
    assert not np.array_equal(a, sketch(200, 50, 8, 11))
    assert np.array_equal(a[:10, :5], sketch(10, 5, 7, 11))


# ----------------------------------------------------------------------------- ND + symbolic
def _dense_symbolic_cholesky(Ap):
    """Structure of the Cholesky factor by boolean elimination (brute force)."""
    M = (Ap.toarray() != 0) | np.eye(Ap.shape[0], dtype=bool)
    # structural pattern: use the CSR pattern, not values
    M = np.zeros(Ap.shape, dtype=bool)
    coo = Ap.tocoo()
    M[coo.row, coo.col] = True
    n = M.shape[0]
    for j in range(n):
        rows = np.nonzero(M[j + 1:, j])[0] + j + 1
        if rows.size:
            M[np.ix_(rows, rows)] = True
    return np.tril(M)


@pytest.mark.parametrize("maker", [lambda: q1_square(10), lambda: q1_square(13),
                                   lambda: hex_cube(6), lambda: p1_jittered(11, 9),
                                   lambda: hex_elasticity(5, lognormal_coefficients(125, 0.5, seed=3))])
def test_nd_and_front_sets_match_brute_force_fill(maker):
    """I_p^f equals the rows (after I_p) of the Cholesky fill of P A P^T in the
    columns of I_p; the permutation is one; the tree is a postorder; the two halves
    below a separator are not adjacent (vector problems: with whole nodes)."""
    p = maker()
    bdof = p.meta.get("dofs_per_node", 1)
    et = nd.nested_dissection(p.coords, leaf_size=8 * bdof, dofs_per_node=bdof)
    if bdof > 1:  # a node's components stay consecutive, in component order
        assert np.all(et.perm.reshape(-1, bdof) == et.perm[::bdof, None] + np.arange(bdof))
        assert np.all(et.first % bdof == 0)
    assert np.array_equal(np.sort(et.perm), np.arange(p.n))
    assert np.array_equal(et.iperm[et.perm], np.arange(p.n))
    nf = et.nfronts
    assert et.parent[-1] == -1 and np.all(et.parent[:-1] > np.arange(nf - 1))
    sym = symbolic.symbolic(p.rowptr, p.colidx, et)
    Ap = dense_mf.permuted_matrix(p.rowptr, p.colidx, p.values, et)
    L = _dense_symbolic_cholesky(Ap)
    owner = np.searchsorted(et.first, np.arange(p.n), side="right") - 1
    for q in range(nf):
        b, e = et.first[q], et.first[q + 1]
        rows = np.nonzero(L[e:, b:e].any(axis=1))[0] + e
        assert np.array_equal(rows, sym.If[q]), q
        # relmap places the child's update inside the parent front
        if et.parent[q] >= 0:
            par = et.parent[q]
            front = dense_mf.front_indices(et, sym, par)
            assert np.array_equal(front[sym.relmap[q]], sym.If[q])
    # separators separate: no edge between distinct subtrees of a separator
    A = Ap.tocoo()
    for q in range(nf):
        ch = sym.children[q]
        if len(ch) == 2:
            def subtree(c):
                s = {c}
                for k in range(c, -1, -1):
                    if et.parent[k] in s:
                        s.add(k)
                return s
            s0, s1 = subtree(ch[0]), subtree(ch[1])
            o_r, o_c = owner[A.row], owner[A.col]
            bad = np.isin(o_r, list(s0)) & np.isin(o_c, list(s1))
            assert not bad.any()


def test_nd_rule_on_a_hand_checked_grid():
    """7x7 interior grid, leaf 4, worked by hand from the stated rule: the root splits
    x at 3 (tie -> x); each 3x7 half splits y at 3; each 3x3 quarter splits x at 1 into
    two 1x3 leaves.  Postorder: leaf, leaf, separator, ..., root."""
    p = q1_square(8)  # 7x7 interior
    et = nd.nested_dissection(p.coords, leaf_size=4)
    parent = [2, 2, 6, 5, 5, 6, 14, 9, 9, 13, 12, 12, 13, 14, -1]
    assert et.parent.tolist() == parent
    assert et.first.tolist() == [0, 3, 6, 9, 12, 15, 18, 21, 24, 27, 30, 33, 36, 39, 42, 49]
    y3 = np.arange(3)
    expect = {
        0: [(0, y) for y in y3], 1: [(2, y) for y in y3], 2: [(1, y) for y in y3],
        3: [(0, y + 4) for y in y3], 4: [(2, y + 4) for y in y3], 5: [(1, y + 4) for y in y3],
        6: [(x, 3) for x in y3],
        7: [(4, y) for y in y3], 8: [(6, y) for y in y3], 9: [(5, y) for y in y3],
        10: [(4, y + 4) for y in y3], 11: [(6, y + 4) for y in y3], 12: [(5, y + 4) for y in y3],
        13: [(x + 4, 3) for x in y3], 14: [(3, y) for y in range(7)],
    }
    for q, pts in expect.items():
        got = p.coords[et.perm[et.first[q]:et.first[q + 1]]]
        assert [tuple(v) for v in got.tolist()] == pts, q
    assert et.level.tolist() == [3, 3, 2, 3, 3, 2, 1, 3, 3, 2, 3, 3, 2, 1, 0]


# ----------------------------------------------------------------------------- dense MF
@pytest.mark.parametrize("maker", [lambda: q1_square(12), lambda: hex_cube(5),
                                   lambda: p1_jittered(10, 3), lambda: hex_elasticity(4)])
def test_dense_mf_equals_global_cholesky(maker):
    """Front factors are the blocks of numpy's Cholesky of P A P^T (Eq. update is the
    Schur complement), and the solve inverts A."""
    p = maker()
    bdof = p.meta.get("dofs_per_node", 1)
    et = nd.nested_dissection(p.coords, leaf_size=8 * bdof, dofs_per_node=bdof)
    sym = symbolic.symbolic(p.rowptr, p.colidx, et)
    Ap = dense_mf.permuted_matrix(p.rowptr, p.colidx, p.values, et)
    Lg = np.linalg.cholesky(Ap.toarray())
    fronts, _ = dense_mf.factor(Ap, et, sym)
    for q, fr in enumerate(fronts):
        b, e = et.first[q], et.first[q + 1]
        Lpp = np.tril(fr.cho[0])
        np.testing.assert_allclose(Lpp, Lg[b:e, b:e], atol=1e-12)
        Lfp = sla.solve_triangular(Lpp, fr.Ffp.T, lower=True).T
        np.testing.assert_allclose(Lfp, Lg[sym.If[q]][:, b:e], atol=1e-12)
    rng = np.random.default_rng(0)
    xs = rng.standard_normal(p.n)
    A = p.scipy()
    x = dense_mf.direct_solve(p.rowptr, p.colidx, p.values, p.coords, A @ xs, leaf_size=8 * bdof, dofs_per_node=bdof)
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-10 * np.abs(xs).max())


# ----------------------------------------------------------------------------- HODLR
def _random_spd_hodlr(n, leaf, r, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) / np.sqrt(n)
    K = X @ X.T + np.eye(n)
    return K


def test_truncated_svd_eckart_young():
    rng = np.random.default_rng(1)
    B = rng.standard_normal((60, 40)) @ np.diag(0.5 ** np.arange(40)) @ rng.standard_normal((40, 40))
    for tol in [1e-2, 1e-6]:
        U, V = hodlr.truncated_svd(B, tol)
        s = np.linalg.svd(B, compute_uv=False)
        r = U.shape[1]
        assert s[r - 1] > tol * s[0] >= s[r]
        err = np.linalg.norm(B - U @ V.T, 2)
        assert abs(err - s[r]) <= 1e-10 * s[0]


def test_rrf_exact_on_low_rank_and_bounded():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((80, 7)) @ rng.standard_normal((7, 90))
    Om = sketch(90, 17, 1, 3)
    U, V = hodlr.randomized_range_finder(B, 1e-12, Om)
    assert U.shape[1] == 7
    np.testing.assert_allclose(U @ V.T, B, atol=1e-10 * np.abs(B).max())
    # decaying spectrum: error within a small multiple of tol * sigma_1
    C = rng.standard_normal((100, 60)) @ np.diag(0.6 ** np.arange(60)) @ rng.standard_normal((60, 70))
    s1 = np.linalg.norm(C, 2)
    U, V = hodlr.randomized_range_finder(C, 1e-4, sketch(70, 40, 2, 3))
    assert np.linalg.norm(C - U @ V.T, 2) <= 10 * 1e-4 * s1


@pytest.mark.parametrize("n,leaf", [(256, 32), (200, 16), (64, 64), (130, 20)])
def test_woodbury_solve_matches_dense(n, leaf):
    """Recursive Woodbury inverse of a HODLR matrix equals the dense inverse of the
    matrix it represents (tol 0: the representation is exact, so also of K)."""
    K = _random_spd_hodlr(n, leaf, 5, n)
    H = hodlr.build(K, leaf, 0.0)
    np.testing.assert_allclose(hodlr.to_dense(H), K, atol=1e-12)
    hodlr.factor(H)
    X = np.random.default_rng(3).standard_normal((n, 3))
    np.testing.assert_allclose(hodlr.solve(H, X), np.linalg.solve(K, X), rtol=1e-9, atol=1e-10)
    # compressed: equals the inverse of the represented (approximate) matrix
    H2 = hodlr.build(K, leaf, 1e-2)
    Kd = hodlr.to_dense(H2)
    hodlr.factor(H2)
    np.testing.assert_allclose(hodlr.solve(H2, X), np.linalg.solve(Kd, X), rtol=1e-8, atol=1e-9)


def test_hodlr_partition_depth():
    assert hodlr.hodlr_depth(64, 64) == 0
    assert hodlr.hodlr_depth(65, 64) == 1
    assert hodlr.hodlr_depth(1023, 64) == 4
    H = hodlr.build(np.eye(1023), 64, 0.0)
    leaves = [nd_ for nd_ in hodlr.iter_nodes(H) if not nd_.children]
    assert len(leaves) == 16 and max(l.hi - l.lo for l in leaves) <= 64
    assert {l.level for l in leaves} == {4}


# ----------------------------------------------------------------------------- HODLR-MF
def _setup(p, leaf_nd=64):
    et = nd.nested_dissection(p.coords, leaf_nd)
    sym = symbolic.symbolic(p.rowptr, p.colidx, et)
    Ap = dense_mf.permuted_matrix(p.rowptr, p.colidx, p.values, et)
    return et, sym, Ap


def test_hodlr_mf_tol0_is_exact_direct_solve():
    """tol 0 keeps every nonzero singular value: the preconditioner is A^{-1} and GMRES
    converges in one iteration."""
    p = q1_square(48, lognormal_coefficients(48 * 48, 1.0, seed=1))
    et, sym, Ap = _setup(p, 16)
    prm = hodlr_mf.Params(tol=0.0, n_c=8, leaf=8)
    fr, _ = hodlr_mf.factor(Ap, et, sym, prm)
    assert any(f.kind == "hodlr" for f in fr)
    r = np.random.default_rng(0).standard_normal((p.n, 2))
    x = hodlr_mf.apply(fr, et, sym, r)
    np.testing.assert_allclose(Ap @ x, r, atol=1e-9)
    xg, info = gmres.gmres(lambda v: Ap @ v, lambda v: hodlr_mf.apply(fr, et, sym, v), r[:, 0])
    assert info["iters"] == 1 and info["relres"] < 1e-10


def test_hodlr_mf_preconditioner_is_symmetric_and_close():
    """M^{-1} built from symmetric HODLR pieces is symmetric; with tol 1e-3 it is a
    good approximation (||I - M^{-1}A|| < 1) and GMRES reaches 1e-10."""
    p = q1_square(32, lognormal_coefficients(32 * 32, 1.0, seed=4))
    et, sym, Ap = _setup(p, 16)
    prm = hodlr_mf.Params(tol=1e-3, n_c=8, leaf=8)
    fr, _ = hodlr_mf.factor(Ap, et, sym, prm)
    Minv = hodlr_mf.apply(fr, et, sym, np.eye(p.n))
    np.testing.assert_allclose(Minv, Minv.T, atol=1e-10 * np.abs(Minv).max())
    E = np.eye(p.n) - Minv @ Ap.toarray()
    assert np.linalg.norm(E, 2) < 0.5
    b = rhs_uniform(p.n, 1, 0)[:, 0]
    x, info = gmres.gmres(lambda v: Ap @ v, lambda v: hodlr_mf.apply(fr, et, sym, v), b)
    assert info["converged"]
    xs = spl.spsolve(Ap.tocsc(), b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8


def test_hodlr_mf_rrf_matches_svd_iterations():
    p = q1_square(64)
    et, sym, Ap = _setup(p)
    b = rhs_uniform(p.n, 1, 0)[:, 0][et.perm]
    its = []
    for comp in ["svd", "rrf"]:
        prm = hodlr_mf.Params(tol=1e-6, n_c=16, leaf=16, compressor=comp, samples=40)
        fr, _ = hodlr_mf.factor(Ap, et, sym, prm)
        x, info = gmres.gmres(lambda v: Ap @ v, lambda v: hodlr_mf.apply(fr, et, sym, v), b)
        assert info["converged"]
        its.append(info["iters"])
    assert abs(its[0] - its[1]) <= 1


# ----------------------------------------------------------------------------- GMRES
def test_gmres_unpreconditioned_matches_solve():
    p = q1_square(12)
    A = p.scipy()
    b = rhs_uniform(p.n, 1, 3)[:, 0]
    x, info = gmres.gmres(lambda v: A @ v, lambda v: v, b, rtol=1e-12, restart=10)
    assert info["converged"]
    np.testing.assert_allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-9)
    h = np.array(info["history"])
    # within one cycle the rotated residual estimate never increases
    for c in range(0, len(h), 10):
        seg = h[c:c + 10]
        assert np.all(np.diff(seg) <= 1e-15)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-12


# ----------------------------------------------------------------------------- BDLR
def test_bdlr_distances_are_graph_distances():
    """BDLR's breadth-first distances equal unweighted shortest-path lengths (SciPy's
    csgraph) from the source set, capped at depth + 1."""
    from scipy.sparse.csgraph import shortest_path
    from oracle import bdlr
    p = q1_square(12, lognormal_coefficients(144, 1.0, seed=2))
    et = nd.nested_dissection(p.coords, 16)
    sym = symbolic.symbolic(p.rowptr, p.colidx, et)
    Ap = dense_mf.permuted_matrix(p.rowptr, p.colidx, p.values, et)
    q = int(np.argmax(et.first[1:] - et.first[:-1]))  # the largest front
    G = bdlr.front_graph(Ap, dense_mf.front_indices(et, sym, q))
    src = np.arange(0, 3)
    D = shortest_path(G, unweighted=True, indices=src).min(axis=0)
    for depth in (1, 2, 4):
        d = bdlr.distances(G, src, depth)
        ref = np.where(D <= depth, D, depth + 1).astype(int)
        assert np.array_equal(d, ref), depth


def test_bdlr_complete_pivoting_hand_example_and_rank_rule():
    """B = [[1, 2], [3, 4]]: first pivot 4 at (1, 1), multiplier 1/2, Schur pivot -1/2,
    L U = B(p, q); with eps = 0.2 the ratio 0.5 / 4 < eps stops at rank 1."""
    from oracle import bdlr
    B = np.array([[1.0, 2.0], [3.0, 4.0]])
    pr, pc, L, U = bdlr.complete_pivoting_lu(B, 0.0)
    assert pr.tolist() == [1, 0] and pc.tolist() == [1, 0]
    np.testing.assert_allclose(L, [[1.0, 0.0], [0.5, 1.0]], atol=1e-15)
    np.testing.assert_allclose(U, [[4.0, 3.0], [0.0, -0.5]], atol=1e-15)
    np.testing.assert_allclose(L @ U, B[np.ix_(pr, pc)], atol=1e-15)
    assert bdlr.complete_pivoting_lu(B, 0.2)[0].tolist() == [1]


def test_bdlr_skeleton_exact_on_low_rank_blocks():
    """With every row and column selected, the skeleton B(:, J_q) B^^-1 B(I_p, :) of an
    exactly rank-5 block reproduces it (rank found = 5), and eps truncates by pivots."""
    from oracle import bdlr
    rng = np.random.default_rng(4)
    B = rng.standard_normal((40, 5)) @ rng.standard_normal((5, 30))
    U, V = bdlr.compress(B, np.arange(40), np.arange(30), 1e-12)
    assert U.shape[1] == 5
    np.testing.assert_allclose(U @ V.T, B, atol=1e-10 * np.abs(B).max())
    # a few rows and columns suffice when they span the block's rows and columns
    U2, V2 = bdlr.compress(B, np.arange(0, 40, 5), np.arange(0, 30, 4), 1e-12)
    np.testing.assert_allclose(U2 @ V2.T, B, atol=1e-10 * np.abs(B).max())


def test_hodlr_mf_with_bdlr_converges():
    """The HODLR-MF preconditioner with BDLR blocks (depth 1 and 2) lets GMRES reach
    1e-10 in far fewer iterations than unpreconditioned GMRES (BDLR reads the graph of A
    on the front's unknowns only, so its blocks are approximate even at eps = 0: fill
    rows out of the graph's reach enter only through B(:, J))."""
    p = q1_square(24, lognormal_coefficients(576, 1.0, seed=6))
    et = nd.nested_dissection(p.coords, 16)
    sym = symbolic.symbolic(p.rowptr, p.colidx, et)
    Ap = dense_mf.permuted_matrix(p.rowptr, p.colidx, p.values, et)
    b = rhs_uniform(p.n, 1, 7)[:, 0][et.perm]
    _, none = gmres.gmres(lambda v: Ap @ v, lambda v: v, b, 1e-10, 30, max_iters=4000)
    for depth in (1, 2):
        prm = hodlr_mf.Params(tol=1e-4, n_c=8, leaf=8, compressor="bdlr", samples=48, bdlr_depth=depth)
        fr, _ = hodlr_mf.factor(Ap, et, sym, prm)
        x, info = gmres.gmres(lambda v: Ap @ v, lambda v: hodlr_mf.apply(fr, et, sym, v), b, 1e-10, 30)
        assert info["converged"] and info["relres"] <= 1e-10
        assert 3 * info["iters"] < none["iters"], (depth, info["iters"], none["iters"])


def test_bdlr_select_orders_by_distance_then_position_and_caps_last():
    """Hand-worked selection on an 8-vertex graph, X = {0, 1, 2, 3}, Y = {4, 5, 6, 7},
    edges 0-4, 3-5, 0-1, 2-3, 4-6, 6-7.  Distances to Y: vertex 0 -> 1 (edge 0-4),
    3 -> 1 (3-5), 1 -> 2 (via 0), 2 -> 2 (via 3).  Distances to X: 4 -> 1, 5 -> 1,
    6 -> 2 (via 4), 7 -> 3.  Ordered by distance, then position: I = [0, 3, 1, 2],
    J = [0, 1, 2] (7 is beyond depth 2).  The cap applies after that ordering: cap 3
    gives I = [0, 3, 1] -- ordering by position first ([0, 1, 2]) or cutting to the cap
    before filtering by distance would both give another list."""
    import scipy.sparse as sp
    from oracle import bdlr
    e = np.array([[0, 4], [3, 5], [0, 1], [2, 3], [4, 6], [6, 7]])
    G = sp.coo_matrix((np.ones(12), (np.r_[e[:, 0], e[:, 1]], np.r_[e[:, 1], e[:, 0]])), shape=(8, 8)).tocsr()
    X, Y = np.arange(4), np.arange(4, 8)
    I, J = bdlr.select(G, X, Y, 2, 8)
    assert I.tolist() == [0, 3, 1, 2] and J.tolist() == [0, 1, 2]
    I, J = bdlr.select(G, X, Y, 2, 3)
    assert I.tolist() == [0, 3, 1] and J.tolist() == [0, 1, 2]
    I, J = bdlr.select(G, X, Y, 2, 2)
    assert I.tolist() == [0, 3] and J.tolist() == [0, 1]
    I, J = bdlr.select(G, X, Y, 1, 8)  # depth 1: only the direct neighbours
    assert I.tolist() == [0, 3] and J.tolist() == [0, 1]


def test_hodlr_mf_compress_ff_update_is_hodlr_of_f_ff():
    """compress_ff=True (the paper's F_ff^HODLR, Section 4.2.1): the update of every
    HODLR front is U_p = H(F_ff) - W T W^T.  Adding W T W^T back must give a matrix whose
    leaf diagonal blocks equal F_ff's exactly and whose off-diagonal blocks are F_ff's
    truncated at tol (Eckart-Young with the SVD compressor: 2-norm error = the first
    dropped singular value <= tol sigma_1).  At tol 0 nothing is dropped and the
    preconditioner is A^{-1}."""
    p = q1_square(40, lognormal_coefficients(40 * 40, 1.0, seed=3))
    et, sym, Ap = _setup(p, 16)
    tol = 1e-3
    prm = hodlr_mf.Params(tol=tol, n_c=8, leaf=8, compress_ff=True)
    fr, tr = hodlr_mf.factor(Ap, et, sym, prm, keep=True)
    checked = 0
    for q, f in enumerate(fr):
        if f.kind != "hodlr" or f.W.shape[0] == 0:
            continue
        npv = f.npiv
        Fff = tr["F"][q][npv:, npv:]
        T = f.V.T @ hodlr.solve(f.H, f.V)
        Hff = tr["U"][q] + f.W @ T @ f.W.T       # = to_dense(H(F_ff))
        ref = hodlr.build(Fff, prm.leaf, 0.0)    # the partition, blocks exact
        for node in hodlr.iter_nodes(ref):
            if node.children:
                a, b = node.children[0], node.children[1]
                B = Fff[a.lo:a.hi, b.lo:b.hi]
                E = Hff[a.lo:a.hi, b.lo:b.hi] - B
                s = np.linalg.svd(B, compute_uv=False)
                assert np.linalg.norm(E, 2) <= tol * s[0] * (1 + 1e-9) + 1e-12, (q, node.level)
                np.testing.assert_allclose(Hff[b.lo:b.hi, a.lo:a.hi], Hff[a.lo:a.hi, b.lo:b.hi].T, atol=1e-12)
            else:
                np.testing.assert_allclose(Hff[node.lo:node.hi, node.lo:node.hi],
                                           Fff[node.lo:node.hi, node.lo:node.hi], atol=1e-10 * np.abs(Fff).max())
        checked += 1
    assert checked > 0
    prm0 = hodlr_mf.Params(tol=0.0, n_c=8, leaf=8, compress_ff=True)
    fr0, _ = hodlr_mf.factor(Ap, et, sym, prm0)
    r = np.random.default_rng(1).standard_normal((p.n, 2))
    np.testing.assert_allclose(Ap @ hodlr_mf.apply(fr0, et, sym, r), r, atol=1e-9)


def test_kappa_estimate_matches_closed_form_spectrum():
    """Q1 Poisson: lambda_min and lambda_max from the closed-form eigenvalues.  Lanczos
    Ritz values approach the extreme eigenvalues from below: lambda_max(A^{-1}) =
    1 / lambda_min converges fast (well separated at the bottom of the spectrum), the
    top of the spectrum is clustered so lambda_max(A) only to about a percent; the
    Gershgorin row sum bounds lambda_max from above."""
    from oracle import condest
    m = 24
    p = q1_square(m)
    h = 1.0 / m
    c = np.cos(np.arange(1, m) * np.pi * h)
    lam = (2.0 / 3.0) * (4 - c[:, None] - c[None, :] - 2 * c[:, None] * c[None, :])
    A = p.scipy()
    lu = spl.splu(A.tocsc())
    inv_max = condest.lanczos_max(lu.solve, p.n, 40, seed=3)
    assert abs(inv_max * lam.min() - 1.0) <= 1e-8
    top = condest.lanczos_max(lambda v: A @ v, p.n, 60, seed=3)
    assert 0.99 * lam.max() <= top <= lam.max() * (1 + 1e-12)
    assert condest.gershgorin_max(A) >= lam.max()
    k = condest.kappa_estimate(A, lu.solve, 60, seed=3)
    kappa = lam.max() / lam.min()
    assert 0.99 * kappa <= k <= kappa * (1 + 1e-8)


def test_hodlr_mf_adaptive_width_meets_the_tolerance_rule():
    """Adaptive rank (Section 2.2: the rank is set by the tolerance, not by the sketch):
    with a 4-column sketch most blocks of this problem have more than 4 singular values
    above tol sigma_1, so the fixed-width range finder truncates them far above tol;
    doubling the width of every level that holds a capped block until none is capped
    brings every block (checked against its SVD) to within 2 tol sigma_1, the range
    finder's error with a one-column oversampling margin at worst."""
    p = q1_square(48, lognormal_coefficients(48 * 48, 1.0, seed=5))
    et, sym, Ap = _setup(p, 16)
    tol = 1e-6
    worst = {}
    for adaptive in (False, True):
        prm = hodlr_mf.Params(tol=tol, n_c=8, leaf=8, compressor="rrf", samples=4, adaptive=adaptive)
        fr, tr = hodlr_mf.factor(Ap, et, sym, prm, keep=True)
        w = 0.0
        for q, f in enumerate(fr):
            if f.kind != "hodlr":
                continue
            F, npv = tr["F"][q], f.npiv
            width = tr["widths"].get(int(et.level[q]), 4)
            blocks = [(F[npv:, :npv], f.W, f.V)] if f.W.shape[0] else []
            for node in hodlr.iter_nodes(f.H):
                if node.children:
                    a, b = node.children
                    blocks.append((F[a.lo:a.hi, b.lo:b.hi], node.U, node.V))
            for B, U, V in blocks:
                s = np.linalg.svd(B, compute_uv=False)
                w = max(w, np.linalg.norm(B - U @ V.T, 2) / s[0])
                if adaptive:  # no block is cut by its width any more
                    assert U.shape[1] < min(width, *B.shape) or width >= min(B.shape), (q, U.shape, width)
        worst[adaptive] = w
        if adaptive:
            assert max(tr["widths"].values()) > 4
            assert all(v <= 96 for v in tr["widths"].values())
    assert worst[False] > 1e3 * tol
    assert worst[True] <= 2 * tol, worst
