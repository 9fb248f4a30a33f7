"""Serving runtime (hm_server_*): requests for several matrices arriving together are
batched per matrix and run on concurrent workers; each result must equal, within the
stated tolerance, the answer the same request gets alone (the mix-vs-alone property),
with its own relative residual <= rtol.  The HBM budget admits matrices by evicting the
least recently used factorization, and a matrix that cannot fit alone fails cleanly."""
import numpy as np
import pytest

from fixtures import hex_cube, lognormal_coefficients, p1_jittered, q1_square, rhs_uniform

pytestmark = pytest.mark.gpu

try:
    import paper_1410_2697_gb300 as hm
except ImportError:  # the library is built on the GPU machine; a CPU-only machine skips
    import torch
    if torch.cuda.is_available():
        raise
    pytest.skip("CUDA library not built on this CPU-only machine", allow_module_level=True)

TOL = 1e-4


def matrices():
    return [q1_square(33, lognormal_coefficients(33 * 33, 1.0, seed=1)),
            q1_square(41, lognormal_coefficients(41 * 41, 1.0, seed=2)),
            hex_cube(9, lognormal_coefficients(9 ** 3, 0.5, seed=3)),
            p1_jittered(37, seed=5)]


def opts(budget=0):
    o = hm.hm_default_opts()
    o.nd_leaf, o.hodlr_leaf, o.n_c, o.samples = 16, 16, 16, 24
    o.hbm_budget = budget
    return o


def solve_alone(p, b):
    s = hm.Solver(p.n, p.rowptr, p.colidx, grid_coords=p.coords, dim=p.dim, nd_leaf=16, hodlr_leaf=16,
                  n_c=16, samples=24)
    s.factor(p.values, TOL)
    x = np.zeros_like(b)
    x, info = s.solve(b, rtol=1e-10, x=x)
    s.close()
    return x


def test_results_are_the_same_alone_and_in_the_mix():
    mats = matrices()
    srv = hm.hm_server_create(opts(), nworkers=2, max_batch_rhs=64)
    try:
        ids = [hm.hm_server_add_matrix(srv, p, TOL) for p in mats]
        rng = np.random.default_rng(7)
        reqs = []
        for k in range(24):  # submitted back to back: requests for one matrix share solves
            mi = int(rng.integers(0, len(mats)))
            nrhs = int(rng.integers(1, 9))
            b = np.asfortranarray(rhs_uniform(mats[mi].n, nrhs, 100 + k))
            x = np.zeros_like(b, order="F")
            reqs.append((mi, b, x, hm.hm_server_submit(srv, ids[mi], b, x)))
        for mi, b, x, rid in reqs:
            r = hm.hm_server_wait(srv, rid)
            assert r["status"] == hm.abi.HM_OK and r["converged"] == 1
            A = mats[mi].scipy()
            for c in range(b.shape[1]):
                assert np.linalg.norm(b[:, c] - A @ x[:, c]) / np.linalg.norm(b[:, c]) <= 1e-10
            xa = solve_alone(mats[mi], b)
            assert np.linalg.norm(x - xa) / np.linalg.norm(xa) <= 1e-8
        st = hm.hm_server_get_stats(srv)
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["factorizations"] == len(mats)
        assert st["batched_rhs"] == sum(b.shape[1] for _, b, _, _ in reqs)
        assert st["batches"] < len(reqs)  # some requests shared a solve
        assert 0 < st["p50_ms"] <= st["p99_ms"]
    finally:
        hm.hm_server_destroy(srv)


def test_budget_evicts_least_recently_used_factorizations():
    mats = matrices()[:3]
    # measure one worker's footprint of the largest matrix, then allow about one at a time
    probe = hm.hm_server_create(opts(), nworkers=1, max_batch_rhs=8)
    try:
        mid = hm.hm_server_add_matrix(probe, mats[1], TOL)
        b = np.asfortranarray(rhs_uniform(mats[1].n, 2, 1))
        x = np.zeros_like(b, order="F")
        assert hm.hm_server_wait(probe, hm.hm_server_submit(probe, mid, b, x))["status"] == hm.abi.HM_OK
        one = hm.hm_server_get_stats(probe)["device_bytes"]
    finally:
        hm.hm_server_destroy(probe)
    # room for the largest matrix with its solve workspace and little more (the
    # factorizations of the three do not fit together)
    srv = hm.hm_server_create(opts(int(1.05 * one)), nworkers=1, max_batch_rhs=8)
    try:
        ids = [hm.hm_server_add_matrix(srv, p, TOL) for p in mats]
        rounds = []
        for rnd in range(2):
            for mi in range(len(mats)):
                b = np.asfortranarray(rhs_uniform(mats[mi].n, 2, 10 * rnd + mi))
                x = np.zeros_like(b, order="F")
                r = hm.hm_server_wait(srv, hm.hm_server_submit(srv, ids[mi], b, x))
                assert r["status"] == hm.abi.HM_OK
                A = mats[mi].scipy()
                assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-9
            rounds.append(hm.hm_server_get_stats(srv))
        st = rounds[-1]
        assert st["evictions"] > rounds[0]["evictions"] > 0 and st["factorizations"] > len(mats)
        assert st["device_bytes"] <= 1.05 * one
        # admission by estimate: once every footprint is known, room is made before the
        # factorization, and no allocation runs into the budget
        assert st["oom_retries"] == rounds[0]["oom_retries"]
    finally:
        hm.hm_server_destroy(srv)


def test_matrix_larger_than_the_budget_fails_cleanly():
    srv = hm.hm_server_create(opts(1 << 16), nworkers=1, max_batch_rhs=4)  # 64 KiB
    try:
        p = matrices()[0]
        mid = hm.hm_server_add_matrix(srv, p, TOL)
        b = np.asfortranarray(rhs_uniform(p.n, 1, 3))
        x = np.zeros_like(b, order="F")
        r = hm.hm_server_wait(srv, hm.hm_server_submit(srv, mid, b, x))
        assert r["status"] == hm.abi.HM_ERR_OUT_OF_MEMORY
        assert hm.hm_server_get_stats(srv)["failed"] == 1
    finally:
        hm.hm_server_destroy(srv)


def test_request_joins_a_running_solve_and_matches_its_alone_result():
    """Continuous batching: request B for a matrix arrives while request A's GMRES on the
    same matrix is running (A needs several restart cycles of 10 at this loose
    compression tolerance).  B enters A's session at the next restart boundary (the server counts it
    as joined, and both are served by one session), both converge, and B's answer equals
    the answer B gets alone within 1e-8."""
    import time
    p = q1_square(120, lognormal_coefficients(120 * 120, 1.0, seed=11))
    tol = 3e-1  # a poor preconditioner: GMRES needs several restart cycles of 10
    o = opts()
    o.restart = 10
    srv = hm.hm_server_create(o, nworkers=1, max_batch_rhs=16)
    try:
        mid = hm.hm_server_add_matrix(srv, p, tol)
        warm_b = np.asfortranarray(rhs_uniform(p.n, 1, 1))
        warm_x = np.zeros_like(warm_b, order="F")
        hm.hm_server_wait(srv, hm.hm_server_submit(srv, mid, warm_b, warm_x))  # analyse + factor
        s0 = hm.hm_server_get_stats(srv)
        a_b = np.asfortranarray(rhs_uniform(p.n, 2, 2))
        a_x = np.zeros_like(a_b, order="F")
        ra = hm.hm_server_submit(srv, mid, a_b, a_x)
        t0 = time.time()
        while hm.hm_server_get_stats(srv)["batches"] == s0["batches"] and time.time() - t0 < 10:
            time.sleep(0.0005)  # until A's session runs
        b_b = np.asfortranarray(rhs_uniform(p.n, 1, 3))
        b_x = np.zeros_like(b_b, order="F")
        rb = hm.hm_server_submit(srv, mid, b_b, b_x)
        res_a = hm.hm_server_wait(srv, ra)
        res_b = hm.hm_server_wait(srv, rb)
        st = hm.hm_server_get_stats(srv)
        assert res_a["status"] == hm.abi.HM_OK and res_b["status"] == hm.abi.HM_OK
        assert res_a["iters"] > 20  # A ran several restart cycles
        assert st["joined"] >= 1 and st["batches"] == s0["batches"] + 1, st
        A = p.scipy()
        assert np.linalg.norm(b_b[:, 0] - A @ b_x[:, 0]) / np.linalg.norm(b_b[:, 0]) <= 1e-10
        s = hm.Solver(p.n, p.rowptr, p.colidx, grid_coords=p.coords, dim=p.dim, nd_leaf=16, hodlr_leaf=16,
                      n_c=16, samples=24, restart=10)
        s.factor(p.values, tol)
        xa = np.zeros_like(b_b)
        xa, _ = s.solve(b_b, rtol=1e-10, x=xa, max_iters=4000)
        s.close()
        assert np.linalg.norm(b_x - xa) / np.linalg.norm(xa) <= 1e-8
    finally:
        hm.hm_server_destroy(srv)


def _footprint(p, nrhs=2):
    """Device bytes one worker holds after serving one request of matrix p."""
    probe = hm.hm_server_create(opts(), nworkers=1, max_batch_rhs=8)
    try:
        mid = hm.hm_server_add_matrix(probe, p, TOL)
        b = np.asfortranarray(rhs_uniform(p.n, nrhs, 1))
        x = np.zeros_like(b, order="F")
        assert hm.hm_server_wait(probe, hm.hm_server_submit(probe, mid, b, x))["status"] == hm.abi.HM_OK
        return hm.hm_server_get_stats(probe)["device_bytes"]
    finally:
        hm.hm_server_destroy(probe)


def test_one_matrix_may_use_most_of_the_shared_budget():
    """The workers share one budget and one memory pool: with 2 workers and a budget of
    1.3 times one matrix's footprint, the matrix is served (a split of budget / workers
    would refuse it), and the bytes held stay within the budget."""
    p = matrices()[1]
    one = _footprint(p)
    budget = int(1.3 * one)
    srv = hm.hm_server_create(opts(budget), nworkers=2, max_batch_rhs=8)
    try:
        mid = hm.hm_server_add_matrix(srv, p, TOL)
        for k in range(3):
            b = np.asfortranarray(rhs_uniform(p.n, 2, 20 + k))
            x = np.zeros_like(b, order="F")
            r = hm.hm_server_wait(srv, hm.hm_server_submit(srv, mid, b, x))
            assert r["status"] == hm.abi.HM_OK
            assert np.linalg.norm(b - p.scipy() @ x) / np.linalg.norm(b) <= 1e-9
        st = hm.hm_server_get_stats(srv)
        assert st["failed"] == 0 and st["factorizations"] == 1
        assert st["device_bytes"] <= budget
    finally:
        hm.hm_server_destroy(srv)


def test_resident_matrix_moves_to_a_free_worker():
    """A matrix resident on a busy worker is served by the free one: its factorization
    moves to the free worker's context (shared pool) instead of being factored again or
    waiting.  Two long requests (relative tolerance 0: every column runs to the 4000
    iteration cap and ends HM_ERR_NO_CONVERGENCE) keep the workers busy in a known order:
    worker X takes A, worker Y factors B and then takes C; once A ends, X is free while
    Y still runs C, and the next request for B moves B to X.  B's answer equals its
    answer alone within 1e-8."""
    import time
    pa = q1_square(150, lognormal_coefficients(150 * 150, 1.0, seed=21))
    pc = q1_square(170, lognormal_coefficients(170 * 170, 1.0, seed=22))
    pb = matrices()[1]
    loose = 3e-1  # poor preconditioners for the long requests
    o = opts()
    o.restart = 10
    srv = hm.hm_server_create(o, nworkers=2, max_batch_rhs=8)
    try:
        ia = hm.hm_server_add_matrix(srv, pa, loose)
        ib = hm.hm_server_add_matrix(srv, pb, TOL)
        ic = hm.hm_server_add_matrix(srv, pc, loose)

        def submit(mid, p, seed, rtol=1e-10, nrhs=1):
            b = np.asfortranarray(rhs_uniform(p.n, nrhs, seed))
            x = np.zeros_like(b, order="F")
            return b, x, hm.hm_server_submit(srv, mid, b, x, rtol=rtol)

        def wait_batches(k):
            t0 = time.time()
            while hm.hm_server_get_stats(srv)["batches"] < k and time.time() - t0 < 30:
                time.sleep(0.0005)
            assert hm.hm_server_get_stats(srv)["batches"] >= k

        # every b and x stays referenced until its request has been waited for: the
        # server reads b and writes x from its worker threads
        ba, xa_, ra = submit(ia, pa, 1, rtol=0.0)       # X: A, runs to the cap
        wait_batches(1)
        b1, x1, rb1 = submit(ib, pb, 2)                 # Y: factor B, solve
        assert hm.hm_server_wait(srv, rb1)["status"] == hm.abi.HM_OK
        bc, xc, rc = submit(ic, pc, 3, rtol=0.0, nrhs=2)  # Y: C, runs to the cap (longer)
        wait_batches(3)
        res_a = hm.hm_server_wait(srv, ra)
        assert res_a["status"] == hm.abi.HM_ERR_NO_CONVERGENCE and res_a["iters"] >= 4000
        b2, x2, rb2 = submit(ib, pb, 4)                 # X is free, B lives on busy Y
        res_b = hm.hm_server_wait(srv, rb2)
        st = hm.hm_server_get_stats(srv)
        res_c = hm.hm_server_wait(srv, rc)
        assert res_b["status"] == hm.abi.HM_OK
        assert res_c["status"] == hm.abi.HM_ERR_NO_CONVERGENCE
        assert st["moved"] >= 1 and st["factorizations"] == 3, st
        A = pb.scipy()
        for b, x in ((b1, x1), (b2, x2)):
            assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-10
        xa = solve_alone(pb, b2)
        assert np.linalg.norm(x2 - xa) / np.linalg.norm(xa) <= 1e-8
    finally:
        hm.hm_server_destroy(srv)
