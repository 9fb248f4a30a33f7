"""GB300 (sm_103a) HODLR-accelerated multifrontal preconditioner + GMRES.

A from-scratch CUDA implementation of the solver of Aminfar & Darve, "A Fast and
Memory Efficient Sparse Solver with Applications to Finite-Element Matrices"
(arXiv 1410.2697): nested-dissection multifrontal elimination whose large fronts are
HODLR matrices (randomized low-rank compression, recursive Woodbury factorization,
low-rank Schur complement and extend-add), used as the preconditioner of GMRES.

The C ABI (``include/hodlr_mf.h``) is the product boundary; :mod:`._binding` mirrors it
name for name, and :class:`Solver` is a small convenience wrapper over it.
"""
from __future__ import annotations

from . import _binding as abi  # noqa: F401  (raises if the CUDA library is missing)
from ._binding import (HM_PREC_FP64, HM_PREC_MIXED, HM_PREC_MIXED_BF16, HmError, hm_analyze,  # noqa: F401
                       hm_analyze_batch, hm_autotune, hm_create,
                       hm_ctx_destroy, hm_default_opts, hm_destroy, hm_direct_solve, hm_factor, hm_get_front_ranks,
                       hm_get_hodlr_block, hm_profile_enable, hm_profile_read,
                       hm_get_ordering, hm_get_sizes, hm_get_symbolic, hm_get_update,
                       hm_last_error, hm_precond_apply, hm_precond_apply_noalloc, hm_server_add_matrix,
                       hm_server_create, hm_server_destroy, hm_server_get_stats, hm_server_submit,
                       hm_server_wait, hm_solve, hm_status_str, hm_tune_force)


class Solver:
    """analyze -> factor -> solve on one problem (owns a context and a system)."""

    def __init__(self, n, rowptr, colidx, grid_coords=None, dim=0, precision=HM_PREC_MIXED,
                 nd_leaf=64, hodlr_leaf=64, n_c=64, samples=48, restart=30, seed=0x5EED, device=0,
                 stream=None, hbm_budget=0, perm=None, first=None, parent=None, **opts):
        o = hm_default_opts()
        o.device, o.precision, o.nd_leaf, o.hodlr_leaf = device, precision, nd_leaf, hodlr_leaf
        o.n_c, o.samples, o.restart, o.seed, o.hbm_budget = n_c, samples, restart, seed, hbm_budget
        o.stream = stream
        for k, v in opts.items():  # any other hm_opts field by name
            if k not in dict(type(o)._fields_):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.ctx = hm_create(o)
        self.n = int(n)
        try:
            if perm is not None:
                self.sys = hm_analyze(self.ctx, n, rowptr, colidx, 0, None, perm, len(parent), first,
                                      parent)
            else:
                self.sys = hm_analyze(self.ctx, n, rowptr, colidx, dim, grid_coords)
        except Exception:
            hm_ctx_destroy(self.ctx)
            self.ctx = None
            raise

    def factor(self, values, tol):
        return hm_factor(self.sys, values, tol)

    def solve(self, b, rtol=1e-10, max_iters=4000, x=None, nrhs=None):
        import numpy as np
        if nrhs is None:
            nrhs = 1 if b.ndim == 1 else b.shape[1] if isinstance(b, np.ndarray) else b.shape[0]
        if x is None:
            x = np.zeros_like(b)
        info = hm_solve(self.sys, nrhs, b, rtol, max_iters, x, raise_on_no_convergence=False)
        return x, info

    def precond(self, r, z, nrhs=1):
        hm_precond_apply(self.sys, nrhs, r, z)
        return z

    def close(self):
        if getattr(self, "sys", None) is not None:
            hm_destroy(self.sys)
            self.sys = None
        if getattr(self, "ctx", None) is not None:
            hm_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
