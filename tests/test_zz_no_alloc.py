"""The allocation-free preconditioner apply (hm_precond_apply_noalloc).

Callers whose device memory belongs to another allocator (or who must not wait on the
driver's allocator) use this entry point instead of hm_precond_apply; it keeps its
per-call temporaries in a fixed file-scope device array.  Checked through the C ABI
against the allocating entry point, on two calls in a row.  This file is collected last
so that a run stopping at the first failure has run every other test already.
"""
import numpy as np
import pytest

from fixtures import lognormal_coefficients, q1_square, rhs_uniform

pytestmark = pytest.mark.gpu

try:
    import paper_1410_2697_gb300 as hm
except ImportError:  # the library is built on the GPU machine; a CPU-only machine skips
    import torch
    if torch.cuda.is_available():
        raise
    pytest.skip("CUDA library not built on this CPU-only machine", allow_module_level=True)

import torch  # noqa: E402

RTOL = 1e-12  # same kernels in the same order as hm_precond_apply


@pytest.mark.parametrize("precision", [hm.HM_PREC_FP64, hm.HM_PREC_MIXED])
def test_noalloc_apply_matches_allocating_apply(precision):
    p = q1_square(40, lognormal_coefficients(40 * 40, 1.0, seed=1))
    s = hm.Solver(p.n, p.rowptr, p.colidx, grid_coords=p.coords, dim=2, precision=precision,
                  nd_leaf=16, hodlr_leaf=16, n_c=16, samples=24)
    try:
        s.factor(p.values, 1e-6)
        nrhs = 3
        rs = [rhs_uniform(p.n, nrhs, seed) for seed in (11, 12)]
        refs = []
        for r in rs:  # the allocating entry point (also creates the per-nrhs workspace)
            z = np.zeros_like(r)
            hm.hm_precond_apply(s.sys, nrhs, r, z)
            refs.append(z)
        for r, ref in zip(rs, refs):  # two allocation-free calls in a row
            d_r = torch.from_numpy(np.ascontiguousarray(r.T)).cuda()
            d_z = torch.full_like(d_r, float("nan"))
            # the call runs on the library's own stream: r must be on the device first
            torch.cuda.synchronize()
            hm.hm_precond_apply_noalloc(s.sys, nrhs, d_r, d_z)
            torch.cuda.synchronize()
            z = d_z.cpu().numpy().T
            err = np.abs(z - ref).max() / np.abs(ref).max()
            assert err <= RTOL, err
    finally:
        s.close()


def test_noalloc_apply_rejects_what_it_cannot_do_without_allocating():
    p = q1_square(80)  # 6241 unknowns: 64 right-hand sides exceed the fixed scratch
    s = hm.Solver(p.n, p.rowptr, p.colidx, grid_coords=p.coords, dim=2,
                  precision=hm.HM_PREC_MIXED, nd_leaf=16, hodlr_leaf=16, n_c=16, samples=24)
    try:
        s.factor(p.values, 1e-4)
        big = torch.zeros((64, p.n), dtype=torch.float64, device="cuda")
        with pytest.raises(hm.HmError) as e:
            hm.hm_precond_apply_noalloc(s.sys, 64, big, big.clone())
        assert e.value.status == hm.abi.HM_ERR_CAPACITY
        one = torch.zeros((2, p.n), dtype=torch.float64, device="cuda")
        with pytest.raises(hm.HmError) as e:  # no workspace for nrhs = 2 yet
            hm.hm_precond_apply_noalloc(s.sys, 2, one, one.clone())
        assert e.value.status == hm.abi.HM_ERR_STATE
        r = rhs_uniform(p.n, 2, 3)
        z = np.zeros_like(r)
        hm.hm_precond_apply(s.sys, 2, r, z)
        with pytest.raises(hm.HmError) as e:  # host pointers are refused
            hm.hm_precond_apply_noalloc(s.sys, 2, r, np.zeros_like(r))
        assert e.value.status == hm.abi.HM_ERR_INVALID_ARG
    finally:
        s.close()
