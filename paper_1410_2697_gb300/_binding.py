"""ctypes binding of ``include/hodlr_mf.h`` -- argument marshalling only.

Every function here forwards to the C entry point of the same name in the in-tree
``libhodlr_mf.so``; all computation happens in its CUDA kernels.  Arrays may be numpy
arrays (host) or torch CUDA tensors (device); the library detects which.  There is no
fallback: if the library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhodlr_mf.so")

HM_OK = 0
HM_ERR_INVALID_ARG = 1
HM_ERR_NOT_SPD = 2
HM_ERR_NO_CONVERGENCE = 3
HM_ERR_OUT_OF_MEMORY = 4
HM_ERR_CUDA = 5
HM_ERR_CAPACITY = 6
HM_ERR_DEVICE_TIMEOUT = 7
HM_ERR_STATE = 8
HM_ERR_BREAKDOWN = 9
HM_PREC_FP64 = 0
HM_PREC_MIXED = 1
HM_PREC_MIXED_BF16 = 2
HM_COMP_RRF, HM_COMP_BDLR = 0, 1

EXPORTED = ["hm_default_opts", "hm_create", "hm_ctx_destroy", "hm_analyze", "hm_analyze_batch", "hm_get_sizes",
            "hm_get_ordering", "hm_get_symbolic", "hm_factor", "hm_autotune", "hm_tune_force", "hm_solve", "hm_direct_solve",
            "hm_precond_apply",
            "hm_precond_apply_noalloc",
            "hm_get_update", "hm_get_front_ranks", "hm_get_hodlr_block", "hm_profile_enable", "hm_profile_read", "hm_destroy", "hm_status_str", "hm_last_error",
            "hm_server_create", "hm_server_add_matrix", "hm_server_submit", "hm_server_wait",
            "hm_server_get_stats", "hm_server_destroy"]


class HmOpts(C.Structure):
    _fields_ = [("device", C.c_int), ("precision", C.c_int), ("nd_leaf", C.c_int),
                ("hodlr_leaf", C.c_int), ("n_c", C.c_int), ("samples", C.c_int),
                ("seed", C.c_uint64), ("restart", C.c_int), ("hbm_budget", C.c_size_t),
                ("stream", C.c_void_p), ("dofs_per_node", C.c_int), ("compressor", C.c_int),
                ("bdlr_depth", C.c_int), ("wait_limit", C.c_int), ("adaptive_rank", C.c_int),
                ("inject_wait_timeout", C.c_int),
                ("compress_ff", C.c_int), ("keep_fronts", C.c_int)]


class HmSolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("relres", C.c_double),
                ("converged", C.c_int32)]


class HmFactorInfo(C.Structure):
    _fields_ = [("nfronts", C.c_int32), ("nlevels", C.c_int32), ("n_hodlr", C.c_int32),
                ("max_rank", C.c_int32), ("rank_capped", C.c_int32), ("factor_bytes", C.c_double),
                ("front_bytes", C.c_double), ("refactorizations", C.c_int32), ("max_width", C.c_int32),
                ("stored_bytes", C.c_double), ("conventional_bytes", C.c_double),
                ("conventional_peak_bytes", C.c_double), ("device_bytes", C.c_double)]


class HmServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("batches", C.c_int64),
                ("batched_rhs", C.c_int64), ("factorizations", C.c_int64), ("evictions", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("device_bytes", C.c_double),
                ("joined", C.c_int64), ("oom_retries", C.c_int64),
                ("moved", C.c_int64), ("memory_waits", C.c_int64)]


class HmProfEntry(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int32), ("kernels", C.c_int32), ("ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


class HmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.hm_status_str(status).decode()
        detail = _lib.hm_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}): {detail}")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1410_2697_gb300.build`"
                          " (no CPU fallback exists)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.hm_default_opts.argtypes = [C.POINTER(HmOpts)]
    lib.hm_create.argtypes = [C.POINTER(vp), C.POINTER(HmOpts)]
    lib.hm_ctx_destroy.argtypes = [vp]
    lib.hm_analyze.argtypes = [vp, i32, vp, vp, i32, vp, vp, i32, vp, vp, C.POINTER(vp)]
    lib.hm_analyze_batch.argtypes = [vp, i32, vp, vp, i32, vp, i32, vp, C.POINTER(vp)]
    lib.hm_get_sizes.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    lib.hm_get_ordering.argtypes = [vp, vp, vp, vp, vp]
    lib.hm_get_symbolic.argtypes = [vp, vp, vp, vp, vp]
    lib.hm_factor.argtypes = [vp, vp, dbl, C.POINTER(HmFactorInfo)]
    lib.hm_autotune.argtypes = [vp, vp, dbl, i32, i32, C.POINTER(i32)]
    lib.hm_tune_force.argtypes = [vp, i32]
    lib.hm_solve.argtypes = [vp, i32, vp, dbl, i32, vp, C.POINTER(HmSolveInfo)]
    lib.hm_direct_solve.argtypes = [vp, i32, vp, i32, vp, C.POINTER(HmSolveInfo)]
    lib.hm_precond_apply.argtypes = [vp, i32, vp, vp]
    lib.hm_precond_apply_noalloc.argtypes = [vp, i32, vp, vp]
    lib.hm_get_update.argtypes = [vp, i32, vp]
    lib.hm_get_front_ranks.argtypes = [vp, i32, C.POINTER(i32), vp, C.POINTER(i32)]
    lib.hm_get_hodlr_block.argtypes = [vp, i32, i32, i32, C.POINTER(i32), C.POINTER(i32),
                                       C.POINTER(i32), C.POINTER(i32), vp, vp]
    lib.hm_profile_enable.argtypes = [vp, C.c_int]
    lib.hm_profile_read.argtypes = [vp, i32, C.POINTER(HmProfEntry), C.POINTER(i32)]
    lib.hm_server_create.argtypes = [C.POINTER(HmOpts), i32, i32, C.POINTER(vp)]
    lib.hm_server_add_matrix.argtypes = [vp, i32, vp, vp, vp, i32, vp, dbl, C.POINTER(i32)]
    lib.hm_server_submit.argtypes = [vp, i32, i32, vp, vp, dbl, C.POINTER(C.c_int64)]
    lib.hm_server_wait.argtypes = [vp, C.c_int64, C.POINTER(HmSolveInfo), C.POINTER(dbl), C.POINTER(i32)]
    lib.hm_server_get_stats.argtypes = [vp, C.POINTER(HmServerStats)]
    lib.hm_server_destroy.argtypes = [vp]
    lib.hm_destroy.argtypes = [vp]
    lib.hm_status_str.argtypes = [C.c_int]
    lib.hm_status_str.restype = C.c_char_p
    lib.hm_last_error.argtypes = []
    lib.hm_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("hm_status_str", "hm_last_error"):
            getattr(lib, name).restype = C.c_int
    return lib


_lib = _load()


def _check(status: int, where: str, ok=(HM_OK,)):
    if status not in ok:
        raise HmError(status, where)
    return status


def _ptr(a, dtype, name: str, count: int | None = None):
    """Pointer of a contiguous numpy array / torch tensor of the given numpy dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype):
            raise TypeError(f"{name}: expected {np.dtype(dtype)}, got {a.dtype}")
        if not (a.flags.c_contiguous or a.flags.f_contiguous):
            raise TypeError(f"{name}: array must be contiguous")
        if count is not None and a.size < count:
            raise ValueError(f"{name}: needs {count} elements, has {a.size}")
        return C.c_void_p(a.ctypes.data)
    # torch tensor (device or host)
    tname = {np.float64: "float64", np.int32: "int32", np.int64: "int64"}[np.dtype(dtype).type]
    if str(a.dtype) != f"torch.{tname}":
        raise TypeError(f"{name}: expected torch.{tname}, got {a.dtype}")
    if not a.is_contiguous():
        raise TypeError(f"{name}: tensor must be contiguous")
    if count is not None and a.numel() < count:
        raise ValueError(f"{name}: needs {count} elements, has {a.numel()}")
    return C.c_void_p(a.data_ptr())


def hm_default_opts() -> HmOpts:
    o = HmOpts()
    _check(_lib.hm_default_opts(C.byref(o)), "hm_default_opts")
    return o


def hm_create(opts: HmOpts | None = None) -> C.c_void_p:
    ctx = C.c_void_p()
    _check(_lib.hm_create(C.byref(ctx), C.byref(opts) if opts is not None else None), "hm_create")
    return ctx


def hm_ctx_destroy(ctx) -> None:
    _check(_lib.hm_ctx_destroy(ctx), "hm_ctx_destroy")


def hm_analyze(ctx, n, rowptr, colidx, dim=0, grid_coords=None, perm_in=None, nfronts_in=0,
               first_in=None, parent_in=None) -> C.c_void_p:
    sys_ = C.c_void_p()
    _check(_lib.hm_analyze(ctx, int(n), _ptr(rowptr, np.int64, "rowptr", n + 1),
                           _ptr(colidx, np.int32, "colidx"), int(dim),
                           _ptr(grid_coords, np.int32, "grid_coords"), _ptr(perm_in, np.int32, "perm_in"),
                           int(nfronts_in), _ptr(first_in, np.int32, "first_in"),
                           _ptr(parent_in, np.int32, "parent_in"), C.byref(sys_)), "hm_analyze")
    return sys_


def hm_analyze_batch(ctx, n, rowptr, colidx, dim, grid_coords, block_ptr) -> C.c_void_p:
    """Independent meshes (block-diagonal A): block b owns unknowns
    [block_ptr[b], block_ptr[b+1]); GMRES then converges per block and RHS."""
    sys_ = C.c_void_p()
    nblocks = len(block_ptr) - 1
    _check(_lib.hm_analyze_batch(ctx, int(n), _ptr(rowptr, np.int64, "rowptr", n + 1),
                                 _ptr(colidx, np.int32, "colidx"), int(dim),
                                 _ptr(grid_coords, np.int32, "grid_coords"), int(nblocks),
                                 _ptr(block_ptr, np.int32, "block_ptr", nblocks + 1), C.byref(sys_)),
           "hm_analyze_batch")
    return sys_


def hm_get_sizes(sys_) -> tuple[int, int]:
    n, nf = C.c_int32(), C.c_int32()
    _check(_lib.hm_get_sizes(sys_, C.byref(n), C.byref(nf)), "hm_get_sizes")
    return n.value, nf.value


def hm_get_ordering(sys_):
    n, nf = hm_get_sizes(sys_)
    perm = np.empty(n, np.int32)
    first = np.empty(nf + 1, np.int32)
    parent = np.empty(nf, np.int32)
    level = np.empty(nf, np.int32)
    _check(_lib.hm_get_ordering(sys_, _ptr(perm, np.int32, "perm"), _ptr(first, np.int32, "first"),
                                _ptr(parent, np.int32, "parent"), _ptr(level, np.int32, "level")),
           "hm_get_ordering")
    return perm, first, parent, level


def hm_get_symbolic(sys_):
    _, nf = hm_get_sizes(sys_)
    nupd = np.empty(nf, np.int32)
    off = np.empty(nf + 1, np.int64)
    _check(_lib.hm_get_symbolic(sys_, _ptr(nupd, np.int32, "nupd"), _ptr(off, np.int64, "if_off"),
                                None, None), "hm_get_symbolic")
    total = int(off[-1])
    lst = np.empty(max(total, 1), np.int32)
    rel = np.empty(max(total, 1), np.int32)
    _check(_lib.hm_get_symbolic(sys_, None, None, _ptr(lst, np.int32, "if_list"),
                                _ptr(rel, np.int32, "relmap")), "hm_get_symbolic")
    return nupd, off, lst[:total], rel[:total]


def hm_factor(sys_, values, tol: float) -> dict:
    info = HmFactorInfo()
    _check(_lib.hm_factor(sys_, _ptr(values, np.float64, "values"), float(tol), C.byref(info)),
           "hm_factor")
    return {f: getattr(info, f) for f, _ in HmFactorInfo._fields_}


def hm_autotune(sys_, values, tol: float, nrhs: int, reps: int = 2) -> int:
    """Time every tunable launch site in each variant on this system; the context keeps
    the faster ones.  Returns the number of sites timed."""
    n = C.c_int32(0)
    _check(_lib.hm_autotune(sys_, _ptr(values, np.float64, "values"), float(tol), int(nrhs), int(reps),
                            C.byref(n)), "hm_autotune")
    return n.value


def hm_tune_force(ctx, variant: int) -> None:
    """Fix every tunable launch site to `variant` (-1: back to the autotuner's choices)."""
    _check(_lib.hm_tune_force(ctx, int(variant)), "hm_tune_force")


def hm_solve(sys_, nrhs: int, b, rtol: float, max_iters: int, x, raise_on_no_convergence=True) -> dict:
    info = HmSolveInfo()
    st = _lib.hm_solve(sys_, int(nrhs), _ptr(b, np.float64, "b"), float(rtol), int(max_iters),
                       _ptr(x, np.float64, "x"), C.byref(info))
    ok = (HM_OK,) if raise_on_no_convergence else (HM_OK, HM_ERR_NO_CONVERGENCE)
    _check(st, "hm_solve", ok)
    return {f: getattr(info, f) for f, _ in HmSolveInfo._fields_}


def hm_direct_solve(sys_, nrhs: int, b, refine: int, x) -> dict:
    """x = M^{-1} b plus `refine` steps of iterative refinement (no Krylov method)."""
    info = HmSolveInfo()
    _check(_lib.hm_direct_solve(sys_, int(nrhs), _ptr(b, np.float64, "b"), int(refine), _ptr(x, np.float64, "x"),
                                C.byref(info)), "hm_direct_solve")
    return {f: getattr(info, f) for f, _ in HmSolveInfo._fields_}


def hm_precond_apply(sys_, nrhs: int, r, z) -> None:
    _check(_lib.hm_precond_apply(sys_, int(nrhs), _ptr(r, np.float64, "r"), _ptr(z, np.float64, "z")),
           "hm_precond_apply")


def hm_precond_apply_noalloc(sys_, nrhs: int, r, z) -> None:
    """Allocation-free z = M^{-1} r: r, z are device tensors (n x nrhs column-major)."""
    _check(_lib.hm_precond_apply_noalloc(sys_, int(nrhs), _ptr(r, np.float64, "r"),
                                         _ptr(z, np.float64, "z")), "hm_precond_apply_noalloc")


def hm_get_update(sys_, front: int, nupd: int) -> np.ndarray:
    U = np.zeros((nupd, nupd), dtype=np.float64, order="F")
    _check(_lib.hm_get_update(sys_, int(front), _ptr(U, np.float64, "U")), "hm_get_update")
    return U


def hm_get_front_ranks(sys_, front: int):
    kind, nr = C.c_int32(), C.c_int32()
    _check(_lib.hm_get_front_ranks(sys_, int(front), C.byref(kind), None, C.byref(nr)),
           "hm_get_front_ranks")
    r = np.zeros(max(nr.value, 1), np.int32)
    _check(_lib.hm_get_front_ranks(sys_, int(front), C.byref(kind), _ptr(r, np.int32, "ranks"),
                                   C.byref(nr)), "hm_get_front_ranks")
    return kind.value, r[:nr.value]


def hm_get_hodlr_block(sys_, front: int, level: int, node: int = 0):
    """Returns ``(U, V, rank)`` of a compressed block (level -1: F_fp ~ W Vf^T)."""
    m, n, k, r = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(_lib.hm_get_hodlr_block(sys_, int(front), int(level), int(node), C.byref(m), C.byref(n),
                                   C.byref(k), C.byref(r), None, None), "hm_get_hodlr_block")
    U = np.zeros((m.value, k.value), np.float64, order="F")
    V = np.zeros((n.value, k.value), np.float64, order="F")
    _check(_lib.hm_get_hodlr_block(sys_, int(front), int(level), int(node), C.byref(m), C.byref(n),
                                   C.byref(k), C.byref(r), _ptr(U, np.float64, "U"),
                                   _ptr(V, np.float64, "V")), "hm_get_hodlr_block")
    return U, V, r.value


def hm_profile_enable(ctx, enable: bool = True) -> None:
    _check(_lib.hm_profile_enable(ctx, 1 if enable else 0), "hm_profile_enable")


def hm_profile_read(ctx) -> dict:
    """{category: {"launches", "ms", "flops", "bytes"}} since the last enable."""
    buf = (HmProfEntry * 64)()
    n = C.c_int32()
    _check(_lib.hm_profile_read(ctx, 64, buf, C.byref(n)), "hm_profile_read")
    return {buf[i].name.decode(): {"launches": buf[i].launches, "kernels": buf[i].kernels, "ms": buf[i].ms,
                                   "flops": buf[i].flops, "bytes": buf[i].bytes}
            for i in range(n.value)}


def hm_destroy(sys_) -> None:
    _check(_lib.hm_destroy(sys_), "hm_destroy")


def hm_status_str(status: int) -> str:
    return _lib.hm_status_str(int(status)).decode()


def hm_last_error() -> str:
    return _lib.hm_last_error().decode()


# ------------------------------------------------------------------------------------
# serving
# ------------------------------------------------------------------------------------
def hm_server_create(opts=None, nworkers: int = 2, max_batch_rhs: int = 64) -> C.c_void_p:
    srv = C.c_void_p()
    o = opts if opts is not None else hm_default_opts()
    _check(_lib.hm_server_create(C.byref(o), int(nworkers), int(max_batch_rhs), C.byref(srv)), "hm_server_create")
    return srv


def hm_server_add_matrix(srv, problem, tol: float) -> int:
    """Registers a matrix (host copies are kept by the server); returns its id."""
    mid = C.c_int32()
    p = problem
    coords = np.ascontiguousarray(p.coords, dtype=np.int32)
    _check(_lib.hm_server_add_matrix(srv, int(p.n), _ptr(p.rowptr, np.int64, "rowptr", p.n + 1),
                                     _ptr(p.colidx, np.int32, "colidx"), _ptr(p.values, np.float64, "values"),
                                     int(p.dim), _ptr(coords, np.int32, "grid_coords"), float(tol), C.byref(mid)),
           "hm_server_add_matrix")
    return mid.value


def hm_server_submit(srv, matrix_id: int, b, x, rtol: float = 1e-10) -> int:
    """b, x: F-contiguous host arrays (n x nrhs) kept alive until hm_server_wait."""
    nrhs = 1 if b.ndim == 1 else b.shape[1]
    rid = C.c_int64()
    _check(_lib.hm_server_submit(srv, int(matrix_id), int(nrhs), _ptr(b, np.float64, "b"),
                                 _ptr(x, np.float64, "x"), float(rtol), C.byref(rid)), "hm_server_submit")
    return rid.value


def hm_server_wait(srv, request_id: int) -> dict:
    info = HmSolveInfo()
    lat = C.c_double()
    brhs = C.c_int32()
    st = _lib.hm_server_wait(srv, C.c_int64(request_id), C.byref(info), C.byref(lat), C.byref(brhs))
    d = {f: getattr(info, f) for f, _ in HmSolveInfo._fields_}
    d.update(status=st, latency_ms=lat.value, batch_rhs=brhs.value)
    return d


def hm_server_get_stats(srv) -> dict:
    st = HmServerStats()
    _check(_lib.hm_server_get_stats(srv, C.byref(st)), "hm_server_get_stats")
    return {f: getattr(st, f) for f, _ in HmServerStats._fields_}


def hm_server_destroy(srv) -> None:
    _check(_lib.hm_server_destroy(srv), "hm_server_destroy")
