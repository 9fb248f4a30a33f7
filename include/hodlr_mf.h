/*
 * hodlr_mf.h -- C ABI of the GB300 (sm_103a) HODLR-accelerated multifrontal solver.
 *
 * The library solves A x = b for a sparse symmetric positive definite finite-element
 * matrix A (Aminfar & Darve, "A Fast and Memory Efficient Sparse Solver with
 * Applications to Finite-Element Matrices", arXiv 1410.2697, Section 1) with GMRES
 * preconditioned by an approximate (HODLR-accelerated) multifrontal factorization
 * (Sections 3 and 4).  Every numerical step runs in CUDA kernels on one GPU.
 *
 * Conventions for every entry point
 *   - Return value: an hm_status code (0 = HM_OK).  No call aborts, traps or throws;
 *     hm_status_str() gives a message, hm_last_error() the detail of the last failure
 *     on the calling thread.
 *   - Array arguments may be host or device (CUDA) pointers; the library detects which
 *     and copies what it needs.  The caller keeps ownership of every array it passes;
 *     nothing is retained after a call returns.
 *   - Sparse matrices are CSR with 64-bit row pointers and 32-bit column indices, the
 *     FULL symmetric pattern (both triangles), columns sorted within each row, no
 *     duplicates, indices 0-based.  Dirichlet rows are removed (not replaced by identity).
 *   - Dense right-hand sides and solutions are column-major n x nrhs (ld = n), FP64.
 *   - Handles are not thread-safe: one thread (one CUDA stream) per hm_sys_t at a time.
 */
#ifndef HODLR_MF_H
#define HODLR_MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_ctx_s* hm_ctx_t;
typedef struct hm_sys_s* hm_sys_t;

enum hm_status {
  HM_OK = 0,
  HM_ERR_INVALID_ARG = 1,    /* bad size, null pointer, malformed CSR or lattice       */
  HM_ERR_NOT_SPD = 2,        /* a pivot block was not positive definite (Cholesky)     */
  HM_ERR_NO_CONVERGENCE = 3, /* GMRES hit max_iters above rtol (x holds the iterate)   */
  HM_ERR_OUT_OF_MEMORY = 4,  /* device allocation failed or HBM budget exceeded         */
  HM_ERR_CUDA = 5,           /* a CUDA runtime call failed (see hm_last_error)          */
  HM_ERR_CAPACITY = 6,       /* a fixed on-chip capacity was exceeded (front too large) */
  HM_ERR_DEVICE_TIMEOUT = 7, /* a bounded device-side wait gave up                      */
  HM_ERR_STATE = 8,          /* call out of order (e.g. solve before factor)           */
  HM_ERR_BREAKDOWN = 9       /* singular Woodbury core / zero pivot in LU               */
};

enum hm_precision {
  HM_PREC_FP64 = 0,      /* factorization, compression and preconditioner apply in FP64 */
  HM_PREC_MIXED = 1,     /* factorization, compression and apply in FP32; GMRES in FP64 */
  HM_PREC_MIXED_BF16 = 2 /* as MIXED, with the range finder's sampling products Y = B Omega
                            and Z = B^T Q on the tensor cores (BF16 operands, FP32
                            accumulation); the compression error then includes BF16
                            rounding of the sampled blocks (about 2^-9 of their size)      */
};

/* Off-diagonal compressor of the HODLR fronts (Section 2.2). */
enum hm_compressor {
  HM_COMP_RRF = 0,       /* randomized range finder (Philox sketch of width `samples`, QR,
                            small SVD; singular values <= tol sigma_1 dropped)            */
  HM_COMP_BDLR = 1       /* boundary-distance low-rank approximation: rows and columns
                            within graph distance bdlr_depth of the other index set (graph
                            of A on the front's unknowns, at most `samples` of each),
                            complete-pivoting LU, rank by |u_rr / u_11| >= tol           */
};

typedef struct hm_opts {
  int device;            /* CUDA device ordinal                                          */
  int precision;         /* enum hm_precision                                            */
  int nd_leaf;           /* nested dissection stops at boxes of <= nd_leaf unknowns (64) */
  int hodlr_leaf;        /* HODLR leaves hold <= hodlr_leaf rows (64)                    */
  int n_c;               /* fronts whose pivot block has > n_c unknowns become HODLR
                            fronts; smaller ones stay dense (the paper's n_c)            */
  int samples;           /* randomized range finder sketch width cap k (1 .. 96; FP64:
                            1 .. 64)                                                     */
  uint64_t seed;         /* seed of the Philox4x32-10 sketch                             */
  int restart;           /* GMRES restart length m (30)                                  */
  size_t hbm_budget;     /* bytes the context may allocate on the device; 0 = no limit  */
  void* stream;          /* cudaStream_t to run on; NULL = a stream the context owns     */
  int dofs_per_node;     /* unknowns per mesh node for geometric nested dissection (1;
                            3 for 3D elasticity): unknown b k + c is component c of node
                            k, all b share the node's grid_coords; separators then hold
                            whole nodes, and a node's unknowns stay consecutive          */
  int compressor;        /* enum hm_compressor (HM_COMP_RRF)                              */
  int bdlr_depth;        /* BDLR graph-distance depth d (1, the paper's usual setting)   */
  int wait_limit;        /* polls of a bounded device-side wait (the tensor-core GEMM's
                            mbarrier waits on its MMAs; the first poll never suspends
                            the thread) before the kernel gives up with
                            HM_ERR_DEVICE_TIMEOUT; 0 = the default, 2^22.  A kernel that
                            gives up still waits (with the default limit) for the MMAs it
                            issued and frees its tensor memory before it returns.        */
  int adaptive_rank;     /* 1 (FP32 and BF16 modes; ignored in FP64): a compressed block
                            whose rank reaches its sketch width was truncated by the
                            width, not by tol: the factorization then doubles the sketch
                            width of that front level (up to 96) and
                            factors again, until no block is capped or no width can
                            grow; the widths are remembered for later analyses of the
                            same shape in this context (0 = off)                        */
  int inject_wait_timeout; /* fault injection for tests (0 = off): 1 makes every tile of
                            the tensor-core GEMM end with one more bounded wait, on a
                            barrier nothing arrives on, so the factorization reports
                            HM_ERR_DEVICE_TIMEOUT through the path a real timeout takes  */
  int compress_ff;       /* 1: a HODLR front's update block F_ff is first replaced by its
                            own HODLR approximation F_ff^HODLR (Section 4.2.1: every
                            off-diagonal block of F_ff's HODLR tree, leaf hodlr_leaf,
                            compressed by the range finder at tol with the level's sketch
                            width), so the update passed to the parent is
                            F_ff^HODLR - W T W^T (Eq. update_HODLR).  The approximation is
                            written back into the dense front (the extend-add stays dense).
                            Range finder only (HM_ERR_INVALID_ARG with BDLR); 0 = off    */
  int keep_fronts;       /* 0 (default): the dense front storage is reused across tree
                            levels (two banks, one for even and one for odd depths: a level's
                            fronts live until their parents have absorbed their updates), so
                            the transient fronts take the two largest level sums instead of
                            all levels; the factor the apply needs is packed out of the
                            fronts level by level.  1: every front keeps its own storage after
                            the factorization, for hm_get_update (which fails with
                            HM_ERR_STATE otherwise)                                      */
} hm_opts;

typedef struct hm_solve_info {
  int32_t iters;         /* GMRES iterations (max over right-hand sides)                 */
  int32_t restarts;      /* completed restart cycles                                     */
  double relres;         /* max over right-hand sides of ||b - A x|| / ||b|| (FP64)      */
  int32_t converged;     /* 1 if every right-hand side reached rtol                      */
} hm_solve_info;

typedef struct hm_factor_info {
  int32_t nfronts;       /* elimination-tree nodes                                       */
  int32_t nlevels;       /* tree depth + 1                                               */
  int32_t n_hodlr;       /* fronts factored as HODLR fronts                              */
  int32_t max_rank;      /* largest off-diagonal rank found                              */
  int32_t rank_capped;   /* blocks whose rank reached their sketch width                 */
  double factor_bytes;   /* bytes of factor data read by one preconditioner apply        */
  double front_bytes;    /* bytes of dense front storage                                 */
  int32_t refactorizations; /* extra factorizations the adaptive rank rule ran            */
  int32_t max_width;     /* largest sketch width in use (per front level)                 */
  /* memory (bytes), the paper's comparison with the conventional method (Section 6):   */
  double stored_bytes;   /* factor data the preconditioner keeps for the apply: dense fronts'
                            F_pp^-1, K and K^T; HODLR fronts' bases U / V / Vf, Vtilde, G,
                            W and leaf inverses                                            */
  double conventional_bytes; /* the conventional multifrontal Cholesky factor L of the same
                            ordering in the same precision: sum of np (np + 1) / 2 + np nu */
  double conventional_peak_bytes; /* the conventional method's peak: L so far plus the live
                            update matrices plus the current front (lower triangles),
                            maximum over the fronts in elimination order                  */
  double device_bytes;   /* device memory this system holds after the factorization
                            (pattern, plan, fronts, factor, scratch)                      */
} hm_factor_info;

/* Fill *opts with defaults (device 0, mixed precision, nd_leaf 64, hodlr_leaf 64,
   n_c 64, samples 48, restart 30, dofs_per_node 1, compressor HM_COMP_RRF,
   bdlr_depth 1, wait_limit 0, adaptive_rank 0, inject_wait_timeout 0, compress_ff 0,
   keep_fronts 0).  Never fails
   for a non-null pointer.                                                            */
int hm_default_opts(hm_opts* opts);

/* Create a context on opts->device.  The context owns a CUDA stream (unless one is
   given) and the device memory of every system created from it.                     */
int hm_create(hm_ctx_t* ctx, const hm_opts* opts);
int hm_ctx_destroy(hm_ctx_t ctx);

/*
 * Symbolic analysis (Section 4.1.1): nested-dissection ordering, elimination tree,
 * coupling sets S_p (Eq. couplingSet), frontal index sets I_p^f and the child-to-parent
 * relative index maps of the extend-add.
 *
 *   n, rowptr[n+1], colidx[nnz]   CSR pattern of A (values are given to hm_factor).
 *   dim, grid_coords[n*dim]       integer lattice coordinates of each unknown (row-major
 *                                 n x dim, dim 2 or 3); the unknowns must fill their
 *                                 bounding box.  The ordering is computed on the GPU:
 *                                 boxes are split along the longest axis (lowest axis on
 *                                 ties) by the plane (lo+hi)/2, halves first, separator
 *                                 last, points lexicographic x-fastest, stop at nd_leaf.
 *   perm_in, nfronts_in, first_in, parent_in
 *                                 optional user ordering instead of grid_coords: perm_in[n]
 *                                 maps new -> original index; tree node p (postorder,
 *                                 children before parents) owns new indices
 *                                 [first_in[p], first_in[p+1]); parent_in[root] = -1
 *                                 (a forest may have several roots).
 *                                 Pass NULL / 0 to use grid_coords.
 *   out                           receives the system handle.
 * Errors: HM_ERR_INVALID_ARG for a malformed CSR / lattice / tree, HM_ERR_CAPACITY if a
 * front's candidate index set exceeds the on-chip sort capacity (32768 indices).
 */
int hm_analyze(hm_ctx_t ctx, int32_t n, const int64_t* rowptr, const int32_t* colidx,
               int32_t dim, const int32_t* grid_coords, const int32_t* perm_in,
               int32_t nfronts_in, const int32_t* first_in, const int32_t* parent_in,
               hm_sys_t* out);

/*
 * Batched analysis of independent meshes (a block-diagonal A): the unknowns are split
 * into nblocks contiguous ranges [block_ptr[b], block_ptr[b+1]); every coupling of A stays
 * inside its range, and each range's grid_coords fill that range's own bounding box.
 * Every block is ordered by the nested dissection of hm_analyze (its unknowns keep their
 * range in the new numbering), and the elimination tree is the forest of the blocks'
 * trees, concatenated in postorder.  hm_factor then processes all fronts of one tree depth
 * across every block in the same launches, and hm_solve runs GMRES independently on every
 * (block, right-hand side) pair: each stops on its own relative residual
 * ||b_b - A_b x_b|| / ||b_b||.  Host or device pointers; block_ptr[nblocks + 1] with
 * block_ptr[0] = 0 and block_ptr[nblocks] = n.  Errors as hm_analyze, and
 * HM_ERR_INVALID_ARG for a coupling between blocks.
 */
int hm_analyze_batch(hm_ctx_t ctx, int32_t n, const int64_t* rowptr, const int32_t* colidx,
                     int32_t dim, const int32_t* grid_coords, int32_t nblocks,
                     const int32_t* block_ptr, hm_sys_t* out);

/* Number of tree nodes and unknowns (either pointer may be NULL).                     */
int hm_get_sizes(hm_sys_t sys, int32_t* n, int32_t* nfronts);

/* Ordering and tree: perm[n] (new -> original), first[nfronts+1], parent[nfronts],
   level[nfronts] (depth, root 0).  Host pointers; any may be NULL.                     */
int hm_get_ordering(hm_sys_t sys, int32_t* perm, int32_t* first, int32_t* parent,
                    int32_t* level);

/* Symbolic result: nupd[p] = |I_p^f|; if_off[nfronts+1] prefix offsets; if_list[] the
   sorted new indices of every I_p^f (front p at if_off[p]); relmap[] the position of each
   entry of I_p^f inside the parent's front [I_parent, I_parent^f] (same offsets; -1
   at the root).  Host pointers; query total = if_off[nfronts] first with if_list NULL. */
int hm_get_symbolic(hm_sys_t sys, int32_t* nupd, int64_t* if_off, int32_t* if_list,
                    int32_t* relmap);

/*
 * Numerical factorization (Sections 4.1.1 and 4.2.1) of A with the pattern given to
 * hm_analyze.  values[nnz] are the CSR values (FP64).  tol is the relative truncation
 * tolerance of the low-rank compression (singular values <= tol * sigma_1 of a block
 * are dropped); tol <= 0 keeps every sampled direction.  May be called repeatedly with
 * new values (refactorization).  While the factorization runs on the device, the host
 * also prepares the preconditioner-apply workspace for the right-hand-side count of the
 * context's most recent solve or apply (device memory of the system, freed by
 * hm_destroy).  Errors: HM_ERR_NOT_SPD, HM_ERR_BREAKDOWN, CUDA errors.
 */
int hm_factor(hm_sys_t sys, const double* values, double tol, hm_factor_info* info);

/*
 * Direct mode (the solver used on its own at a tight tolerance, Section 6): x = M^{-1} b
 * with the factorization M of A, followed by `refine` steps of iterative refinement
 * x += M^{-1} (b - A x) with the residual in FP64; no Krylov method.  b and x are
 * n x nrhs column-major FP64 in the ORIGINAL numbering (host or device), nrhs <= 64,
 * 0 <= refine <= 100.  info (may be NULL): iters = number of applications of M^{-1},
 * relres = largest ||b - A x|| / ||b|| over the right-hand sides (and blocks of a batch),
 * converged = 1.  The accuracy is what the factorization's tolerance delivers: tol = 0
 * (every sampled direction kept) with FP64 gives x to rounding.
 */
int hm_direct_solve(hm_sys_t sys, int32_t nrhs, const double* b, int32_t refine, double* x,
                    hm_solve_info* info);

/*
 * Autotuner of the batched launches (one launch per elimination-tree level and stage,
 * Section 4): every tunable launch site -- the batched GEMMs of factorization and apply
 * (k-slice depth, register- or cp.async-staged operands), the range finder's panel QR
 * (shared-memory-resident or global), the
 * dense fronts' apply kernels (threads per front) -- is keyed by the shapes of its batch.
 * Runs the factorization with values[] and tol plus two GMRES iterations on nrhs
 * right-hand sides, reps times per variant, with every site forced to each variant in
 * turn; keeps per site the variant with the least mean launch time (the default unless
 * another is more than 3% faster) in the CONTEXT, so later systems of the same shapes
 * analysed on it use the choices too; then refactors sys with them.  values may be host
 * or device memory.  *nsites (may be NULL) = number of sites timed.  The variants
 * compute the same quantities (the SIMT GEMM variants bit-identically; the tensor-core
 * GEMM, the QR and the apply variants to rounding).  Requires the launch profiler off
 * (HM_ERR_STATE).  1 <= nrhs <= 64, 1 <= reps <= 16.
 */
int hm_autotune(hm_sys_t sys, const double* values, double tol, int32_t nrhs, int32_t reps,
                int32_t* nsites);

/* Fix every tunable launch site of the context to one variant (0 = the built-in
   default; GEMM sites: 1 deeper k-slices, 2 cp.async staging, 3 FP32 128 x 128 tiles
   where the batch has such products, 4 FP32 on the tensor cores (3xTF32, tcgen05) where
   the batch has a product of at least 64 x 32 x 64; QR sites: 1 global memory; dense
   apply levels: 1 the other thread count, 2 and 3 a quarter of the right-hand sides per
   block (with the default / the other thread count); HODLR-front apply levels: 1 the
   batched-GEMM path, 0 / 2 / 3 the fused cluster kernels with a quarter / an eighth / a
   sixteenth of the widest right-hand-side group per cluster; a variant a site lacks acts
   as 0), or -1 to return to the autotuner's choices.  For reproducing a configuration
   and for tests; hm_autotune clears it.  Applies to launches issued afterwards (apply
   graphs captured earlier keep their variants until the solve plan is rebuilt).      */
int hm_tune_force(hm_ctx_t ctx, int32_t variant);

/*
 * Solve A X = B by GMRES(restart) preconditioned with the factorization (Section 3):
 * right preconditioning, flexible form (the preconditioned vectors are stored), FP64
 * residuals, Arnoldi by classical Gram-Schmidt applied twice, Givens least squares.
 * b and x are n x nrhs column-major FP64 in the ORIGINAL numbering; x0 = 0.  Stops when
 * every column reaches ||b - A x|| / ||b|| <= rtol (true residual) or after max_iters.
 * nrhs <= 64.  Returns HM_ERR_NO_CONVERGENCE (x holds the last iterate) if the cap is hit.
 */
int hm_solve(hm_sys_t sys, int32_t nrhs, const double* b, double rtol, int32_t max_iters,
             double* x, hm_solve_info* info);

/* One preconditioner application z = M^{-1} r (Eqs. upward / downward with the HODLR
   pivot solves of Section 4.2.2); r, z n x nrhs FP64, original numbering.  The apply
   workspace is built per right-hand-side count on first use (a system keeps the four
   most recently used ones); an apply whose input buffer repeats is replayed from a
   captured CUDA graph.                                                                 */
int hm_precond_apply(hm_sys_t sys, int32_t nrhs, const double* r, double* z);

/*
 * hm_precond_apply without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot let a library call cudaMalloc -- programs
 * whose device memory is owned by another allocator (a framework's caching pool or a
 * fixed budget), allocator callbacks that must not re-enter the CUDA allocator, and
 * latency-critical loops that cannot wait on the driver.  It computes the same
 * z = M^{-1} r as hm_precond_apply with the same kernels, launched one by one: it never
 * captures or instantiates a CUDA graph.
 *   r, z      DEVICE pointers, n x nrhs column-major FP64, original numbering.  The call
 *             runs on the context's stream (hm_opts.stream, else the context's own
 *             non-blocking stream): r must already hold its values when the call is made
 *             -- work that produces r on another stream must be complete (synchronize
 *             that stream) unless the context was created on that same stream.
 *   Returns   after synchronizing the context's stream: z is complete on return.  The
 *             call is blocking.
 *   Limits    n * nrhs <= 262144 (HM_ERR_CAPACITY beyond).  The per-nrhs workspace of
 *             the system must exist already: make one hm_precond_apply or hm_solve call
 *             with the same nrhs first (HM_ERR_STATE otherwise; that call allocates).
 *             A system keeps the workspaces of its four most recently used nrhs values.
 *   Scratch   the per-call temporaries live in one file-scope device array of 6 MiB that
 *             every GPU loading the library holds until the process exits.  All calls
 *             share it, so calls that overlap on the GPU (from several threads or
 *             streams) race; serialise them.  Each call overwrites every temporary it
 *             reads, so nothing needs clearing between calls.
 *   Set-up    the first call on each context looks up the array's device address
 *             (cudaGetSymbolAddress, which allocates nothing) with the context's device
 *             current; make that first call before any stream capture.
 */
int hm_precond_apply_noalloc(hm_sys_t sys, int32_t nrhs, const double* r, double* z);

/* Inspection for tests: the dense Schur-complement update U_p = F_ff - F_fp F_pp^-1 F_pf
   of front p as computed by the last hm_factor (nupd[p]^2 entries, column-major, lower
   triangle valid, FP64).  Host pointer.  With front storage reuse (keep_fronts 0) only
   fronts of depth 0 and 1 keep their update; deeper ones give HM_ERR_STATE.            */
int hm_get_update(hm_sys_t sys, int32_t front, double* U);

/* Inspection: front kind (0 dense, 1 HODLR) and ranks of the last hm_factor.  ranks
   receives, for a HODLR front, the rank of F_fp followed by the ranks of the pivot
   block's off-diagonal blocks level by level (node order); returns the count in *nr. */
int hm_get_front_ranks(hm_sys_t sys, int32_t front, int32_t* kind, int32_t* ranks,
                       int32_t* nr);

/* Inspection: the low-rank factors of one compressed block of HODLR front `front` from
   the last hm_factor.  level = -1 selects the coupling block F_fp ~ W Vf^T (U = W is
   nupd x k, V = Vf is npiv x k); level >= 0 selects the off-diagonal block of node
   (level, node) of the pivot block's HODLR tree, F_pp[a, b] ~ U V^T with a / b the rows
   of its first / second child (U is |a| x k, V is |b| x k).  k is the column capacity;
   columns at or beyond *rank are zero.  Pass U = V = NULL to query m, n, k, rank.
   U, V: host, column-major FP64.                                                     */
int hm_get_hodlr_block(hm_sys_t sys, int32_t front, int32_t level, int32_t node, int32_t* m,
                       int32_t* n, int32_t* k, int32_t* rank, double* U, double* V);

/* Launch profiler of a context.  While enabled, every kernel launch of the context's
   systems is bracketed by CUDA events on the launching stream and tagged with a
   category and its algorithmic work (minimum flops and HBM bytes of what it computes).
   hm_profile_enable(ctx, 1) clears the records; hm_profile_read synchronizes and returns
   one entry per category with launches, summed device time (ms), flops and bytes.   */
typedef struct hm_prof_entry {
  char name[24];
  int32_t launches;      /* bracketed launch groups                                    */
  int32_t kernels;       /* CUDA kernels inside them (copies and memsets count 0)      */
  double ms;
  double flops;
  double bytes;
} hm_prof_entry;
int hm_profile_enable(hm_ctx_t ctx, int enable);
int hm_profile_read(hm_ctx_t ctx, int32_t max_entries, hm_prof_entry* out, int32_t* n);

int hm_destroy(hm_sys_t sys);

const char* hm_status_str(int status);
const char* hm_last_error(void);

/*
 * Serving (many matrices, requests arriving over time).  A server owns nworkers worker
 * threads, each with its own context (stream; opts->stream is ignored); the contexts
 * share one stream-ordered memory pool and the one budget opts->hbm_budget, so a single
 * matrix may use all of it.  Registered matrices (host copies of the CSR, FP64 values
 * and lattice coordinates) are analysed + factored on their first request by the worker
 * that takes it, and the factorization stays resident until evicted (least recently used
 * first, among the systems no worker holds, whichever worker holds them) to admit other
 * work within the budget.  Admission is by estimate, before the work allocates: a
 * matrix's estimate is its footprint when last resident (plus an eighth), else the bytes
 * per nonzero of the largest matrix of its dimension seen so far; a session's is its
 * slots times (2 restart + 10) FP64 vectors (plus a quarter and 4 MiB); the worker evicts
 * until the bytes held plus the estimate fit.  A shortfall of the estimate is caught by
 * the budget check of the allocation itself (one more eviction and a retry, counted in
 * oom_retries); with nothing left to evict while other workers run sessions, the worker
 * waits for one of them to end (memory_waits; meanwhile sessions take no new requests),
 * and the request fails with HM_ERR_OUT_OF_MEMORY only when it does not fit with no other
 * session running.  Requests wait in one queue; a free worker takes the oldest one whose
 * matrix no worker holds (one resident on another, idle worker is left to that worker;
 * one resident on a busy worker moves to the taker's context, counted in moved) and runs
 * a GMRES session on the matrix: a fixed number of right-hand-side slots (twice the
 * starting columns, at most max_batch_rhs, within a quarter of budget / nworkers for the
 * GMRES workspace), every waiting request for the matrix that fits put in; after every
 * restart cycle the requests whose columns all converged leave with their answers and
 * requests that arrived meanwhile take the free slots (continuous batching).  Each
 * right-hand side is its own GMRES instance with its own restart boundaries, so a
 * request's answer equals (to rounding) the answer it gets alone.  Workers run
 * concurrently, so different matrices overlap on the GPU.  Latency = completion -
 * submission, host clock.
 *
 *   hm_server_submit: b, x are host arrays (n x nrhs column-major) that must stay valid
 *   until hm_server_wait returns for the request; nrhs <= max_batch_rhs.
 *   hm_server_wait: blocks until the request completes; returns its status (HM_OK,
 *   HM_ERR_NO_CONVERGENCE, HM_ERR_OUT_OF_MEMORY if the matrix does not fit the budget
 *   alone, ...) and, if non-null, its solve info, latency and the number of right-hand
 *   sides in the solve that served it.
 */
typedef struct hm_server_s* hm_server_t;
typedef struct hm_server_stats {
  int64_t completed, failed;     /* requests finished with / without success            */
  int64_t batches, batched_rhs;  /* solves run and right-hand sides they carried        */
  int64_t factorizations;        /* analyze + factor runs (misses)                      */
  int64_t evictions;             /* resident systems destroyed to admit others          */
  double p50_ms, p99_ms;         /* latency percentiles of the successful requests      */
  double device_bytes;           /* device memory held by the workers' contexts         */
  int64_t joined;                /* requests that entered a session already running     */
  int64_t oom_retries;           /* budget misses the admission estimate did not foresee
                                    (the step was retried after one more eviction, or
                                    after another worker's session ended)               */
  int64_t moved;                 /* resident systems moved to another worker's context  */
  int64_t memory_waits;          /* waits for another worker's session to end, for room */
} hm_server_stats;

int hm_server_create(const hm_opts* opts, int32_t nworkers, int32_t max_batch_rhs, hm_server_t* out);
int hm_server_add_matrix(hm_server_t server, int32_t n, const int64_t* rowptr, const int32_t* colidx,
                         const double* values, int32_t dim, const int32_t* grid_coords, double tol,
                         int32_t* matrix_id);
int hm_server_submit(hm_server_t server, int32_t matrix_id, int32_t nrhs, const double* b, double* x,
                     double rtol, int64_t* request_id);
int hm_server_wait(hm_server_t server, int64_t request_id, hm_solve_info* info, double* latency_ms,
                   int32_t* batch_rhs);
int hm_server_get_stats(hm_server_t server, hm_server_stats* stats);
int hm_server_destroy(hm_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* HODLR_MF_H */
