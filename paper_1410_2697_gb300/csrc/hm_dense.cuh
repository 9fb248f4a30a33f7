// hm_dense.cuh -- batched dense kernels (SIMT, FP32/FP64) used by the factorization and
// the preconditioner apply.  Every kernel takes an array of task descriptors so that all
// fronts (and all blocks of all fronts) of one elimination-tree level run in one launch.
#pragma once

#include <vector>

#include "hm_common.cuh"

namespace hm {

// C[m x n] = alpha * op(A)[m x k] * op(B)[k x n] + beta * C.  Column-major; op 0 = N,
// 1 = T.  lower = 1 writes only entries with row >= column (SYRK-style updates).
struct GemmTask {
  const void* A;
  const void* B;
  void* C;
  int m, n, k;
  int lda, ldb, ldc;
  int opA, opB, lower, pad;
  double alpha, beta;
};

// One output tile (64 x BN) over the k range [k0, k1): task index and tile coordinates
// (tm << 16 | tn).  A tile whose k range is split over nsplit CTAs has a slot >= 0: each
// part writes its partial sums to the split workspace at woff + part * 64 * BN, and the
// last part to finish (counted on the slot's counter) adds the parts in order 0 .. nsplit-1
// and applies the epilogue, so the result does not depend on the finishing order.
struct GemmTile {
  int task;
  int mn;
  int k0, k1;
  int slot, part, nsplit, pad;
  int64_t woff;
};

constexpr int kGemmBM = 64;
constexpr int kGemmBN = 64;

// In-place lower Cholesky of an n x n block (n <= 128), ld >= n.
struct PotrfTask {
  void* A;
  int n, ld;
  int front, pad;
};

// B[rows] <- B[rows] * L^{-T}; L n x n lower (n <= 128), B has `m` rows; one launch
// item covers rows [row0, row0 + 64).
struct TrsmTask {
  const void* L;
  void* B;
  int n, ldl, m, ldb;
  int row0, pad;
};

// Householder QR of Y (m x k, ld): Q overwrites Y; R (k x k, ld k) written if non-null.
struct QrTask {
  void* Y;
  void* R;         // upper k x k factor (NULL: not wanted), leading dimension ldr (0: k)
  int m, k, ld, pad;
  void* Q;         // the explicit Q goes here (leading dimension ldq) instead of into Y
  int ldr, ldq;    // (shared-memory kernel only)
};

// Tall-skinny QR of an m x k panel (same contract as QrTask) in nb row blocks; the
// stacked R factors and the block reflector scalars live at element offset soff of a
// scratch arena (nb k x k, then nb k).
struct TsqrTask {
  void* Y;
  void* R;
  int64_t soff;
  int m, k, ld, nb;
};
struct TsqrBlock {
  int task, block;
};

// SVD of M = R^T (R k x k upper triangular, ld k) by one-sided Jacobi; writes
// UhS = Uhat_r Sigma_r (k x k, ld k; columns >= rank zero) and Vh = Vhat_r (same),
// sorted by decreasing singular value; rank = #{sigma_i > tol * sigma_1}.
// Boundary-distance low-rank approximation (BDLR, Section 2.2) of one off-diagonal block
// B = K[x0 : x0 + mx, y0 : y0 + my] of front q (nhat x nhat, column-major, lower triangle
// assembled; trans = 1: B(i, j) is stored at (y0 + j, x0 + i)).  Rows of X within graph
// distance depth of Y and columns of Y within depth of X (graph of A restricted to the
// front's unknowns; at most cap each, nearer first, then lower position) give B^ =
// B(I, J); complete-pivoting LU of B^ with rank r = pivots while |u_ss| >= tol |u_11|;
// U = B(:, J_q) U_r^{-1} (mx x r, ld ldu) and V = (L_r^{-1} B(I_p, :))^T (my x r, ld
// ldv), so B ~ U V^T; *rank = r.  Columns r.. of U and V are left as they are (zero).
struct BdlrTask {
  const void* F;
  void* U;
  void* V;
  int* rank;
  int q, nh, x0, mx, y0, my, trans, ldu, ldv, cap;
};

struct SvdTask {
  const void* R;
  void* UhS;
  void* Vh;
  int* rank;
  int k, pad;
};

// Sketch Omega (rows x cols, ld) of block `blk` (Philox4x32-10, 24-bit uniform).
struct OmegaTask {
  void* out;
  uint64_t blk;
  int rows, cols, ld, pad;
};

// Woodbury core C (n2 = 2k, ld n2): the GEMMs have written the two diagonal k x k
// blocks; this sets the off-diagonal blocks to I, LU-factors C with partial pivoting and
// writes the explicit inverse to Cinv (n2 x n2, ld n2).
// A rows x cols block copied from src (ld lds) to dst (ld ldd).
struct CopyTask {
  const void* src;
  void* dst;
  int rows, cols, lds, ldd;
};

// A dense front (nhat x nhat, ld nhat, nhat <= 128) factored in one pass by np
// Gauss-Jordan sweeps into F_pp^{-1}, K^T, K and U_p.  The rows of the pivot block
// [F_pp^{-1} | K^T] go to P (ld ldp, or np when ldp is 0), K (nu x np) to
// P + packed_k_offset (ld nu), the lower triangle of U_p back into F (where the parent's
// extend-add reads it).  A HODLR leaf (np = nhat) sends its inverse to the packed leaf
// store this way.
struct SweepTask {
  void* F;
  void* P;
  int np, nhat, front, ld;  // ld: leading dimension of F (0: nhat)
  int ldp, pad;
};

struct CoreLuTask {
  void* C;
  void* Cinv;
  int* piv;
  int k, front;
};

// From a Cholesky factor L (lower triangle of A, n <= 128, ld): A <- A^{-1} (full n x n)
// and, if m > 0, B (m x n, ldb) <- B L^{-1}  (so that B L^{-1} = F_fp F_pp^{-1} when B
// holds L_fp = F_fp L^{-T}).
struct CholInvTask {
  void* A;
  void* B;
  int n, ld, m, ldb;
  void* BT;   // if set, (B Linv)^T is also written here (n x m, leading dimension ldbt)
  int ldbt, pad;
};

// deep: 0 = 16-deep k-slices, 1 = the deeper variant (64 for bn 16, 32 for bn 64),
// 2 = 32-deep slices copied by cp.async several slices ahead.
template <typename T>
void launch_gemm(const GemmTask* tasks, const GemmTile* tiles, int ntiles, int bn, int deep, T* split_ws,
                 unsigned* split_cnt, cudaStream_t s);
template <typename T>
void launch_front_sweep(const SweepTask* tasks, int ntasks, int maxn, int* err, cudaStream_t s);
template <typename T>
void launch_potrf(const PotrfTask* tasks, int ntasks, int maxn, int* err, cudaStream_t s);
template <typename T>
void launch_trsm(const TrsmTask* tasks, int ntasks, int maxn, cudaStream_t s);
template <typename T>
void launch_qr(const QrTask* tasks, int ntasks, int maxm, int64_t maxmk, int max_smem, cudaStream_t s);
// Bytes the shared-memory panel QR needs beyond its panel and reflector block (its static
// shared memory and a margin), es = element size.
size_t qr_smem_overhead(int es);
template <typename T>
void launch_tsqr(const TsqrTask* tasks, int ntasks, const TsqrBlock* blocks, int nblocks, size_t smem_block,
                 size_t smem_stack, T* scratch, cudaStream_t s);
template <typename T>
void launch_svd(const SvdTask* tasks, int ntasks, int maxk, double tol, cudaStream_t s);
template <typename T>
void launch_bdlr(const BdlrTask* tasks, int ntasks, int maxnh, int maxcap, int depth, double tol,
                 const int32_t* first, const int* npiv, const int64_t* ifoff, const int32_t* iflist,
                 const int64_t* prowptr, const int32_t* pcol, cudaStream_t s);
template <typename T>
void launch_omega(const OmegaTask* tasks, int ntasks, uint64_t seed, cudaStream_t s);
template <typename T>
void launch_core_lu(const CoreLuTask* tasks, int ntasks, int maxk, int max_smem, int* err,
                    cudaStream_t s);
template <typename T>
void launch_chol_inverse(const CholInvTask* tasks, int ntasks, int maxn, cudaStream_t s);

// Host-side: tile width (64, or 16 when every task has at most 16 columns) and the tiles
// of one task (all tiles, or those touching the lower triangle when t.lower).
int gemm_bn_for(const std::vector<GemmTask>& t);
int gemm_tile_count(const GemmTask& t, int bm, int bn);
// Appends the bm x bn tiles of task t; with nsplit > 1 every tile's k range is split into
// parts that take consecutive split slots (*slots) and workspace (*ws elements).
void gemm_tiles_for(const GemmTask& t, int task_index, int bm, int bn, int nsplit, std::vector<GemmTile>* out,
                    int* slots, int64_t* ws);
// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) batched GEMM on 128 x 64 tiles;
// FP32 data in memory.  A mbarrier wait that runs out (after wait_limit polls; <= 0: the
// default) raises HM_ERR_DEVICE_TIMEOUT in err.
constexpr int kTcBM = 128, kTcBN = 64;
// inject_timeout != 0: every tile ends with one more bounded wait, on a barrier nothing
// arrives on, which runs out (fault injection for the tests of the timeout path).
void launch_gemm_tc(const GemmTask* tasks, const GemmTile* tiles, int ntiles, float* split_ws,
                    unsigned* split_cnt, int* err, int wait_limit, int inject_timeout, cudaStream_t s);
// FP32 products at FP32 accuracy on the tensor cores (tcgen05 kind::tf32, every operand
// split into a TF32 hi part and its remainder, three MMAs per step), same tiles.
void launch_gemm_tf32x3(const GemmTask* tasks, const GemmTile* tiles, int ntiles, float* split_ws,
                        unsigned* split_cnt, int* err, int wait_limit, cudaStream_t s);
int dense_tc_setup(int max_smem);

int dense_fact_setup(int max_dyn_smem);
int dense_comp_setup(int max_dyn_smem);
int gemm_async_setup(int max_dyn_smem);
// FP32 128 x 128-tile variant (tiles built with kBigTile x kBigTile).
constexpr int kBigTile = 128;
void launch_gemm_big(const GemmTask* tasks, const GemmTile* tiles, int ntiles, float* split_ws,
                     unsigned* split_cnt, cudaStream_t s);

}  // namespace hm
