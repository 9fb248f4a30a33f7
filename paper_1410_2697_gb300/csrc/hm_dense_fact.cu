// hm_dense_fact.cu -- small batched factorizations: Cholesky (dense pivot blocks and
// HODLR leaves), triangular solves, and the LU of the Woodbury cores.
#include "hm_dense.cuh"

namespace hm {

// =====================================================================================
// Cholesky of one pivot block per CTA (n <= 128), right-looking, in shared memory.
// A non-positive pivot raises HM_ERR_NOT_SPD (front id, column) and the factorization of
// that block continues on |d| so no NaN spreads; the host reports the error.
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) k_potrf(const PotrfTask* __restrict__ tasks, int* err) {
  extern __shared__ unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  const PotrfTask t = tasks[blockIdx.x];
  const int n = t.n, ls = n + 1;
  T* A = (T*)t.A;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    if (i >= j) S[i + j * ls] = A[(size_t)i + (size_t)j * t.ld];
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      T d = S[j + j * ls];
      if (!(d > T(0))) {
        raise_error(err, HM_ERR_NOT_SPD, t.front, j);
        d = fabs(d) > T(0) ? fabs(d) : T(1);
      }
      S[j + j * ls] = sqrt(d);
    }
    __syncthreads();
    const T inv = T(1) / S[j + j * ls];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) S[i + j * ls] *= inv;
    __syncthreads();
    const int m = n - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e % m, c = j + 1 + e / m;
      if (i >= c) S[i + c * ls] -= S[i + j * ls] * S[c + j * ls];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    if (i >= j) A[(size_t)i + (size_t)j * t.ld] = S[i + j * ls];
  }
}

template <typename T>
void launch_potrf(const PotrfTask* tasks, int ntasks, int maxn, int* err, cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t smem = (size_t)maxn * (maxn + 1) * sizeof(T);
  k_potrf<T><<<ntasks, 256, smem, s>>>(tasks, err);
}

// =====================================================================================
// B <- B L^{-T}: each of 64 threads owns one row of a 64-row slab; the row lives in
// shared memory as x[j][row] (row fastest) so the solve is conflict free.
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(64) k_trsm(const TrsmTask* __restrict__ tasks) {
  extern __shared__ unsigned char smem_raw[];
  const TrsmTask t = tasks[blockIdx.x];
  const int n = t.n, ls = n + 1;
  T* Ls = reinterpret_cast<T*>(smem_raw);
  T* X = Ls + n * ls;  // [n][64]
  const T* L = (const T*)t.L;
  T* B = (T*)t.B;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    if (i >= j) Ls[i + j * ls] = L[(size_t)i + (size_t)j * t.ldl];
  }
  const int rows = min(64, t.m - t.row0);
  for (int e = threadIdx.x; e < 64 * n; e += blockDim.x) {
    const int r = e % 64, j = e / 64;
    X[j * 64 + r] = r < rows ? B[(size_t)(t.row0 + r) + (size_t)j * t.ldb] : T(0);
  }
  __syncthreads();
  const int r = threadIdx.x;
  if (r < rows) {
    for (int j = 0; j < n; ++j) {
      T v = X[j * 64 + r];
      for (int i = 0; i < j; ++i) v -= X[i * 64 + r] * Ls[j + i * ls];
      X[j * 64 + r] = v / Ls[j + j * ls];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * n; e += blockDim.x) {
    const int rr = e % 64, j = e / 64;
    if (rr < rows) B[(size_t)(t.row0 + rr) + (size_t)j * t.ldb] = X[j * 64 + rr];
  }
}

template <typename T>
void launch_trsm(const TrsmTask* tasks, int ntasks, int maxn, cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t smem = ((size_t)maxn * (maxn + 1) + 64 * (size_t)maxn) * sizeof(T);
  k_trsm<T><<<ntasks, 64, smem, s>>>(tasks);
}

// =====================================================================================
// Woodbury core: C = [[U^T Uhat, I], [I, V^T Vhat]] (n = 2k).  The GEMMs have written the
// two diagonal k x k blocks; this kernel sets the identity blocks and inverts C by
// Gauss-Jordan elimination with partial pivoting on [C | I] (C is symmetric indefinite),
// one CTA per core.  The augmented matrix lives in shared memory when it fits, otherwise
// in place in global memory, where the core slot (C then C^{-1}, contiguous) is exactly
// the n x 2n column-major [C | C^{-1}].  A zero pivot column raises HM_ERR_BREAKDOWN.
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) k_core_lu(const CoreLuTask* __restrict__ tasks, int* err,
                                                 int use_smem) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T sval[32];
  __shared__ int sidx[32];
  __shared__ int piv_s;
  const CoreLuTask t = tasks[blockIdx.x];
  const int k = t.k, n = 2 * k;
  T* C = (T*)t.C;
  T* Ci = (T*)t.Cinv;
  T* M;
  int ld;
  T* fcol = reinterpret_cast<T*>(smem_raw);  // multipliers of the pivot column, n
  if (use_smem) {
    ld = n + 1;
    M = fcol + n;
  } else {
    ld = n;
    M = C;  // [C | Cinv] contiguous, column-major n x 2n
  }
  // assemble [C | I]
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const bool diag_blk = (i < k) == (c < k);
    const T cv = diag_blk ? C[(size_t)i + (size_t)c * n] : ((i % k == c % k) ? T(1) : T(0));
    M[i + (size_t)c * ld] = cv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, c = e / n;
    M[i + (size_t)(n + c) * ld] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < n; ++j) {
    // pivot: largest |M(i, j)|, i >= j (lowest row on ties)
    T best = T(-1);
    int bi = n;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
      const T v = fabs(M[i + (size_t)j * ld]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sval[wid] = best; sidx[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      T b = T(-1);
      int ii = n;
      for (int w = 0; w < nw; ++w)
        if (sval[w] > b || (sval[w] == b && sidx[w] < ii)) { b = sval[w]; ii = sidx[w]; }
      if (!(b > T(0))) {
        raise_error(err, HM_ERR_BREAKDOWN, t.front, j);
        ii = j;
      }
      piv_s = ii;
      t.piv[j] = ii;
    }
    __syncthreads();
    const int p = piv_s;
    if (p != j)
      for (int c = j + threadIdx.x; c < 2 * n; c += blockDim.x) {
        const T a = M[j + (size_t)c * ld];
        M[j + (size_t)c * ld] = M[p + (size_t)c * ld];
        M[p + (size_t)c * ld] = a;
      }
    __syncthreads();
    T d = M[j + (size_t)j * ld];
    if (d == T(0)) d = T(1);
    const T inv = T(1) / d;
    for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = (i == j) ? T(0) : M[i + (size_t)j * ld];
    __syncthreads();
    // scale the pivot row and eliminate column j from every other row: a warp per column,
    // lanes over rows; columns whose pivot-row entry is zero are untouched
    for (int c = j + wid; c < 2 * n; c += nw) {
      const T mjc = M[j + (size_t)c * ld] * inv;
      __syncwarp();
      if (lane == 0) M[j + (size_t)c * ld] = mjc;
      if (mjc != T(0))
        for (int i = lane; i < n; i += 32)
          if (i != j) M[i + (size_t)c * ld] -= fcol[i] * mjc;
    }
    __syncthreads();
  }
  if (use_smem)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e % n, c = e / n;
      Ci[(size_t)i + (size_t)c * n] = M[i + (size_t)(n + c) * ld];
    }
}

// =====================================================================================
// Woodbury core by its Schur complement: with A = U^T Uhat and B = V^T Vhat (the two
// diagonal k x k blocks the GEMMs wrote), C = [[A, I], [I, B]] is invertible exactly when
// M = I - A B is, and
//   C^{-1} = [[X11, X12], [X21, X22]],  X21 = M^{-1},  X11 = -B M^{-1},
//            X22 = -M^{-1} A,           X12 = I - X11 A
// (multiply out C C^{-1} = I block by block).  So one k x k Gauss-Jordan inversion with
// partial pivoting replaces the 2k x 2k one, with k steps instead of 2k.  One CTA per
// core, everything in shared memory (5 k^2 elements).  A zero pivot raises
// HM_ERR_BREAKDOWN.
// =====================================================================================

// P (k x k) = alpha * X Y (+ I if add_identity); all k x k column-major in shared memory
template <typename T>
__device__ __forceinline__ void smem_gemm(T* __restrict__ P, const T* __restrict__ X, const T* __restrict__ Y,
                                          int k, T alpha, bool add_identity) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    T s = T(0);
    for (int p = 0; p < k; ++p) s = fma(X[i + p * k], Y[p + j * k], s);
    P[e] = alpha * s + ((add_identity && i == j) ? T(1) : T(0));
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_core_inv_schur(const CoreLuTask* __restrict__ tasks, int* err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T sval[8];
  __shared__ int sidx[8];
  __shared__ int piv_s;
  const CoreLuTask t = tasks[blockIdx.x];
  const int k = t.k, n = 2 * k;
  const T* C = (const T*)t.C;
  T* Ci = (T*)t.Cinv;
  T* As = reinterpret_cast<T*>(smem_raw);  // k x k
  T* Bs = As + k * k;                      // k x k
  T* G = Bs + k * k;                       // [M | M^{-1}], k x 2k (ld k)
  T* W = G + 2 * k * k;                    // k x k work
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    As[e] = C[(size_t)i + (size_t)j * n];
    Bs[e] = C[(size_t)(k + i) + (size_t)(k + j) * n];
  }
  __syncthreads();
  smem_gemm<T>(G, As, Bs, k, T(-1), true);  // M = I - A B
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) G[k * k + e] = (e % k == e / k) ? T(1) : T(0);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    // pivot: largest |M(i, j)|, i >= j (lowest row on ties), found by warp 0
    if (wid == 0) {
      T best = T(-1);
      int bi = k;
      for (int i = j + lane; i < k; i += 32) {
        const T v = fabs(G[i + j * k]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        if (!(best > T(0))) {
          raise_error(err, HM_ERR_BREAKDOWN, t.front, j);
          bi = j;
        }
        piv_s = bi;
        t.piv[j] = bi;
      }
    }
    __syncthreads();
    const int p = piv_s;
    if (p != j)
      for (int c = j + threadIdx.x; c < 2 * k; c += blockDim.x) {
        const T a = G[j + c * k];
        G[j + c * k] = G[p + c * k];
        G[p + c * k] = a;
      }
    __syncthreads();
    T d = G[j + j * k];
    if (d == T(0)) d = T(1);
    const T inv = T(1) / d;
    // multipliers of the pivot column (W's first column), then a warp per column
    for (int i = threadIdx.x; i < k; i += blockDim.x) W[i] = (i == j) ? T(0) : G[i + j * k];
    __syncthreads();
    for (int c = j + wid; c < 2 * k; c += nw) {
      const T mjc = G[j + c * k] * inv;
      __syncwarp();
      if (lane == 0) G[j + c * k] = mjc;
      if (mjc != T(0))
        for (int i = lane; i < k; i += 32)
          if (i != j) G[i + c * k] -= W[i] * mjc;
    }
    __syncthreads();
  }
  const T* Mi = G + k * k;
  // X21 = M^{-1}; X11 = -B M^{-1} (into W); X22 = -M^{-1} A (into G's first half)
  smem_gemm<T>(W, Bs, Mi, k, T(-1), false);
  smem_gemm<T>(G, Mi, As, k, T(-1), false);
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    Ci[(size_t)i + (size_t)j * n] = W[e];                  // X11
    Ci[(size_t)(k + i) + (size_t)j * n] = Mi[e];           // X21
    Ci[(size_t)(k + i) + (size_t)(k + j) * n] = G[e];      // X22
  }
  // X12 = I - X11 A (into Bs, which is no longer needed)
  smem_gemm<T>(Bs, W, As, k, T(-1), true);
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    Ci[(size_t)i + (size_t)(k + j) * n] = Bs[e];           // X12
  }
}

template <typename T>
void launch_core_lu(const CoreLuTask* tasks, int ntasks, int maxk, int max_smem, int* err,
                    cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t schur = (size_t)5 * maxk * maxk * sizeof(T);
  if (schur + 1024 <= (size_t)max_smem) {
    k_core_inv_schur<T><<<ntasks, 256, schur, s>>>(tasks, err);
    return;
  }
  const int n = 2 * maxk;
  const size_t smem = ((size_t)(n + 1) * 2 * n + n) * sizeof(T);
  const int use = smem + 1024 <= (size_t)max_smem ? 1 : 0;
  k_core_lu<T><<<ntasks, 256, use ? smem : n * sizeof(T), s>>>(tasks, err, use);
}

// =====================================================================================
// Explicit SPD inverse from a Cholesky factor (one CTA per block, n <= 128, in shared
// memory).  L^{-1} is formed in place, last column first: with the trailing block
// already inverted, column j becomes -Linv[j+1:, j+1:] L[j+1:, j] / L[j][j] (a parallel
// triangular matrix-vector product).  Then A^{-1} = Linv^T Linv is written as a full
// n x n block, and B <- B Linv for the m rows below (64 rows per pass), optionally also
// stored transposed.
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) k_chol_inverse(const CholInvTask* __restrict__ tasks) {
  extern __shared__ unsigned char smem_raw[];
  const CholInvTask t = tasks[blockIdx.x];
  const int n = t.n, ls = n + 1;
  T* Li = reinterpret_cast<T*>(smem_raw);  // L, overwritten by Linv (lower), n x (n+1)
  T* col = Li + (size_t)n * ls;            // saved column of L, n
  T* R = col + n;                          // row slab [n][64]
  T* A = (T*)t.A;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    Li[i + j * ls] = (i >= j) ? A[(size_t)i + (size_t)j * t.ld] : T(0);
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) col[i] = Li[i + j * ls];
    __syncthreads();
    const T dinv = T(1) / col[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      T s = T(0);
      for (int k = j + 1; k <= i; ++k) s += Li[i + k * ls] * col[k];
      Li[i + j * ls] = -s * dinv;
    }
    if (threadIdx.x == 0) Li[j + j * ls] = dinv;
    __syncthreads();
  }
  // A^{-1}(i, j) = sum_{k >= max(i, j)} Linv(k, i) Linv(k, j)
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    T s = T(0);
    for (int k = max(i, j); k < n; ++k) s += Li[k + i * ls] * Li[k + j * ls];
    A[(size_t)i + (size_t)j * t.ld] = s;
  }
  if (t.m <= 0) return;
  T* B = (T*)t.B;
  for (int r0 = 0; r0 < t.m; r0 += 64) {
    const int rows = min(64, t.m - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * n; e += blockDim.x) {
      const int r = e % 64, j = e / 64;
      R[j * 64 + r] = r < rows ? B[(size_t)(r0 + r) + (size_t)j * t.ldb] : T(0);
    }
    __syncthreads();
    // row r of B Linv, column j: sum_{i >= j} B(r, i) Linv(i, j)
    for (int e = threadIdx.x; e < 64 * n; e += blockDim.x) {
      const int r = e % 64, j = e / 64;
      if (r >= rows) continue;
      T s = T(0);
      for (int i = j; i < n; ++i) s += R[i * 64 + r] * Li[i + j * ls];
      B[(size_t)(r0 + r) + (size_t)j * t.ldb] = s;
    }
    if (t.BT) {  // transpose of the finished rows (global writes of this block are visible)
      __syncthreads();
      T* BT = (T*)t.BT;
      for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
        const int j = e % n, r = e / n;
        BT[(size_t)j + (size_t)(r0 + r) * t.ldbt] = B[(size_t)(r0 + r) + (size_t)j * t.ldb];
      }
    }
  }
}

template <typename T>
void launch_chol_inverse(const CholInvTask* tasks, int ntasks, int maxn, cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t smem = ((size_t)maxn * (maxn + 1) + maxn + 64 * (size_t)maxn) * sizeof(T);
  k_chol_inverse<T><<<ntasks, 256, smem, s>>>(tasks);
}


// =====================================================================================
// Dense front in one pass: np Gauss-Jordan sweeps of the whole front F (nhat x nhat,
// rows/columns [I_p, I_p^f]) on the pivots 0 .. np-1.  The sweep on pivot k with d = F[k,k]
// sets F[i,j] -= F[i,k] F[k,j] / d (i, j != k), F[i,k] /= d, F[k,j] /= d, F[k,k] = -1/d;
// sweeps compose (the sweep operator of regression computing), and after the np sweeps
//   F = [[-F_pp^{-1}, F_pp^{-1} F_pf], [F_fp F_pp^{-1}, F_ff - F_fp F_pp^{-1} F_pf]],
// so negating the pivot block leaves exactly what the apply and the parent need:
// F_pp^{-1}, K^T beside it, K = F_fp F_pp^{-1} below it and the update matrix U_p.  For an
// SPD front every pivot is positive (a ratio of leading principal minors); a non-positive
// one raises HM_ERR_NOT_SPD and the sweep goes on with |d|.  The input is the lower
// triangle (what assembly and extend-add fill); the output is the full matrix.
// One CTA of 16 x 16 threads per front: the front is staged through shared memory with
// coalesced accesses, and thread (tx, ty) keeps the TT x TT entries (ty + 16 a, tx + 16 b)
// in registers; a sweep costs every thread TT^2 FMAs and 2 TT shared-memory reads of the
// published pivot row and column, with one barrier per sweep (double-buffered).
// =====================================================================================
template <typename T, int TT>
__global__ void __launch_bounds__(256) k_front_sweep(const SweepTask* __restrict__ tasks, int* err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T colk[2][16 * TT];
  __shared__ T rowk[2][16 * TT];
  const SweepTask t = tasks[blockIdx.x];
  const int nh = t.nhat, np = t.np, ls = nh + 1, ldf = t.ld > 0 ? t.ld : nh;
  T* S = reinterpret_cast<T*>(smem_raw);  // nh x nh staging, ld nh + 1
  T* F = (T*)t.F;
  for (int e = threadIdx.x; e < nh * nh; e += blockDim.x) S[e % nh + (e / nh) * ls] = F[e % nh + (size_t)(e / nh) * ldf];
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T a[TT][TT];
#pragma unroll
  for (int i = 0; i < TT; ++i)
#pragma unroll
    for (int j = 0; j < TT; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;  // assembly fills the lower triangle
      a[i][j] = (r < nh && c < nh) ? (r >= c ? S[r + c * ls] : S[c + r * ls]) : T(0);
    }
  // pivot k = 16 KB + kr: the block index KB is a compile-time constant of the unrolled
  // outer loop, so the owners of row / column k address their registers statically
#pragma unroll
  for (int KB = 0; KB < TT; ++KB) {
    for (int kr = 0; kr < 16; ++kr) {
      const int k = 16 * KB + kr;
      if (k >= np) break;  // uniform over the block
      const int buf = k & 1;
      if (tx == kr) {
#pragma unroll
        for (int i = 0; i < TT; ++i) colk[buf][ty + 16 * i] = a[i][KB];
      }
      if (ty == kr) {
#pragma unroll
        for (int j = 0; j < TT; ++j) rowk[buf][tx + 16 * j] = a[KB][j];
      }
      __syncthreads();
      T d = rowk[buf][k];
      if (!(d > T(0))) {
        if (threadIdx.x == 0) raise_error(err, HM_ERR_NOT_SPD, t.front, k);
        d = fabs(d) > T(0) ? fabs(d) : T(1);
      }
      const T inv = T(1) / d;
      T ci[TT], rk[TT];
#pragma unroll
      for (int i = 0; i < TT; ++i) ci[i] = colk[buf][ty + 16 * i] * inv;
#pragma unroll
      for (int j = 0; j < TT; ++j) rk[j] = rowk[buf][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) a[i][j] = fma(-ci[i], rk[j], a[i][j]);
      // row k and column k (the generic update left them at zero)
      if (tx == kr) {
#pragma unroll
        for (int i = 0; i < TT; ++i) a[i][KB] = (ty + 16 * i == k) ? -inv : ci[i];
      }
      if (ty == kr) {
#pragma unroll
        for (int j = 0; j < TT; ++j)
          if (tx + 16 * j != k) a[KB][j] = rk[j] * inv;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < TT; ++i)
#pragma unroll
    for (int j = 0; j < TT; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      if (r < nh && c < nh) S[r + c * ls] = (r < np && c < np) ? -a[i][j] : a[i][j];
    }
  __syncthreads();
  for (int e = threadIdx.x; e < nh * nh; e += blockDim.x) F[e % nh + (size_t)(e / nh) * ldf] = S[e % nh + (e / nh) * ls];
}

template <typename T>
void launch_front_sweep(const SweepTask* tasks, int ntasks, int maxn, int* err, cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t smem = (size_t)maxn * (maxn + 1) * sizeof(T);
  if (maxn <= 64) k_front_sweep<T, 4><<<ntasks, 256, smem, s>>>(tasks, err);
  else if (maxn <= 96) k_front_sweep<T, 6><<<ntasks, 256, smem, s>>>(tasks, err);
  else k_front_sweep<T, 8><<<ntasks, 256, smem, s>>>(tasks, err);
}

template void launch_potrf<float>(const PotrfTask*, int, int, int*, cudaStream_t);
template void launch_potrf<double>(const PotrfTask*, int, int, int*, cudaStream_t);
template void launch_front_sweep<float>(const SweepTask*, int, int, int*, cudaStream_t);
template void launch_front_sweep<double>(const SweepTask*, int, int, int*, cudaStream_t);
template void launch_trsm<float>(const TrsmTask*, int, int, cudaStream_t);
template void launch_trsm<double>(const TrsmTask*, int, int, cudaStream_t);
template void launch_core_lu<float>(const CoreLuTask*, int, int, int, int*, cudaStream_t);
template void launch_core_lu<double>(const CoreLuTask*, int, int, int, int*, cudaStream_t);
template void launch_chol_inverse<float>(const CholInvTask*, int, int, cudaStream_t);
template void launch_chol_inverse<double>(const CholInvTask*, int, int, cudaStream_t);

int dense_fact_setup(int max_smem) {
  HM_CUDA(allow_max_dyn_smem(k_potrf<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_potrf<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_trsm<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_trsm<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_chol_inverse<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_chol_inverse<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_lu<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_schur<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_front_sweep<float, 4>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_front_sweep<float, 6>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_front_sweep<float, 8>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_front_sweep<double, 4>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_front_sweep<double, 6>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_front_sweep<double, 8>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_schur<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_lu<double>, max_smem));
  return HM_OK;
}

}  // namespace hm
