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
// with leading dimension ld.  Thread (tx, ty) of a 16 x 16 layout computes the 4 x 4
// entries (i0 + ty + 16 a, j0 + tx + 16 b) of each 64 x 64 tile of P, so every pair of
// shared-memory loads feeds two FMAs instead of one (sums over p in order, as a plain
// inner product).  With ld odd the 16 column reads of a row of Y fall in distinct banks.
template <typename T>
__device__ __forceinline__ void smem_gemm(T* __restrict__ P, const T* __restrict__ X, const T* __restrict__ Y,
                                          int k, int ld, T alpha, bool add_identity) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int i0 = 0; i0 < k; i0 += 64)
    for (int j0 = 0; j0 < k; j0 += 64) {
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
      for (int p = 0; p < k; ++p) {
        T x[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int r = i0 + ty + 16 * a;
          x[a] = r < k ? X[r + p * ld] : T(0);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int c = j0 + tx + 16 * b;
          y[b] = c < k ? Y[p + c * ld] : T(0);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int r = i0 + ty + 16 * a, c = j0 + tx + 16 * b;
          if (r < k && c < k) P[r + c * ld] = alpha * acc[a][b] + ((add_identity && r == c) ? T(1) : T(0));
        }
    }
}

// Rows per lane in the Gauss-Jordan steps (k <= 32 kCoreRows).
constexpr int kCoreRows = 4;

template <typename T>
__global__ void __launch_bounds__(256) k_core_inv_schur(const CoreLuTask* __restrict__ tasks, int* err) {
  extern __shared__ unsigned char smem_raw[];
  const CoreLuTask t = tasks[blockIdx.x];
  const int k = t.k, n = 2 * k, ld = k | 1;
  const T* C = (const T*)t.C;
  T* Ci = (T*)t.Cinv;
  T* As = reinterpret_cast<T*>(smem_raw);  // k x k (ld)
  T* Bs = As + ld * k;                     // k x k
  T* G = Bs + ld * k;                      // [M | M^{-1}], k x 2k (ld)
  T* W = G + 2 * ld * k;                   // k x k work
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < k; c += nw)
    for (int i = lane; i < k; i += 32) {
      As[i + c * ld] = C[(size_t)i + (size_t)c * n];
      Bs[i + c * ld] = C[(size_t)(k + i) + (size_t)(k + c) * n];
      G[i + (k + c) * ld] = i == c ? T(1) : T(0);
    }
  __syncthreads();
  smem_gemm<T>(G, As, Bs, k, ld, T(-1), true);  // M = I - A B
  __syncthreads();
  // [M | I] -> [. | M^{-1}] by Gauss-Jordan with partial pivoting.  Each warp reads the
  // multipliers (column j) and picks the pivot itself, and owns whole columns of the
  // working set (c > j; column j is only read), so the swap and the elimination need no
  // barrier and a step ends with one.
  for (int j = 0; j < k; ++j) {
    T m[kCoreRows];
    T best = T(-1);
    int bi = k;
#pragma unroll
    for (int r = 0; r < kCoreRows; ++r) {
      const int i = lane + 32 * r;
      m[r] = i < k ? G[i + j * ld] : T(0);
      if (i >= j && i < k) {
        const T v = fabs(m[r]);
        if (v > best) { best = v; bi = i; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {  // largest |M(i, j)|, i >= j, lowest row on ties
      const T ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    const bool ok = best > T(0);
    const int p = ok ? bi : j;
    if (threadIdx.x == 0) {
      if (!ok) raise_error(err, HM_ERR_BREAKDOWN, t.front, j);
      t.piv[j] = p;
    }
    T d = G[p + j * ld];
    if (d == T(0)) d = T(1);
    const T inv = T(1) / d;
    const T mjj = G[j + j * ld];  // the multiplier of row p after the swap
    for (int c = j + 1 + wid; c < 2 * k; c += nw) {
      const T mjc = G[p + c * ld] * inv;  // new pivot row (old row p), scaled
      const T rj = G[j + c * ld];         // old row j, moving to row p
      __syncwarp();
#pragma unroll
      for (int r = 0; r < kCoreRows; ++r) {
        const int i = lane + 32 * r;
        if (i < k) {
          T v;
          if (i == j) v = mjc;
          else if (i == p) v = rj - mjj * mjc;
          else v = G[i + c * ld] - m[r] * mjc;
          G[i + c * ld] = v;
        }
      }
    }
    __syncthreads();
  }
  const T* Mi = G + ld * k;
  // X21 = M^{-1}; X11 = -B M^{-1} (into W); X22 = -M^{-1} A (into G's first half)
  smem_gemm<T>(W, Bs, Mi, k, ld, T(-1), false);
  smem_gemm<T>(G, Mi, As, k, ld, T(-1), false);
  __syncthreads();
  for (int c = wid; c < k; c += nw)
    for (int i = lane; i < k; i += 32) {
      Ci[(size_t)i + (size_t)c * n] = W[i + c * ld];                  // X11
      Ci[(size_t)(k + i) + (size_t)c * n] = Mi[i + c * ld];           // X21
      Ci[(size_t)(k + i) + (size_t)(k + c) * n] = G[i + c * ld];      // X22
    }
  // X12 = I - X11 A (into Bs, which is no longer needed)
  smem_gemm<T>(Bs, W, As, k, ld, T(-1), true);
  __syncthreads();
  for (int c = wid; c < k; c += nw)
    for (int i = lane; i < k; i += 32) Ci[(size_t)i + (size_t)(k + c) * n] = Bs[i + c * ld];  // X12
}

// P (k x k) = alpha * X Y (+ I if add_identity), k <= 16 RA, column-major in shared memory
// (ld): thread (tx, ty) of a 16 x 16 layout computes the RA x RA entries
// (ty + 16 a, tx + 16 b), sums over p in order.
template <typename T, int RA>
__device__ __forceinline__ void smem_gemm_r(T* __restrict__ P, const T* __restrict__ X, const T* __restrict__ Y,
                                            int k, int ld, T alpha, bool add_identity) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[RA][RA];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < RA; ++b) acc[a][b] = T(0);
  for (int p = 0; p < k; ++p) {
    T x[RA], y[RA];
#pragma unroll
    for (int a = 0; a < RA; ++a) {
      const int r = ty + 16 * a;
      x[a] = r < k ? X[r + p * ld] : T(0);
    }
#pragma unroll
    for (int b = 0; b < RA; ++b) {
      const int c = tx + 16 * b;
      y[b] = c < k ? Y[p + c * ld] : T(0);
    }
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int b = 0; b < RA; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < RA; ++b) {
      const int r = ty + 16 * a, c = tx + 16 * b;
      if (r < k && c < k) P[r + c * ld] = alpha * acc[a][b] + ((add_identity && r == c) ? T(1) : T(0));
    }
}

// The same Woodbury core inverse for k <= 16 RA with [M | I] held in registers: thread
// (tx, ty) keeps rows ty + 16 a and columns tx + 16 b of the k x 2k working matrix.
// Gauss-Jordan with partial pivoting by row selection instead of row swaps: step j takes
// as pivot the unused row p_j with the largest |M(p_j, j)| (lowest row on ties), scales
// it and eliminates column j from every other row.  The row operations E then satisfy
// E M = Pi with Pi(p_j, j) = 1, so row j of M^{-1} = Pi^T E is row p_j of the right half.
// A step costs two barriers (the candidates of column j, then the pivot row) and RA x 2RA
// FMAs per thread; the multipliers and the pivot row go through double-buffered shared
// memory.
template <typename T, int RA>
__global__ void __launch_bounds__(256) k_core_inv_reg(const CoreLuTask* __restrict__ tasks, int* err) {
  constexpr int RB = 2 * RA;
  extern __shared__ unsigned char smem_raw[];
  __shared__ T pcol[2][16 * RA];  // column j, by row
  __shared__ T prow[2][32 * RA];  // pivot row, by column
  __shared__ T cabs[2][16], cval[2][16];
  __shared__ int cidx[2][16];
  __shared__ int invp[16 * RA];
  const CoreLuTask t = tasks[blockIdx.x];
  const int k = t.k, n = 2 * k, ld = k | 1;
  const T* C = (const T*)t.C;
  T* Ci = (T*)t.Cinv;
  T* As = reinterpret_cast<T*>(smem_raw);  // k x k (ld)
  T* Bs = As + ld * k;
  T* Mi = Bs + ld * k;                     // M, then M^{-1}
  T* W = Mi + ld * k;
  T* P2 = W + ld * k;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int c = wid; c < k; c += nw)
    for (int i = lane; i < k; i += 32) {
      As[i + c * ld] = C[(size_t)i + (size_t)c * n];
      Bs[i + c * ld] = C[(size_t)(k + i) + (size_t)(k + c) * n];
    }
  __syncthreads();
  smem_gemm_r<T, RA>(Mi, As, Bs, k, ld, T(-1), true);  // M = I - A B
  __syncthreads();
  T g[RA][RB];
  bool used[RA];
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    used[a] = false;
    const int r = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const int c = tx + 16 * b;
      g[a][b] = r >= k ? T(0) : c < k ? Mi[r + c * ld] : (c - k == r ? T(1) : T(0));
    }
  }
  // pivot column j = 16 JB + jt: JB is a compile-time constant of the unrolled loop, so
  // the owners of column j address their registers statically
#pragma unroll
  for (int JB = 0; JB < RA; ++JB) {
    for (int jt = 0; jt < 16; ++jt) {
      const int j = 16 * JB + jt;
      if (j >= k) break;  // uniform over the block
      const int buf = j & 1;
      if (tx == jt) {
        T best = T(-1), bval = T(0);
        int bi = k;
#pragma unroll
        for (int a = 0; a < RA; ++a) {
          const int r = ty + 16 * a;
          if (r < k) {
            const T v = g[a][JB];
            pcol[buf][r] = v;
            if (!used[a] && fabs(v) > best) { best = fabs(v); bi = r; bval = v; }
          }
        }
        cabs[buf][ty] = best;
        cidx[buf][ty] = bi;
        cval[buf][ty] = bval;
      }
      __syncthreads();
      T best = T(-1), d = T(0);
      int p = k;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const T v = cabs[buf][q];
        const int i = cidx[buf][q];
        if (v > best || (v == best && i < p)) { best = v; p = i; d = cval[buf][q]; }
      }
      if (threadIdx.x == 0) {
        if (!(best > T(0))) raise_error(err, HM_ERR_BREAKDOWN, t.front, j);
        t.piv[j] = p;
        invp[p] = j;
      }
      if (d == T(0)) d = T(1);
      const T inv = T(1) / d;
      const int pa = p >> 4;
      const bool prow_owner = ty == (p & 15);
      if (prow_owner) {
#pragma unroll
        for (int a = 0; a < RA; ++a)
          if (a == pa) {
            used[a] = true;
#pragma unroll
            for (int b = 0; b < RB; ++b) prow[buf][tx + 16 * b] = g[a][b];
          }
      }
      __syncthreads();
      T pr[RB];
#pragma unroll
      for (int b = 0; b < RB; ++b) pr[b] = prow[buf][tx + 16 * b] * inv;
#pragma unroll
      for (int a = 0; a < RA; ++a) {
        const int r = ty + 16 * a;
        const T mult = r < k ? pcol[buf][r] : T(0);
        const bool isp = prow_owner && a == pa;
#pragma unroll
        for (int b = 0; b < RB; ++b) g[a][b] = isp ? pr[b] : g[a][b] - mult * pr[b];
      }
    }
  }
  __syncthreads();  // invp complete; M no longer read
  // M^{-1}(invp[r], c) = E(r, c) for the right-half columns
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int r = ty + 16 * a;
    if (r < k) {
      const int row = invp[r];
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int c = tx + 16 * b - k;
        if (c >= 0 && c < k) Mi[row + c * ld] = g[a][b];
      }
    }
  }
  __syncthreads();
  // X21 = M^{-1}; X11 = -B M^{-1} (W); X22 = -M^{-1} A (P2); X12 = I - X11 A (Bs)
  smem_gemm_r<T, RA>(W, Bs, Mi, k, ld, T(-1), false);
  smem_gemm_r<T, RA>(P2, Mi, As, k, ld, T(-1), false);
  __syncthreads();
  smem_gemm_r<T, RA>(Bs, W, As, k, ld, T(-1), true);
  for (int c = wid; c < k; c += nw)
    for (int i = lane; i < k; i += 32) {
      Ci[(size_t)i + (size_t)c * n] = W[i + c * ld];              // X11
      Ci[(size_t)(k + i) + (size_t)c * n] = Mi[i + c * ld];       // X21
      Ci[(size_t)(k + i) + (size_t)(k + c) * n] = P2[i + c * ld];  // X22
    }
  __syncthreads();
  for (int c = wid; c < k; c += nw)
    for (int i = lane; i < k; i += 32) Ci[(size_t)i + (size_t)(k + c) * n] = Bs[i + c * ld];  // X12
}

template <typename T>
void launch_core_lu(const CoreLuTask* tasks, int ntasks, int maxk, int max_smem, int* err,
                    cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t schur = (size_t)5 * (maxk | 1) * maxk * sizeof(T);
  if (maxk <= 64 && schur + 1024 <= (size_t)max_smem) {
    if (maxk <= 16) k_core_inv_reg<T, 1><<<ntasks, 256, schur, s>>>(tasks, err);
    else if (maxk <= 32) k_core_inv_reg<T, 2><<<ntasks, 256, schur, s>>>(tasks, err);
    else if (maxk <= 48) k_core_inv_reg<T, 3><<<ntasks, 256, schur, s>>>(tasks, err);
    else k_core_inv_reg<T, 4><<<ntasks, 256, schur, s>>>(tasks, err);
    return;
  }
  if (maxk <= 32 * kCoreRows && schur + 1024 <= (size_t)max_smem) {
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
// (a0, a1) += m (r0, r1) by one packed FP32 instruction (fma.rn.f32x2: the two lanes
// are the same round-to-nearest FMAs as two fma.rn.f32).
__device__ __forceinline__ void fma_pair_f32(float& a0, float& a1, float m, float r0, float r1) {
  asm("{\n.reg .b64 acc, mm, rr;\n"
      "mov.b64 acc, {%0, %1};\n"
      "mov.b64 mm, {%2, %2};\n"
      "mov.b64 rr, {%3, %4};\n"
      "fma.rn.f32x2 acc, mm, rr, acc;\n"
      "mov.b64 {%0, %1}, acc;\n}"
      : "+f"(a0), "+f"(a1)
      : "f"(m), "f"(r0), "f"(r1));
}
__device__ __forceinline__ void fma_pair_f32(double&, double&, double, double, double) {}

template <typename T, int TT>
__global__ void __launch_bounds__(256) k_front_sweep(const SweepTask* __restrict__ tasks, int* err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T colk[2][16 * TT];
  __shared__ T rowk[2][16 * TT];
  const SweepTask t = tasks[blockIdx.x];
  const int nh = t.nhat, np = t.np, ls = nh + 1, ldf = t.ld > 0 ? t.ld : nh;
  T* S = reinterpret_cast<T*>(smem_raw);  // nh x nh staging, ld nh + 1
  T* F = (T*)t.F;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // lower triangle in, a warp per column (no index division)
  for (int c = warp; c < nh; c += 8)
    for (int r = c + lane; r < nh; r += 32) S[r + c * ls] = F[r + (size_t)c * ldf];
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
      const T inv = recip_rn(d);
      T ci[TT], rk[TT];
#pragma unroll
      for (int i = 0; i < TT; ++i) ci[i] = colk[buf][ty + 16 * i] * inv;
#pragma unroll
      for (int j = 0; j < TT; ++j) rk[j] = rowk[buf][tx + 16 * j];
      if constexpr (sizeof(T) == 4) {  // two FMAs per instruction (packed FP32 pairs)
#pragma unroll
        for (int i = 0; i < TT; ++i)
#pragma unroll
          for (int j = 0; j < TT; j += 2) fma_pair_f32(a[i][j], a[i][j + 1], -ci[i], rk[j], rk[j + 1]);
      } else {
#pragma unroll
        for (int i = 0; i < TT; ++i)
#pragma unroll
          for (int j = 0; j < TT; ++j) a[i][j] = fma(-ci[i], rk[j], a[i][j]);
      }
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
  T* P = (T*)t.P;
  const int ldp = t.ldp > 0 ? t.ldp : np, nu = nh - np;
  T* PK = P + packed_k_offset(np, nh, (int)sizeof(T));
  for (int c = warp; c < nh; c += 8) {  // one pass over the column, each entry to its store
    for (int r = lane; r < nh; r += 32) {
      const T v = S[r + c * ls];
      if (r < np) P[r + (size_t)c * ldp] = v;
      else if (c < np) PK[(r - np) + (size_t)c * nu] = v;
      else if (r >= c) F[r + (size_t)c * ldf] = v;  // U_p: the lower triangle only
    }
  }
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
  HM_CUDA(allow_max_dyn_smem(k_core_inv_schur<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_reg<float, 1>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_reg<float, 2>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_reg<float, 3>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_reg<float, 4>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_reg<double, 1>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_reg<double, 2>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_reg<double, 3>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_core_inv_reg<double, 4>, max_smem));
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
