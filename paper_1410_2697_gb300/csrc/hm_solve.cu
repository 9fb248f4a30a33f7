// hm_solve.cu -- preconditioner apply z = M^{-1} r: the multifrontal upward pass
// (Eq. upward: b_f <- b_f - F_fp F_pp^-1 b_p, leaves to root) and downward pass
// (Eq. downward: x_p = F_pp^-1 (b_p - F_pf x_f), root to leaves), with the HODLR pivot
// solves and low-rank coupling blocks of Section 4.2.2 for HODLR fronts.
//
// Every front p owns a vector block fv_p (nhat_p x nrhs, nhat_p = |I_p| + |I_p^f|).
// Dense fronts run one fused kernel per level and pass.  Upward: fv_p = [r(I_p); 0], the
// children's update parts added through the relative maps (children in a fixed order),
// then b_f <- b_f - K b_p with K = F_fp F_pp^{-1} kept by the factorization.  Downward:
// x_p = F_pp^{-1} b_p - K^T x_f as one product with the first np rows of the front,
// [F_pp^{-1} | K^T] (K^T is stored beside the pivot block), so both passes read the
// front with one row per thread.  HODLR fronts use flat vector kernels and batched GEMMs:
// Vf^T F_pp^{-1} = Vtilde^T (F_pp^HODLR is symmetric), so the upward coupling is
// b_f -= W (Vtilde^T b_p) with no pivot solve; downward, y = F_pp^{-1} b_p by recursive
// Woodbury (explicit leaf inverses, then per level y -= Zhat C^{-1} Z^T y with explicit
// core inverses) and x_p = y - Vtilde (W^T x_f).  Nothing is solved by sequential
// substitution.
#include <algorithm>

#include "hm_internal.h"

namespace hm {

// Flat vector kernels of the apply: one warp per (front, right-hand side, chunk of 256
// rows); grid = (ceil(fronts / 8), nrhs, chunks), 8 warps per block.
constexpr int kVecChunk = 256;

// The vector assembly loops go kLdBatch iterations at a time, all loads of the batch
// before its stores: the compiler must assume that a store may alias a later load, so
// one load-then-store iteration at a time waits a full memory round trip (two where an
// index is loaded first) per element.  A batch slot past the end reads an in-range
// element (its index is clamped) and stores nothing.
constexpr int kLdBatch = 4;

// Upward assembly of HODLR fronts in one launch: one block per (front, right-hand side)
// forms fv_q = [r(I_q); 0] and adds the children's update parts through the relative
// maps, one child after another (a fixed order of the sums).
template <typename T>
__global__ void __launch_bounds__(256) k_vassemble(const int* __restrict__ fronts, int n,
                                                   const T* __restrict__ win, const int32_t* __restrict__ first,
                                                   const int* __restrict__ npiv, const int* __restrict__ nhat,
                                                   const int64_t* __restrict__ fvoff,
                                                   const int32_t* __restrict__ child_ptr,
                                                   const int32_t* __restrict__ child_list,
                                                   const int64_t* __restrict__ ifoff,
                                                   const int32_t* __restrict__ relmap, T* __restrict__ FV) {
  const int q = fronts[blockIdx.x], r = blockIdx.y;
  const int np = npiv[q], nh = nhat[q];
  T* fv = FV + fvoff[q] + (int64_t)r * nh;
  const T* w = win + first[q] + (int64_t)r * n;
  for (int e = threadIdx.x; e < nh; e += blockDim.x) fv[e] = e < np ? w[e] : T(0);
  for (int ci = child_ptr[q]; ci < child_ptr[q + 1]; ++ci) {
    __syncthreads();
    const int c = child_list[ci];
    const int npc = npiv[c], nhc = nhat[c], nuc = nhc - npc;
    const T* fc = FV + fvoff[c] + npc + (int64_t)r * nhc;
    const int32_t* rm = relmap + ifoff[c];
    for (int t0 = threadIdx.x; t0 < nuc; t0 += blockDim.x * kLdBatch) {
      int d[kLdBatch];
      T a[kLdBatch], o[kLdBatch];
#pragma unroll
      for (int u = 0; u < kLdBatch; ++u) {
        const int t = min(t0 + u * (int)blockDim.x, nuc - 1);
        d[u] = rm[t];
        a[u] = fc[t];
      }
#pragma unroll
      for (int u = 0; u < kLdBatch; ++u) o[u] = fv[d[u]];
#pragma unroll
      for (int u = 0; u < kLdBatch; ++u)  // relmap is injective: no two updates meet
        if (t0 + u * (int)blockDim.x < nuc) fv[d[u]] = o[u] + a[u];
    }
  }
}

// Downward gather: fv_q[np + t] = -x(I_q^f[t]) (negated, so that a dense front's solve
// is the single product x_p = [F_pp^{-1}; K]^T fv_q).
template <typename T>
__global__ void __launch_bounds__(256) k_vgather(const int* __restrict__ fronts, int nfronts, int n,
                                                 const T* __restrict__ xv, const int* __restrict__ npiv,
                                                 const int* __restrict__ nhat,
                                                 const int64_t* __restrict__ fvoff,
                                                 const int64_t* __restrict__ ifoff,
                                                 const int32_t* __restrict__ iflist, T* __restrict__ FV) {
  const int fi = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (fi >= nfronts) return;
  const int q = fronts[fi], r = blockIdx.y;
  const int np = npiv[q], nh = nhat[q], nu = nh - np;
  const int e0 = blockIdx.z * kVecChunk, e1 = min(nu, e0 + kVecChunk);
  if (e0 >= e1) return;
  T* fv = FV + fvoff[q] + np + (int64_t)r * nh;
  const int32_t* If = iflist + ifoff[q];
  const T* x = xv + (int64_t)r * n;
  for (int t0 = e0 + lane; t0 < e1; t0 += 32 * kLdBatch) {
    int g[kLdBatch];
    T v[kLdBatch];
#pragma unroll
    for (int u = 0; u < kLdBatch; ++u) g[u] = If[min(t0 + 32 * u, e1 - 1)];
#pragma unroll
    for (int u = 0; u < kLdBatch; ++u) v[u] = -x[g[u]];
#pragma unroll
    for (int u = 0; u < kLdBatch; ++u) {
      const int t = t0 + 32 * u;
      if (t < e1) fv[t] = v[u];
    }
  }
}

// -------------------------------------------------------------------------------------
// Dense fronts: one block of 256 threads per (front, group of RB right-hand sides).
// Both passes are row-block products M (rows x kdim, column-major) times a staged
// block X (kdim x RB) with one row of M per thread, so consecutive threads read
// consecutive rows of a column (coalesced) and every thread reads the same X entries
// (shared-memory broadcast).  When a front has fewer than 256 rows, the reduction
// dimension is split over S warp slices whose partial sums meet in shared memory.
//   up:   f -= K b_p,            K = F_fp F_pp^{-1}  (nu x np, below the pivot block)
//   down: x_p = [F_pp^{-1} | K^T] [b_p; -x_f]        (np x nhat, the first np rows)
// -------------------------------------------------------------------------------------
constexpr int kDenseKC = 256;  // rows of the staged block per chunk in the down pass

__device__ __forceinline__ int pow2_floor8(int v) { return v >= 8 ? 8 : v >= 4 ? 4 : v >= 2 ? 2 : 1; }

// acc[r] += sum_{k in [k0, k1)} M[row + k ld] X[(k - kx) RB + r]; eight loads of M are
// issued before their products, so each thread keeps several HBM requests in flight.
template <typename T, int RB>
__device__ __forceinline__ void rowblock_acc(const T* __restrict__ M, int64_t ld, int row, int k0, int k1,
                                             const T* __restrict__ X, int kx, T (&acc)[RB]) {
  constexpr int U = 8;
  int k = k0;
  for (; k + U <= k1; k += U) {
    T m[U];
#pragma unroll
    for (int u = 0; u < U; ++u) m[u] = M[row + (int64_t)(k + u) * ld];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const T* x = X + (k + u - kx) * RB;
#pragma unroll
      for (int r = 0; r < RB; ++r) acc[r] = fma(m[u], x[r], acc[r]);
    }
  }
  for (; k < k1; ++k) {
    const T m = M[row + (int64_t)k * ld];
    const T* x = X + (k - kx) * RB;
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = fma(m, x[r], acc[r]);
  }
}

// Adds the partial sums of the S - 1 other slices of a warp group into acc of the group's
// first warp (warps g S .. g S + S - 1 form group g).  Every thread of the block calls it.
template <typename T, int RB>
__device__ __forceinline__ void slice_reduce(T* __restrict__ red, int S, T (&acc)[RB]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < RB; ++r) red[(warp * RB + r) * 32 + lane] = acc[r];
  __syncthreads();
  if (warp % S == 0)
    for (int s = 1; s < S; ++s) {
#pragma unroll
      for (int r = 0; r < RB; ++r) acc[r] += red[((warp + s) * RB + r) * 32 + lane];
    }
  __syncthreads();
}

// Upward pass of a dense front, NT threads.  The whole front vector [b_p; b_f] for RB
// right-hand sides is formed in shared memory (r(I_p), then the children's update parts
// through the relative maps, one child after another), then b_f -= K b_p with one row
// of K per thread, and [b_p; b_f] is written to fv once.  The packed factor of front q
// starts at D + cf_off[q]: [F_pp^-1 | K^T] (np x nhat, ld np), then K (nu x np, ld nu)
// at packed_k_offset.
template <typename T, int RB, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_dense_up(const int* __restrict__ fronts, int nrhs, int n,
                                                 const T* __restrict__ win, const int32_t* __restrict__ first,
                                                 const int* __restrict__ npiv, const int* __restrict__ nhat,
                                                 const int64_t* __restrict__ cf_off,
                                                 const int64_t* __restrict__ fvoff,
                                                 const int32_t* __restrict__ child_ptr,
                                                 const int32_t* __restrict__ child_list,
                                                 const int64_t* __restrict__ ifoff,
                                                 const int32_t* __restrict__ relmap, const T* __restrict__ D,
                                                 T* __restrict__ FV, int smem_rows) {
  constexpr int W = NT / 32;
  extern __shared__ unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);  // nhat x RB, row-major
  T* red = X + smem_rows * RB;            // W x RB x 32
  const int q = fronts[blockIdx.x];
  const int r0 = blockIdx.y * RB, nr = min(RB, nrhs - r0);
  const int np = npiv[q], nh = nhat[q], nu = nh - np, b0 = first[q];
  // one row per thread, its loads eight at a time in flight (as in the downward pass)
  constexpr int VB = RB < 8 ? RB : 8;
  for (int i = threadIdx.x; i < nh; i += NT) {
    const T* src = win + b0 + i + (int64_t)r0 * n;
#pragma unroll
    for (int rb = 0; rb < RB; rb += VB) {
      T v[VB];
#pragma unroll
      for (int r = 0; r < VB; ++r) v[r] = (i < np && rb + r < nr) ? src[(int64_t)(rb + r) * n] : T(0);
#pragma unroll
      for (int r = 0; r < VB; ++r) X[i * RB + rb + r] = v[r];
    }
  }
  __syncthreads();
  for (int ci = child_ptr[q]; ci < child_ptr[q + 1]; ++ci) {
    const int c = child_list[ci];
    const int npc = npiv[c], nhc = nhat[c], nuc = nhc - npc;
    const T* fc = FV + fvoff[c] + npc;
    const int32_t* rm = relmap + ifoff[c];
    for (int t = threadIdx.x; t < nuc; t += NT) {  // the child's rows go to distinct rows here
      const T* src = fc + t + (int64_t)r0 * nhc;
      T* dst = X + rm[t] * RB;
#pragma unroll
      for (int rb = 0; rb < RB; rb += VB) {
        T v[VB];
#pragma unroll
        for (int r = 0; r < VB; ++r) v[r] = rb + r < nr ? src[(int64_t)(rb + r) * nhc] : T(0);
#pragma unroll
        for (int r = 0; r < VB; ++r) dst[rb + r] += v[r];
      }
    }
    __syncthreads();
  }
  T* fv = FV + fvoff[q];
  for (int e = threadIdx.x; e < np * nr; e += NT) {
    const int i = e % np, r = e / np;
    fv[i + (int64_t)(r0 + r) * nh] = X[i * RB + r];
  }
  if (nu == 0) return;
  const T* K = D + cf_off[q] + packed_k_offset(np, nh, (int)sizeof(T));  // nu x np, ld nu
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrc = (nu + 31) / 32, ng = min(W, pow2_floor8(nrc)), S = W / ng;
  const int g = warp / S, sl = warp % S;
  const int j0 = sl * np / S, j1 = (sl + 1) * np / S;
  for (int base = 0; base < nrc; base += ng) {
    const int t = (base + g) * 32 + lane;
    const bool active = base + g < nrc && t < nu;
    T acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = T(0);
    if (active) rowblock_acc<T, RB>(K, nu, t, j0, j1, X, 0, acc);
    if (S > 1) slice_reduce<T, RB>(red, S, acc);
    if (active && sl == 0) {
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if (r < nr) fv[np + t + (int64_t)(r0 + r) * nh] = X[(np + t) * RB + r] - acc[r];
    }
  }
}

// Downward pass of a dense front, NT threads: x_p = [F_pp^{-1} | K^T] [b_p; -x(I_p^f)],
// the right-hand block staged in chunks of kDenseKC rows, one row of the product per
// thread.
template <typename T, int RB, int NT>
__global__ void __launch_bounds__(NT) k_dense_down(const int* __restrict__ fronts, int nrhs, int n,
                                                   T* __restrict__ xv, const int32_t* __restrict__ first,
                                                   const int* __restrict__ npiv, const int* __restrict__ nhat,
                                                   const int64_t* __restrict__ cf_off,
                                                   const int64_t* __restrict__ fvoff,
                                                   const int64_t* __restrict__ ifoff,
                                                   const int32_t* __restrict__ iflist, const T* __restrict__ D,
                                                   const T* __restrict__ FV, int smem_rows) {
  constexpr int W = NT / 32;
  extern __shared__ unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);  // smem_rows x RB
  T* red = X + smem_rows * RB;
  const int q = fronts[blockIdx.x];
  const int r0 = blockIdx.y * RB, nr = min(RB, nrhs - r0);
  const int np = npiv[q], nh = nhat[q], b0 = first[q];
  const T* fv = FV + fvoff[q];
  const int32_t* If = iflist + ifoff[q];
  const T* H = D + cf_off[q];  // np x nhat, ld np; row j: [F_pp^{-1}(j, :) | K^T(j, :)]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrc = (np + 31) / 32, ng = min(W, pow2_floor8(nrc)), S = W / ng;
  const int g = warp / S, sl = warp % S;
  for (int base = 0; base < nrc; base += ng) {
    const int j = (base + g) * 32 + lane;
    const bool active = base + g < nrc && j < np;
    T acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = T(0);
    for (int kc0 = 0; kc0 < nh; kc0 += smem_rows) {
      const int kc1 = min(nh, kc0 + smem_rows), len = kc1 - kc0;
      __syncthreads();
      // one row of the right-hand block per thread: its loads are independent, so they
      // go in flight eight at a time (the update rows gather x through I_p^f)
      constexpr int VB = RB < 8 ? RB : 8;
      for (int i = kc0 + threadIdx.x; i < kc1; i += NT) {
        const bool piv = i < np;
        const T* src = piv ? fv + i + (int64_t)r0 * nh : xv + If[i - np] + (int64_t)r0 * n;
        const int64_t ld = piv ? nh : n;
        const T sgn = piv ? T(1) : T(-1);
        T* dst = X + (i - kc0) * RB;
#pragma unroll
        for (int rb = 0; rb < RB; rb += VB) {
          T v[VB];
#pragma unroll
          for (int r = 0; r < VB; ++r) v[r] = rb + r < nr ? src[(int64_t)(rb + r) * ld] : T(0);
#pragma unroll
          for (int r = 0; r < VB; ++r) dst[rb + r] = sgn * v[r];
        }
      }
      __syncthreads();
      if (active) rowblock_acc<T, RB>(H, np, j, kc0 + sl * len / S, kc0 + (sl + 1) * len / S, X, kc0, acc);
    }
    if (S > 1) slice_reduce<T, RB>(red, S, acc);
    if (active && sl == 0) {
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if (r < nr) xv[b0 + j + (int64_t)(r0 + r) * n] = acc[r];
    }
  }
}

static int rhs_block(int nrhs) { return nrhs >= 16 ? 16 : nrhs > 4 ? 8 : nrhs > 2 ? 4 : nrhs; }

// 64 threads per front when every front of the level is small (more fronts in flight per
// SM); 256 otherwise.  The autotuner's variants 1 and 3 take the other width, 2 and 3 a
// quarter of the right-hand sides per block (four times the blocks, for levels with few
// fronts; each block reads the front again).
static uint64_t dense_sig(const LevelSolvePlan& lp, int nrhs) {
  Sig sg;
  sg << nrhs << lp.dense.count << lp.dense_max_nhat << lp.dense_max_np;
  return sg.h;
}
static bool narrow_level(const hm_ctx_s* ctx, int site, const LevelSolvePlan& lp, int nrhs) {
  const int v = ctx->tune.variant(site, dense_sig(lp, nrhs));
  return (lp.dense_max_nhat <= 128) != (v == 1 || v == 3);
}
static int dense_rhs_block(const hm_ctx_s* ctx, int site, const LevelSolvePlan& lp, int nrhs) {
  const int rb = rhs_block(nrhs);
  return ctx->tune.variant(site, dense_sig(lp, nrhs)) >= 2 ? std::max(1, rb / 4) : rb;
}

template <typename T, int RB, int NT>
static void dense_up_launch(const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys,
                            SolvePlan* sp, int nrhs, const T* win, cudaStream_t s) {
  const Plan& P = sys->plan;
  const int rows = lp.dense_max_nhat;
  const size_t smem = sizeof(T) * (size_t)RB * (rows + NT);
  const dim3 grid((unsigned)lp.dense.count, (unsigned)((nrhs + RB - 1) / RB));
  k_dense_up<T, RB, NT><<<grid, NT, smem, s>>>(lp.dense.dev(base), nrhs, sys->n, win, sys->d_first, P.d_np,
                                               P.d_nhat, P.d_cf_off, sp->d_fvoff, sys->d_child_ptr,
                                               sys->d_child_list, sys->d_ifoff, sys->d_relmap,
                                               (const T*)sys->d_dfac, (T*)sp->d_fv, rows);
}

template <typename T, int RB, int NT>
static void dense_down_launch(const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys,
                              SolvePlan* sp, int nrhs, T* xv, cudaStream_t s) {
  const Plan& P = sys->plan;
  const int rows = std::min(lp.dense_max_nhat, kDenseKC);
  const size_t smem = sizeof(T) * (size_t)RB * (rows + NT);
  const dim3 grid((unsigned)lp.dense.count, (unsigned)((nrhs + RB - 1) / RB));
  k_dense_down<T, RB, NT><<<grid, NT, smem, s>>>(lp.dense.dev(base), nrhs, sys->n, xv, sys->d_first, P.d_np,
                                                 P.d_nhat, P.d_cf_off, sp->d_fvoff, sys->d_ifoff,
                                                 sys->d_iflist, (const T*)sys->d_dfac, (const T*)sp->d_fv,
                                                 rows);
}

template <typename T, int RB>
static void dense_up_rb(const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys, SolvePlan* sp,
                        int nrhs, const T* win, cudaStream_t s) {
  if (narrow_level(sys->ctx, TS_DENSE_UP, lp, nrhs)) dense_up_launch<T, RB, 64>(lp, base, sys, sp, nrhs, win, s);
  else dense_up_launch<T, RB, 256>(lp, base, sys, sp, nrhs, win, s);
}

template <typename T, int RB>
static void dense_down_rb(const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys, SolvePlan* sp,
                          int nrhs, T* xv, cudaStream_t s) {
  if (narrow_level(sys->ctx, TS_DENSE_DOWN, lp, nrhs)) dense_down_launch<T, RB, 64>(lp, base, sys, sp, nrhs, xv, s);
  else dense_down_launch<T, RB, 256>(lp, base, sys, sp, nrhs, xv, s);
}

// Right-hand sides per block of the upward kernel: the block of the whole front vector
// must fit in shared memory next to the reduction buffer.
template <typename T>
static int up_rhs_block(const hm_ctx_s* ctx, const LevelSolvePlan& lp, int nrhs, int max_smem) {
  const int nt = narrow_level(ctx, TS_DENSE_UP, lp, nrhs) ? 64 : 256;
  int rb = dense_rhs_block(ctx, TS_DENSE_UP, lp, nrhs);
  while (rb > 1 && sizeof(T) * (size_t)rb * (lp.dense_max_nhat + nt) > (size_t)max_smem) rb /= 2;
  return rb;
}

template <typename T>
static int dense_up(const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys, SolvePlan* sp,
                    int nrhs, const T* win, cudaStream_t s) {
  const int rb = up_rhs_block<T>(sys->ctx, lp, nrhs, sys->ctx->max_smem);
  if (sizeof(T) * (size_t)rb * (lp.dense_max_nhat + 256) > (size_t)sys->ctx->max_smem) {
    set_last_error("preconditioner apply: dense front too large for the upward kernel");
    return HM_ERR_CAPACITY;
  }
  switch (rb) {
    case 1: dense_up_rb<T, 1>(lp, base, sys, sp, nrhs, win, s); break;
    case 2: dense_up_rb<T, 2>(lp, base, sys, sp, nrhs, win, s); break;
    case 4: dense_up_rb<T, 4>(lp, base, sys, sp, nrhs, win, s); break;
    case 8: dense_up_rb<T, 8>(lp, base, sys, sp, nrhs, win, s); break;
    default: dense_up_rb<T, 16>(lp, base, sys, sp, nrhs, win, s); break;
  }
  return HM_OK;
}

template <typename T>
static void dense_down(const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys, SolvePlan* sp,
                       int nrhs, T* xv, cudaStream_t s) {
  switch (dense_rhs_block(sys->ctx, TS_DENSE_DOWN, lp, nrhs)) {
    case 1: dense_down_rb<T, 1>(lp, base, sys, sp, nrhs, xv, s); break;
    case 2: dense_down_rb<T, 2>(lp, base, sys, sp, nrhs, xv, s); break;
    case 4: dense_down_rb<T, 4>(lp, base, sys, sp, nrhs, xv, s); break;
    case 8: dense_down_rb<T, 8>(lp, base, sys, sp, nrhs, xv, s); break;
    default: dense_down_rb<T, 16>(lp, base, sys, sp, nrhs, xv, s); break;
  }
}

template <typename T>
static void gemm_b(hm_ctx_s* ctx, const SolvePlan* sp, const GemmBatch& b) {
  if (b.tiles.count == 0) return;
  ProfScope ps(ctx, PC_GEMM_APPLY, b.tasks.work);
  TuneScope ts(ctx, TS_GEMM, b.sig);
  const int v = ctx->tune.variant(TS_GEMM, b.sig);
  if (v == 3 && b.tiles_big.count > 0 && sizeof(T) == 4) {  // FP32 large-tile kernel
    launch_gemm_big(b.tasks.dev(sp->d_tasks), b.tiles_big.dev(sp->d_tasks), b.tiles_big.count,
                    (float*)sp->d_split_ws, sp->d_split_cnt, ctx->stream);
    return;
  }
  launch_gemm<T>(b.tasks.dev(sp->d_tasks), b.tiles.dev(sp->d_tasks), b.tiles.count, b.bn,
                 v >= 3 ? 0 : v, (T*)sp->d_split_ws,
                 sp->d_split_cnt, ctx->stream);
}

static dim3 vgrid(int nitems, int nrhs, int maxlen) {
  return dim3((unsigned)((nitems + 7) / 8), (unsigned)nrhs,
              (unsigned)std::max(1, (maxlen + kVecChunk - 1) / kVecChunk));
}

// A level's HODLR fronts take the fused cluster kernels where they fit: variant 0 with
// a quarter of the plan's widest right-hand-side group per cluster, 2 and 3 with an
// eighth and a sixteenth (more clusters in flight, each reading the factor again, mostly
// from L2), 4 as 0 with 512 threads per CTA instead of 256 (twice the loads in flight
// on the few clusters of the top levels; groups of up to four right-hand sides);
// variant 1 is the batched-GEMM path.
static bool fused_level(const hm_ctx_s* ctx, const LevelSolvePlan& lp) {
  return lp.ha_ok && ctx->tune.variant(TS_HODLR_APPLY, lp.ha_sig) != 1;
}
static int fused_rb(const hm_ctx_s* ctx, const LevelSolvePlan& lp) {
  const int v = ctx->tune.variant(TS_HODLR_APPLY, lp.ha_sig);
  return std::max(1, lp.ha_RB >> (v == 2 ? 3 : v == 3 ? 4 : 2));
}
static int fused_nt(const hm_ctx_s* ctx, const LevelSolvePlan& lp) {
  return ctx->tune.variant(TS_HODLR_APPLY, lp.ha_sig) == 4 ? 512 : 256;
}

// The launches of one apply (input win, output in the plan's fixed buffer).
template <typename T>
static int apply_launches(hm_sys_s* sys, SolvePlan* sp, int nrhs, const T* win) {
  Plan& P = sys->plan;
  hm_ctx_s* ctx = sys->ctx;
  cudaStream_t s = ctx->stream;
  const unsigned char* base = sp->d_tasks;
  T* FV = (T*)sp->d_fv;
  T* xfix = (T*)sp->d_xfix;  // the task tables write the solution here
  const int n = sys->n;
  for (int l = P.nlevels - 1; l >= 0; --l) {
    const LevelSolvePlan& lp = sp->levels[l];
    if (lp.dense.count) {
      ProfScope ps(ctx, PC_UP, lp.up_work);
      TuneScope ts(ctx, TS_DENSE_UP, dense_sig(lp, nrhs));
      HM_TRY(dense_up<T>(lp, base, sys, sp, nrhs, win, s));
    }
    if (lp.n_hodlr && fused_level(ctx, lp)) {
      ProfScope ps(ctx, PC_HODLR_UP, lp.ha_up_work);
      TuneScope ts(ctx, TS_HODLR_APPLY, lp.ha_sig);
      HM_TRY(launch_hodlr_apply<T>(false, lp, base, sys, sp, nrhs, win, nullptr, fused_rb(ctx, lp),
                                    fused_nt(ctx, lp)));
    } else if (lp.n_hodlr) {
      TuneScope ts(ctx, TS_HODLR_APPLY, lp.ha_sig);
      {
        ProfScope ps(ctx, PC_VECTOR, lp.hup_work);
        k_vassemble<T><<<dim3((unsigned)lp.n_hodlr, (unsigned)nrhs), 256, 0, s>>>(
            lp.hfronts.dev(base), n, win, sys->d_first, P.d_np, P.d_nhat, sp->d_fvoff, sys->d_child_ptr,
            sys->d_child_list, sys->d_ifoff, sys->d_relmap, FV);
      }
      gemm_b<T>(ctx, sp, lp.up_gemm);  // tf = Vtilde^T b_p
      gemm_b<T>(ctx, sp, lp.up2);      // f -= W tf
    }
  }
  for (int l = 0; l < P.nlevels; ++l) {
    const LevelSolvePlan& lp = sp->levels[l];
    if (lp.dense.count) {
      ProfScope ps(ctx, PC_DOWN, lp.down_work);
      TuneScope ts(ctx, TS_DENSE_DOWN, dense_sig(lp, nrhs));
      dense_down<T>(lp, base, sys, sp, nrhs, xfix, s);
    }
    if (lp.n_hodlr && fused_level(ctx, lp)) {
      ProfScope ps(ctx, PC_HODLR_DOWN, lp.ha_down_work);
      TuneScope ts(ctx, TS_HODLR_APPLY, lp.ha_sig);  // one key for both passes: one choice
      HM_TRY(launch_hodlr_apply<T>(true, lp, base, sys, sp, nrhs, nullptr, xfix, fused_rb(ctx, lp),
                                    fused_nt(ctx, lp)));
    } else if (lp.n_hodlr) {
      TuneScope ts(ctx, TS_HODLR_APPLY, lp.ha_sig);  // one key for both passes: one choice
      if (lp.hodlr_max_nu > 0) {
        ProfScope ps(ctx, PC_VECTOR, lp.hdown_work);
        k_vgather<T><<<vgrid(lp.n_hodlr, nrhs, lp.hodlr_max_nu), 256, 0, s>>>(
            lp.hfronts.dev(base), lp.n_hodlr, n, xfix, P.d_np, P.d_nhat, sp->d_fvoff, sys->d_ifoff,
            sys->d_iflist, FV);
      }
      gemm_b<T>(ctx, sp, lp.down_gemm);  // y = K_leaf^{-1} b on the HODLR leaves
      for (const auto& H : lp.heights) {
        gemm_b<T>(ctx, sp, H.t);
        gemm_b<T>(ctx, sp, H.upd);
      }
      gemm_b<T>(ctx, sp, lp.down1);
      gemm_b<T>(ctx, sp, lp.down2);  // x_p = y - Vtilde (W^T x_f), in place in xfix
    }
  }
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

// z = M^{-1} r.  An apply whose input buffer repeats (GMRES applies the preconditioner to
// the same staging buffer every iteration) is captured once into a CUDA graph and
// replayed: its ~10^2 dependent launches then cost one graph launch.  The first apply
// with a new input runs eagerly; with the launch profiler on, applies always run eagerly.
// dst (row-major n x nrhs: element (i, r) at i nrhs + r) = src (column-major, ld n),
// 64 rows and every right-hand side (<= 64) per tile through shared memory, so both
// sides are coalesced.
constexpr int kRmRows = 64;
template <typename T>
__global__ void __launch_bounds__(256) k_to_rowmajor(const T* __restrict__ src, T* __restrict__ dst, int n,
                                                     int nrhs) {
  __shared__ T tile[kRmRows][65];
  const int i0 = blockIdx.x * kRmRows, rows = min(kRmRows, n - i0), cnt = rows * nrhs;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int r = e / rows, ii = e - r * rows;
    tile[ii][r] = src[i0 + ii + (int64_t)r * n];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int ii = e / nrhs, r = e - ii * nrhs;
    dst[(int64_t)(i0 + ii) * nrhs + r] = tile[ii][r];
  }
}

template <typename T>
static int apply_t(hm_sys_s* sys, int nrhs, const T* win, T* xout, bool rowmajor_out = false,
                   bool eager = false) {
  SolvePlan* sp = nullptr;
  HM_TRY(get_solve_plan(sys, nrhs, &sp));
  hm_ctx_s* ctx = sys->ctx;
  cudaStream_t s = ctx->stream;
  const bool graphs = !eager && !ctx->prof.on && !ctx->tune.rec && s != nullptr;
  if (graphs && sp->graph_exec && sp->graph_in == (const void*)win) {
    HM_CUDA(cudaGraphLaunch(sp->graph_exec, s));
  } else if (graphs && sp->last_in == (const void*)win) {
    cudaGraph_t g = nullptr;
    HM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int st = apply_launches<T>(sys, sp, nrhs, win);
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (st != HM_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (st != HM_OK) return st;
      HM_CUDA(ce);
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    HM_CUDA(ie);
    if (sp->graph_exec) cudaGraphExecDestroy(sp->graph_exec);
    sp->graph_exec = ex;
    sp->graph_in = win;
    HM_CUDA(cudaGraphLaunch(sp->graph_exec, s));
  } else {
    HM_TRY(apply_launches<T>(sys, sp, nrhs, win));
  }
  if (!eager) sp->last_in = win;
  T* xfix = (T*)sp->d_xfix;
  if (rowmajor_out) {
    ProfScope ps(ctx, PC_VECTOR, Work{0.0, 2.0 * sizeof(T) * (double)sys->n * nrhs});
    k_to_rowmajor<T><<<(sys->n + kRmRows - 1) / kRmRows, 256, 0, s>>>(xfix, xout, sys->n, nrhs);
  } else if (xout != xfix) {
    HM_CUDA(cudaMemcpyAsync(xout, xfix, sizeof(T) * (size_t)sys->n * nrhs, cudaMemcpyDeviceToDevice, s));
  }
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

template <typename T, int RB, int NT>
static int dense_setup_one(int max_smem) {
  HM_CUDA(allow_max_dyn_smem(k_dense_up<T, RB, NT>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_dense_down<T, RB, NT>, max_smem));
  return HM_OK;
}

template <typename T>
static int dense_setup(int max_smem) {
  HM_TRY((dense_setup_one<T, 1, 64>(max_smem)));
  HM_TRY((dense_setup_one<T, 2, 64>(max_smem)));
  HM_TRY((dense_setup_one<T, 4, 64>(max_smem)));
  HM_TRY((dense_setup_one<T, 8, 64>(max_smem)));
  HM_TRY((dense_setup_one<T, 16, 64>(max_smem)));
  HM_TRY((dense_setup_one<T, 1, 256>(max_smem)));
  HM_TRY((dense_setup_one<T, 2, 256>(max_smem)));
  HM_TRY((dense_setup_one<T, 4, 256>(max_smem)));
  HM_TRY((dense_setup_one<T, 8, 256>(max_smem)));
  HM_TRY((dense_setup_one<T, 16, 256>(max_smem)));
  return HM_OK;
}

int solve_setup(int max_smem) {
  HM_TRY(dense_setup<float>(max_smem));
  HM_TRY(dense_setup<double>(max_smem));
  return HM_OK;
}

int apply_impl(hm_sys_s* sys, int nrhs, const void* rT, void* zT) {
  if (sys->precision == HM_PREC_FP64) return apply_t<double>(sys, nrhs, (const double*)rT, (double*)zT);
  return apply_t<float>(sys, nrhs, (const float*)rT, (float*)zT);
}

int apply_impl_eager(hm_sys_s* sys, int nrhs, const void* rT, void* zT) {
  if (sys->precision == HM_PREC_FP64)
    return apply_t<double>(sys, nrhs, (const double*)rT, (double*)zT, false, true);
  return apply_t<float>(sys, nrhs, (const float*)rT, (float*)zT, false, true);
}

int apply_impl_rowmajor(hm_sys_s* sys, int nrhs, const void* rT, void* zT) {
  if (sys->precision == HM_PREC_FP64) return apply_t<double>(sys, nrhs, (const double*)rT, (double*)zT, true);
  return apply_t<float>(sys, nrhs, (const float*)rT, (float*)zT, true);
}

// ------------------------------------------------------------------------------------
// Permutations and casts.
// ------------------------------------------------------------------------------------
__global__ void k_permute_in(const double* src, double* dst, const int32_t* perm, int n, int nrhs) {
  const int64_t total = (int64_t)n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n);
    const int64_t r = e / n;
    dst[e] = src[perm[i] + r * n];
  }
}

__global__ void k_permute_out(const double* src, double* dst, const int32_t* perm, int n, int nrhs) {
  const int64_t total = (int64_t)n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n);
    const int64_t r = e / n;
    dst[perm[i] + r * n] = src[e];
  }
}

// Grid of the grid-stride vector kernels: eight CTAs per SM of the current device.
static unsigned stride_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 8u * (unsigned)std::max(sms, 1);
}

void launch_permute_in(const double* src, double* dst, const int32_t* perm, int n, int nrhs,
                       cudaStream_t s) {
  k_permute_in<<<stride_grid(), 256, 0, s>>>(src, dst, perm, n, nrhs);
}
void launch_permute_out(const double* src, double* dst, const int32_t* perm, int n, int nrhs,
                        cudaStream_t s) {
  k_permute_out<<<stride_grid(), 256, 0, s>>>(src, dst, perm, n, nrhs);
}

template <typename T>
__global__ void k_cast_to(const double* src, T* dst, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (T)src[e];
}
template <typename T>
__global__ void k_cast_from(const T* src, double* dst, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}
template <typename T>
void launch_cast_to(const double* src, T* dst, int64_t count, cudaStream_t s) {
  k_cast_to<T><<<stride_grid(), 256, 0, s>>>(src, dst, count);
}
template <typename T>
void launch_cast_from(const T* src, double* dst, int64_t count, cudaStream_t s) {
  k_cast_from<T><<<stride_grid(), 256, 0, s>>>(src, dst, count);
}
template void launch_cast_to<float>(const double*, float*, int64_t, cudaStream_t);
template void launch_cast_to<double>(const double*, double*, int64_t, cudaStream_t);
template void launch_cast_from<float>(const float*, double*, int64_t, cudaStream_t);
template void launch_cast_from<double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace hm
