// hm_solve.cu -- preconditioner apply z = M^{-1} r: the multifrontal upward pass
// (Eq. upward: b_f <- b_f - F_fp F_pp^-1 b_p, leaves to root) and downward pass
// (Eq. downward: x_p = F_pp^-1 (b_p - F_pf x_f), root to leaves), with the HODLR pivot
// solves and low-rank coupling blocks of Section 4.2.2 for HODLR fronts.
//
// Every front p owns a vector block fv_p (nhat_p x nrhs, nhat_p = |I_p| + |I_p^f|).
// Upward, per tree level: fv_p = [r(I_p); 0] (flat kernel), then the children's update
// parts are added through the relative maps one child slot at a time (fixed order), then
// b_f <- b_f - F_fp F_pp^{-1} b_p as batched GEMMs: dense fronts keep K = F_fp F_pp^{-1}
// from the factorization; HODLR fronts use Vf^T F_pp^{-1} = Vtilde^T (F_pp^HODLR is
// symmetric), so b_f -= W (Vtilde^T b_p) needs no pivot solve.  Downward: fv_p's update
// part receives -x(I_p^f) from the finished ancestors; a dense front's solution is the
// single GEMM x_p = [F_pp^{-1}; K]^T fv_p = F_pp^{-1} b_p - K^T x_f; a HODLR front solves
// y = F_pp^{-1} b_p by recursive Woodbury (explicit leaf inverses, then per level
// y -= Zhat C^{-1} Z^T y with explicit core inverses) and x_p = y - Vtilde (W^T x_f).
// Every step is a flat vector kernel or a batched GEMM; nothing is solved by sequential
// substitution.
#include <algorithm>

#include "hm_internal.h"

namespace hm {

// Flat vector kernels of the apply: one warp per (front, right-hand side, chunk of 256
// rows); grid = (ceil(fronts / 8), nrhs, chunks), 8 warps per block.
constexpr int kVecChunk = 256;

// fv_q = [r(I_q); 0] for every front q of the level.
template <typename T>
__global__ void __launch_bounds__(256) k_vinit(const int* __restrict__ fronts, int nfronts, int n,
                                               const T* __restrict__ win, const int32_t* __restrict__ first,
                                               const int* __restrict__ npiv, const int* __restrict__ nhat,
                                               const int64_t* __restrict__ fvoff, T* __restrict__ FV) {
  const int fi = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (fi >= nfronts) return;
  const int q = fronts[fi], r = blockIdx.y;
  const int np = npiv[q], nh = nhat[q], b0 = first[q];
  T* fv = FV + fvoff[q] + (int64_t)r * nh;
  const T* w = win + b0 + (int64_t)r * n;
  const int e0 = blockIdx.z * kVecChunk, e1 = min(nh, e0 + kVecChunk);
  for (int e = e0 + lane; e < e1; e += 32) fv[e] = e < np ? w[e] : T(0);
}

// Extend-add of vectors for child slot `slot`: fv_parent[relmap] += update part of the
// child (slots run one after another, so sums are formed in a fixed order).
template <typename T>
__global__ void __launch_bounds__(256) k_vadd(const int* __restrict__ parents, int nparents, int slot,
                                              const int32_t* __restrict__ child_ptr,
                                              const int32_t* __restrict__ child_list,
                                              const int* __restrict__ npiv, const int* __restrict__ nhat,
                                              const int64_t* __restrict__ fvoff,
                                              const int64_t* __restrict__ ifoff,
                                              const int32_t* __restrict__ relmap, T* __restrict__ FV) {
  const int fi = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (fi >= nparents) return;
  const int q = parents[fi], r = blockIdx.y;
  const int c = child_list[child_ptr[q] + slot];
  const int npc = npiv[c], nhc = nhat[c], nuc = nhc - npc;
  const int e0 = blockIdx.z * kVecChunk, e1 = min(nuc, e0 + kVecChunk);
  if (e0 >= e1) return;
  T* fv = FV + fvoff[q] + (int64_t)r * nhat[q];
  const T* fc = FV + fvoff[c] + npc + (int64_t)r * nhc;
  const int32_t* rm = relmap + ifoff[c];
  for (int t = e0 + lane; t < e1; t += 32) fv[rm[t]] += fc[t];
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
  for (int t = e0 + lane; t < e1; t += 32) fv[t] = -x[If[t]];
}

// HODLR fronts: x_p (= y - Vtilde W^T x_f, in the front's y buffer) -> output vector.
template <typename T>
__global__ void k_hodlr_out(const int* __restrict__ fronts, int nrhs, int n, T* __restrict__ xout,
                            const int32_t* __restrict__ first, const int* __restrict__ npiv,
                            const int64_t* __restrict__ yvoff, const T* __restrict__ SB) {
  const int q = fronts[blockIdx.x];
  const int64_t yo = yvoff[q];
  if (yo < 0) return;
  const int np = npiv[q], b0 = first[q];
  const T* y = SB + yo;
  for (int e = threadIdx.x; e < np * nrhs; e += blockDim.x) {
    const int i = e % np, r = e / np;
    xout[b0 + i + (int64_t)r * n] = y[i + (int64_t)r * np];
  }
}

template <typename T>
static void gemm_b(hm_ctx_s* ctx, const GemmBatch& b, const unsigned char* base) {
  if (b.tiles.count == 0) return;
  ProfScope ps(ctx, PC_GEMM_APPLY, b.tasks.work);
  launch_gemm<T>(b.tasks.dev(base), b.tiles.dev(base), b.tiles.count, b.bn, ctx->stream);
}

static dim3 vgrid(int nitems, int nrhs, int maxlen) {
  return dim3((unsigned)((nitems + 7) / 8), (unsigned)nrhs,
              (unsigned)std::max(1, (maxlen + kVecChunk - 1) / kVecChunk));
}

template <typename T>
static int apply_t(hm_sys_s* sys, int nrhs, const T* win, T* xout) {
  SolvePlan* sp = nullptr;
  HM_TRY(get_solve_plan(sys, nrhs, &sp));
  Plan& P = sys->plan;
  hm_ctx_s* ctx = sys->ctx;
  cudaStream_t s = ctx->stream;
  const unsigned char* base = sp->d_tasks;
  T* FV = (T*)sp->d_fv;
  T* xfix = (T*)sp->d_xfix;  // the task tables write the solution here
  const int n = sys->n;
  for (int l = P.nlevels - 1; l >= 0; --l) {
    const LevelSolvePlan& lp = sp->levels[l];
    {
      ProfScope ps(ctx, PC_UP, lp.up_work, 1 + (int)lp.slots.size());
      k_vinit<T><<<vgrid(lp.nfronts, nrhs, lp.max_nhat), 256, 0, s>>>(
          lp.fronts.dev(base), lp.nfronts, n, win, sys->d_first, P.d_np, P.d_nhat, sp->d_fvoff, FV);
      for (size_t sl = 0; sl < lp.slots.size(); ++sl) {
        const Span<int>& par = lp.slots[sl];
        if (par.count == 0) continue;
        k_vadd<T><<<vgrid(par.count, nrhs, lp.slot_max_nu[sl]), 256, 0, s>>>(
            par.dev(base), par.count, (int)sl, sys->d_child_ptr, sys->d_child_list, P.d_np, P.d_nhat,
            sp->d_fvoff, sys->d_ifoff, sys->d_relmap, FV);
      }
    }
    gemm_b<T>(ctx, lp.up_gemm, base);  // dense: f -= K b_p; HODLR: tf = Vtilde^T b_p
    gemm_b<T>(ctx, lp.up2, base);      // HODLR: f -= W tf
  }
  for (int l = 0; l < P.nlevels; ++l) {
    const LevelSolvePlan& lp = sp->levels[l];
    if (lp.max_nu > 0) {
      ProfScope ps(ctx, PC_DOWN, lp.down_work);
      k_vgather<T><<<vgrid(lp.nfronts, nrhs, lp.max_nu), 256, 0, s>>>(
          lp.fronts.dev(base), lp.nfronts, n, xfix, P.d_np, P.d_nhat, sp->d_fvoff, sys->d_ifoff,
          sys->d_iflist, FV);
    }
    gemm_b<T>(ctx, lp.down_gemm, base);  // dense: x_p = G^T fv; HODLR leaves: y = K_leaf^{-1} b
    if (lp.n_hodlr) {
      for (const auto& H : lp.heights) {
        gemm_b<T>(ctx, H.t, base);
        gemm_b<T>(ctx, H.s, base);
        gemm_b<T>(ctx, H.upd, base);
      }
      gemm_b<T>(ctx, lp.down1, base);
      gemm_b<T>(ctx, lp.down2, base);
      ProfScope ps(ctx, PC_VECTOR, Work{});
      k_hodlr_out<T><<<lp.nfronts, 256, 0, s>>>(lp.fronts.dev(base), nrhs, n, xfix, sys->d_first,
                                                P.d_np, sp->d_yvoff, (const T*)sp->d_sb);
    }
  }
  if (xout != xfix)
    HM_CUDA(cudaMemcpyAsync(xout, xfix, sizeof(T) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, s));
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

int solve_setup(int max_smem) {
  (void)max_smem;
  return HM_OK;
}

int apply_impl(hm_sys_s* sys, int nrhs, const void* rT, void* zT) {
  if (sys->precision == HM_PREC_FP64) return apply_t<double>(sys, nrhs, (const double*)rT, (double*)zT);
  return apply_t<float>(sys, nrhs, (const float*)rT, (float*)zT);
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

void launch_permute_in(const double* src, double* dst, const int32_t* perm, int n, int nrhs,
                       cudaStream_t s) {
  k_permute_in<<<1216, 256, 0, s>>>(src, dst, perm, n, nrhs);
}
void launch_permute_out(const double* src, double* dst, const int32_t* perm, int n, int nrhs,
                        cudaStream_t s) {
  k_permute_out<<<1216, 256, 0, s>>>(src, dst, perm, n, nrhs);
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
  k_cast_to<T><<<1216, 256, 0, s>>>(src, dst, count);
}
template <typename T>
void launch_cast_from(const T* src, double* dst, int64_t count, cudaStream_t s) {
  k_cast_from<T><<<1216, 256, 0, s>>>(src, dst, count);
}
template void launch_cast_to<float>(const double*, float*, int64_t, cudaStream_t);
template void launch_cast_to<double>(const double*, double*, int64_t, cudaStream_t);
template void launch_cast_from<float>(const float*, double*, int64_t, cudaStream_t);
template void launch_cast_from<double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace hm
