// hm_solve.cu -- preconditioner apply z = M^{-1} r: the multifrontal upward pass
// (Eq. upward: b_f <- b_f - F_fp F_pp^-1 b_p, leaves to root) and downward pass
// (Eq. downward: x_p = F_pp^-1 (b_p - F_pf x_f), root to leaves), with the HODLR pivot
// solves and low-rank coupling blocks of Section 4.2.2 for HODLR fronts.
//
// Every front p owns a vector fv_p of length nhat_p = |I_p| + |I_p^f| (per RHS).
// Upward: fv_p = [r(I_p); 0] (+) the children's update parts (extend-add of vectors in
// fixed child order), then b_f <- b_f - F_fp F_pp^{-1} b_p: dense fronts keep
// K = F_fp F_pp^{-1} from the factorization (a GEMV), HODLR fronts use
// Vf^T F_pp^{-1} = Vtilde^T (F_pp^HODLR symmetric) so b_f -= W (Vtilde^T b_p) needs no
// pivot solve.  Downward: x_f is gathered from the finished ancestors; dense fronts
// x_p = F_pp^{-1} b_p - K^T x_f (F_pp^{-1} stored explicitly); HODLR fronts solve
// y = F_pp^{-1} b_p by recursive Woodbury (explicit leaf inverses, then per level
// y -= Zhat C^{-1} Z^T y with explicit core inverses) and x_p = y - Vtilde (W^T x_f).
// Every step is a GEMV / batched GEMM; nothing is solved by sequential substitution.
#include "hm_internal.h"

namespace hm {

template <typename T>
__global__ void __launch_bounds__(256) k_up(const int* __restrict__ fronts, int nrhs, int n,
                                            const T* __restrict__ win, const int32_t* __restrict__ first,
                                            const int* __restrict__ npiv, const int* __restrict__ nhat,
                                            const int* __restrict__ hkind, const int64_t* __restrict__ front_off,
                                            const int64_t* __restrict__ fvoff,
                                            const int32_t* __restrict__ child_ptr,
                                            const int32_t* __restrict__ child_list,
                                            const int64_t* __restrict__ ifoff,
                                            const int32_t* __restrict__ relmap, const T* __restrict__ F,
                                            T* __restrict__ FV) {
  const int q = fronts[blockIdx.x];
  const int np = npiv[q], nh = nhat[q], nu = nh - np, b0 = first[q];
  T* fv = FV + fvoff[q];
  for (int e = threadIdx.x; e < np * nrhs; e += blockDim.x) {
    const int i = e % np, r = e / np;
    fv[i + (int64_t)r * nh] = win[b0 + i + (int64_t)r * n];
  }
  for (int e = threadIdx.x; e < nu * nrhs; e += blockDim.x) {
    const int t = e % nu, r = e / nu;
    fv[np + t + (int64_t)r * nh] = T(0);
  }
  __syncthreads();
  for (int ci = child_ptr[q]; ci < child_ptr[q + 1]; ++ci) {
    const int c = child_list[ci];
    const int npc = npiv[c], nhc = nhat[c], nuc = nhc - npc;
    const T* fvc = FV + fvoff[c];
    const int32_t* rm = relmap + ifoff[c];
    for (int e = threadIdx.x; e < nuc * nrhs; e += blockDim.x) {
      const int t = e % nuc, r = e / nuc;
      fv[rm[t] + (int64_t)r * nh] += fvc[npc + t + (int64_t)r * nhc];
    }
    __syncthreads();
  }
  if (hkind[q] >= 0 || nu == 0) return;
  const T* K = F + front_off[q] + np;  // K(t, j) = K[t + j * nh]
  for (int e = threadIdx.x; e < nu * nrhs; e += blockDim.x) {
    const int t = e % nu, r = e / nu;
    const T* bp = fv + (int64_t)r * nh;
    T s = T(0);
    for (int j = 0; j < np; ++j) s += K[t + (int64_t)j * nh] * bp[j];
    fv[np + t + (int64_t)r * nh] -= s;
  }
}

// Downward pass of one front per CTA.  x_f is gathered from the finished ancestors into
// the update part of fv.  Dense fronts: x_p = G^T [b_p; -x_f] with G = [F_pp^{-1}; K]
// the front's first np columns (nhat x np, column-major, F_pp^{-1} symmetric), computed
// as a small GEMM: 32-row slabs of G and of the vector block are staged in shared memory
// (coalesced), each thread accumulates up to kDownAcc outputs (j, r) in registers.
constexpr int kDownKC = 32;
constexpr int kDownAcc = 32;  // np * nrhs <= 256 * kDownAcc (np <= 128, nrhs <= 64)

template <typename T>
__global__ void __launch_bounds__(256) k_down(const int* __restrict__ fronts, int nrhs, int n,
                                              T* __restrict__ xout, const int32_t* __restrict__ first,
                                              const int* __restrict__ npiv, const int* __restrict__ nhat,
                                              const int* __restrict__ hkind,
                                              const int64_t* __restrict__ front_off,
                                              const int64_t* __restrict__ fvoff,
                                              const int64_t* __restrict__ ifoff,
                                              const int32_t* __restrict__ iflist, const T* __restrict__ F,
                                              T* __restrict__ FV) {
  extern __shared__ unsigned char smem_raw[];
  const int q = fronts[blockIdx.x];
  const int np = npiv[q], nh = nhat[q], nu = nh - np, b0 = first[q];
  T* fv = FV + fvoff[q];
  const int32_t* If = iflist + ifoff[q];
  for (int e = threadIdx.x; e < nu * nrhs; e += blockDim.x) {
    const int t = e % nu, r = e / nu;
    fv[np + t + (int64_t)r * nh] = xout[If[t] + (int64_t)r * n];
  }
  __syncthreads();
  if (hkind[q] >= 0) return;
  const T* G = F + front_off[q];
  T* Gs = reinterpret_cast<T*>(smem_raw);   // [kDownKC][np + 1]
  T* Vs = Gs + kDownKC * (np + 1);          // [kDownKC][nrhs]
  const int nout = np * nrhs;
  T acc[kDownAcc];
#pragma unroll
  for (int a = 0; a < kDownAcc; ++a) acc[a] = T(0);
  for (int k0 = 0; k0 < nh; k0 += kDownKC) {
    const int kc = min(kDownKC, nh - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kc * np; e += blockDim.x) {
      const int kk = e % kc, j = e / kc;
      Gs[kk * (np + 1) + j] = G[(k0 + kk) + (int64_t)j * nh];
    }
    for (int e = threadIdx.x; e < kc * nrhs; e += blockDim.x) {
      const int kk = e % kc, r = e / kc;
      const T v = fv[(k0 + kk) + (int64_t)r * nh];
      Vs[kk * nrhs + r] = (k0 + kk < np) ? v : -v;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < kDownAcc; ++a) {
      const int e = threadIdx.x + a * 256;
      if (e < nout) {
        const int j = e % np, r = e / np;
        T s = acc[a];
        for (int kk = 0; kk < kc; ++kk) s += Gs[kk * (np + 1) + j] * Vs[kk * nrhs + r];
        acc[a] = s;
      }
    }
  }
#pragma unroll
  for (int a = 0; a < kDownAcc; ++a) {
    const int e = threadIdx.x + a * 256;
    if (e < nout) {
      const int j = e % np, r = e / np;
      xout[b0 + j + (int64_t)r * n] = acc[a];
    }
  }
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
  launch_gemm<T>(b.tasks.dev(base), b.tiles.dev(base), b.tiles.count, ctx->stream);
}

template <typename T>
static int apply_t(hm_sys_s* sys, int nrhs, const T* win, T* xout) {
  SolvePlan* sp = nullptr;
  HM_TRY(get_solve_plan(sys, nrhs, &sp));
  Plan& P = sys->plan;
  hm_ctx_s* ctx = sys->ctx;
  cudaStream_t s = ctx->stream;
  const unsigned char* base = sp->d_tasks;
  const T* F = (const T*)sys->d_front;
  T* FV = (T*)sp->d_fv;
  const int n = sys->n;
  for (int l = P.nlevels - 1; l >= 0; --l) {
    const LevelSolvePlan& lp = sp->levels[l];
    {
      ProfScope ps(ctx, PC_UP, lp.up_work);
      k_up<T><<<lp.nfronts, 256, 0, s>>>(lp.fronts.dev(base), nrhs, n, win, sys->d_first, P.d_np,
                                         P.d_nhat, P.d_hkind, P.d_front_off, sp->d_fvoff,
                                         sys->d_child_ptr, sys->d_child_list, sys->d_ifoff,
                                         sys->d_relmap, F, FV);
    }
    gemm_b<T>(ctx, lp.up1, base);
    gemm_b<T>(ctx, lp.up2, base);
  }
  for (int l = 0; l < P.nlevels; ++l) {
    const LevelSolvePlan& lp = sp->levels[l];
    {
      ProfScope ps(ctx, PC_DOWN, lp.down_work);
      const size_t smem = (size_t)kDownKC * (129 + nrhs) * sizeof(T);
      k_down<T><<<lp.nfronts, 256, smem, s>>>(lp.fronts.dev(base), nrhs, n, xout, sys->d_first, P.d_np,
                                           P.d_nhat, P.d_hkind, P.d_front_off, sp->d_fvoff,
                                           sys->d_ifoff, sys->d_iflist, F, FV);
    }
    if (lp.n_hodlr) {
      gemm_b<T>(ctx, lp.leaf, base);
      for (const auto& H : lp.heights) {
        gemm_b<T>(ctx, H.t, base);
        gemm_b<T>(ctx, H.s, base);
        gemm_b<T>(ctx, H.upd, base);
      }
      gemm_b<T>(ctx, lp.down1, base);
      gemm_b<T>(ctx, lp.down2, base);
      ProfScope ps(ctx, PC_VECTOR, Work{});
      k_hodlr_out<T><<<lp.nfronts, 256, 0, s>>>(lp.fronts.dev(base), nrhs, n, xout, sys->d_first,
                                                P.d_np, sp->d_yvoff, (const T*)sp->d_sb);
    }
  }
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

int solve_setup(int max_smem) {
  HM_CUDA(allow_max_dyn_smem(k_down<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_down<double>, max_smem));
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
