// hm_factor.cu -- numerical factorization (Sections 4.1.1 and 4.2.1 of the paper).
//
// Per elimination-tree level, deepest first:
//   F_p = F_bar_p (+) U_c1 (+) ...            assembly (Eq. fbar) and extend-add
//   dense fronts (|I_p| <= n_c):  F_pp = L L^T, L_fp = F_fp L^-T, U_p = F_ff - L_fp L_fp^T
//   HODLR fronts: compress every off-diagonal block of F_pp's HODLR tree and F_fp ~ W Vf^T
//   by the randomized range finder; factor F_pp^HODLR by recursive Woodbury on the column
//   block X = [Vf | B_0 | ... | B_{L-1}] (each level's ancestor columns form a prefix);
//   U_p = F_ff - W (Vf^T F_pp^-1 Vf) W^T  (Eq. update_HODLR_Parent).
#include <cstdio>
#include <cstdlib>

#include "hm_internal.h"

namespace hm {

// The permuted FP64 values of A for the GMRES residual, and the same split as FP32
// hi + lo (48 of the 53 bits) for the double-float SpMV.
__global__ void k_perm_values(const double* __restrict__ vals, const int64_t* __restrict__ psrc, int64_t nnz,
                              double* __restrict__ pvals, float2* __restrict__ pvals2) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double v = vals[psrc[k]];
    pvals[k] = v;
    const float hi = (float)v;
    pvals2[k] = make_float2(hi, (float)(v - (double)hi));
  }
}

// F-bar of one tree level (Eq. fbar): A's lower-triangle entries whose front is at
// depth l, at their positions in the front storage.
template <typename T>
__global__ void k_scatter_level(const double* __restrict__ vals, const int64_t* __restrict__ src,
                                const int64_t* __restrict__ dst, const int64_t* __restrict__ range, int l,
                                T* __restrict__ F) {
  const int64_t m1 = range[2 * l + 1];
  for (int64_t m = range[2 * l] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < m1;
       m += (int64_t)gridDim.x * blockDim.x)
    F[dst[m]] = (T)vals[src[m]];
}

// Packs the factor of a level out of the front storage (one task per block, a warp per
// column, lanes along the rows).
template <typename T>
__global__ void __launch_bounds__(256) k_copy2d(const CopyTask* __restrict__ tasks) {
  const CopyTask t = tasks[blockIdx.x];
  const T* src = (const T*)t.src;
  T* dst = (T*)t.dst;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < t.cols; c += 8) {
    const T* s = src + (int64_t)c * t.lds;
    T* d = dst + (int64_t)c * t.ldd;
    for (int r = lane; r < t.rows; r += 32) d[r] = s[r];
  }
}

// Extend-add of child slot `slot` of every listed parent q: warp w of block (x, y) adds
// column 8 y + w (lower part) of the child's update matrix U_c = F_ff of c into the front
// of q at rows/columns relmap.  Slots run one launch after another, so every entry of a
// parent receives its children's contributions in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_extend_add(const int* __restrict__ parents, int slot,
                                                    const int32_t* __restrict__ child_ptr,
                                                    const int32_t* __restrict__ child_list,
                                                    const int64_t* __restrict__ front_off,
                                                    const int* __restrict__ nhat, const int* __restrict__ npiv,
                                                    const int64_t* __restrict__ ifoff,
                                                    const int32_t* __restrict__ relmap, T* __restrict__ F) {
  const int q = parents[blockIdx.x];
  const int c = child_list[child_ptr[q] + slot];
  const int col = blockIdx.y * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int ldc = nhat[c], npc = npiv[c], nuc = ldc - npc;
  if (col >= nuc) return;
  const int ldp = nhat[q];
  const T* Fc = F + front_off[c] + npc + (int64_t)(npc + col) * ldc;
  T* Fp = F + front_off[q];
  const int32_t* rm = relmap + ifoff[c];
  const int64_t cc = (int64_t)rm[col] * ldp;
  // four rows per lane at a time: their map entries, then the values and destinations
  for (int r0 = col + lane; r0 < nuc; r0 += 128) {
    int d[4];
    T v[4], o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = min(r0 + 32 * u, nuc - 1);
      d[u] = rm[r];
      v[u] = Fc[r];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) o[u] = Fp[d[u] + cc];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (r0 + 32 * u < nuc) Fp[d[u] + cc] = o[u] + v[u];
  }
}

template <typename T>
static void run_qr(hm_sys_s* sys, const QrBatch& b, const unsigned char* base) {
  if (b.plain.count == 0 && b.ts.count == 0 && b.stack.count == 0) return;
  cudaStream_t s = sys->ctx->stream;
  ProfScope ps(sys->ctx, PC_QR, b.work, (b.plain.count ? 1 : 0) + (b.ts.count ? 3 : 0) + (b.stack.count ? 2 : 0));
  TuneScope ts(sys->ctx, TS_QR, b.sig);
  // variant 1: keep the panels in global memory even where they fit in shared memory
  // (not with row blocks, whose outputs only the shared-memory kernel redirects)
  const bool global = sys->ctx->tune.variant(TS_QR, b.sig) == 1 && b.stack.count == 0;
  const int64_t maxmk = global ? INT64_MAX / 16 : b.plain_maxmk;
  launch_qr<T>(b.plain.dev(base), b.plain.count, b.plain_maxm, maxmk, sys->ctx->max_smem, s);
  launch_tsqr<T>(b.ts.dev(base), b.ts.count, b.blocks.dev(base), b.blocks.count, b.smem_block, b.smem_stack,
                 (T*)sys->d_qrs, s);
  if (b.stack.count) {  // row-blocked panels: the stacked R factors, then Y_b = Q_b Q_stack,b
    launch_qr<T>(b.stack.dev(base), b.stack.count, b.stack_maxm, b.stack_maxmk, sys->ctx->max_smem, s);
    launch_gemm<T>(b.combine.tasks.dev(base), b.combine.tiles.dev(base), b.combine.tiles.count, b.combine.bn, 0,
                   (T*)sys->plan.d_split_ws, sys->plan.d_split_cnt, s);
  }
}

// Debug facility (environment HM_DEBUG_SYNC=1): after each stage of the factorization,
// synchronize, report the device error word and count non-finite entries of the arenas.
template <typename T>
__global__ void k_count_nonfinite(const T* __restrict__ p, int64_t n, unsigned long long* out) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += isfinite((double)p[i]) ? 0ull : 1ull;
  if (c) atomicAdd(out, c);
}

template <typename T>
static void debug_stage(hm_sys_s* sys, const char* stage, int level) {
  static const bool on = getenv("HM_DEBUG_SYNC") && getenv("HM_DEBUG_SYNC")[0] == '1';
  if (!on) return;
  cudaStream_t s = sys->ctx->stream;
  const Plan& P = sys->plan;
  const cudaError_t le = cudaPeekAtLastError();  // a launch of this stage refused
  unsigned long long* d = nullptr;
  cudaMalloc(&d, 6 * sizeof(unsigned long long));
  cudaMemsetAsync(d, 0, 6 * sizeof(unsigned long long), s);
  const void* bufs[6] = {sys->d_front, sys->d_comp, sys->d_bo, sys->d_x, sys->d_core, sys->d_tb};
  const int64_t lens[6] = {P.front_total, P.comp_total, P.bo_total, P.bo_total, P.core_total, P.tb_total};
  for (int i = 0; i < 6; ++i)
    if (lens[i] > 0) k_count_nonfinite<T><<<256, 256, 0, s>>>((const T*)bufs[i], lens[i], d + i);
  unsigned long long h[6];
  int e[4];
  cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(e, sys->d_err, sizeof(e), cudaMemcpyDeviceToHost, s);
  cudaError_t ce = cudaStreamSynchronize(s);
  cudaFree(d);
  fprintf(stderr, "[hm debug] level %d %-10s launch=%s cuda=%s err=%d(%d,%d) nonfinite front=%llu comp=%llu bo=%llu x=%llu core=%llu tb=%llu\n",
          level, stage, cudaGetErrorString(le), cudaGetErrorString(ce), e[0], e[1], e[2], h[0], h[1], h[2], h[3], h[4], h[5]);
}

template <typename T>
static void run_gemm(hm_sys_s* sys, const GemmBatch& b, const unsigned char* base, int cat) {
  if (b.tiles.count == 0) return;
  const int vt = sys->ctx->tune.variant(TS_GEMM, b.sig);
  const bool on_tc = sizeof(T) == 4 && (b.tc || (vt == 4 && b.tiles_tc.count > 0));
  ProfScope ps(sys->ctx, on_tc ? PC_GEMM_TC : cat, b.tasks.work);  // tensor-core launches apart
  if (b.tc && sizeof(T) == 4) {
    launch_gemm_tc(b.tasks.dev(base), b.tiles.dev(base), b.tiles.count, (float*)sys->plan.d_split_ws,
                   sys->plan.d_split_cnt, sys->d_err, sys->ctx->opts.wait_limit,
                   sys->ctx->opts.inject_wait_timeout, sys->ctx->stream);
    return;
  }
  TuneScope ts(sys->ctx, TS_GEMM, b.sig);
  const int v = sys->ctx->tune.variant(TS_GEMM, b.sig);
  if (v == 4 && b.tiles_tc.count > 0 && sizeof(T) == 4) {  // FP32 on the tensor cores (3xTF32)
    launch_gemm_tf32x3(b.tasks.dev(base), b.tiles_tc.dev(base), b.tiles_tc.count, (float*)sys->plan.d_split_ws,
                       sys->plan.d_split_cnt, sys->d_err, sys->ctx->opts.wait_limit, sys->ctx->stream);
    return;
  }
  if (v == 3 && b.tiles_big.count > 0 && sizeof(T) == 4) {  // FP32 large-tile kernel
    launch_gemm_big(b.tasks.dev(base), b.tiles_big.dev(base), b.tiles_big.count, (float*)sys->plan.d_split_ws,
                    sys->plan.d_split_cnt, sys->ctx->stream);
    return;
  }
  launch_gemm<T>(b.tasks.dev(base), b.tiles.dev(base), b.tiles.count, b.bn, v >= 3 ? 0 : v,
                 (T*)sys->plan.d_split_ws, sys->plan.d_split_cnt, sys->ctx->stream);
}

template <typename T>
static int factor_t(hm_sys_s* sys, const double* d_values, double tol) {
  Plan& P = sys->plan;
  hm_ctx_s* ctx = sys->ctx;
  cudaStream_t s = ctx->stream;
  const unsigned char* base = P.d_tasks;
  T* F = (T*)sys->d_front;
  const int es = sizeof(T);
  HM_CUDA(cudaMemsetAsync(sys->d_err, 0, 4 * sizeof(int), s));
  {
    ProfScope ps(ctx, PC_MEMSET, Work{0.0, (double)es * (P.bo_total + P.w_total)}, 0);
    if (P.bo_total) HM_CUDA(cudaMemsetAsync(sys->d_bo, 0, (size_t)P.bo_total * sizeof(T), s));
    if (P.w_total) HM_CUDA(cudaMemsetAsync(sys->d_w, 0, (size_t)P.w_total * sizeof(T), s));
  }
  {
    const int64_t nnz = sys->nnz;
    ProfScope ps(ctx, PC_SCATTER, Work{0.0, nnz * 32.0});
    const int grid = (int)std::min<int64_t>((nnz + 255) / 256, (int64_t)ctx->num_sms * 16);
    k_perm_values<<<std::max(grid, 1), 256, 0, s>>>(d_values, sys->d_psrc, nnz, sys->d_pvals, sys->d_pvals2);
  }
  for (int l = P.nlevels - 1; l >= 0; --l) {
    const LevelFactorPlan& lp = P.levels[l];
    {  // the level's fronts: zero, then A's entries (their children's level is still live)
      const int64_t f0 = P.level_front_begin[l], f1 = P.level_front_end[l];
      ProfScope ps(ctx, PC_SCATTER, Work{0.0, (double)es * (f1 - f0) + (16.0 + 8.0 + es) * P.level_entries[l]});
      if (f1 > f0) HM_CUDA(cudaMemsetAsync(F + f0, 0, (size_t)(f1 - f0) * sizeof(T), s));
      // the entry count of a level is known on the device only: a grid for about the
      // nonzeros the level's fronts hold, read bounds from the device
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((P.level_entries[l] + 255) / 256,
                                                                    (int64_t)ctx->num_sms * 16));
      k_scatter_level<T><<<grid, 256, 0, s>>>(d_values, sys->d_scat_src, sys->d_scat_dst, sys->d_lev_range, l, F);
    }
    for (size_t si = 0; si < lp.ea_parents.size(); ++si) {
      const auto& par = lp.ea_parents[si];
      if (par.count == 0 || lp.ea_max_nu[si] == 0) continue;
      ProfScope ps(ctx, PC_EXTEND_ADD, lp.ea_work[si]);
      const dim3 grid((unsigned)par.count, (unsigned)((lp.ea_max_nu[si] + 7) / 8));
      k_extend_add<T><<<grid, 256, 0, s>>>(par.dev(base), (int)si, sys->d_child_ptr, sys->d_child_list,
                                           P.d_front_off, P.d_nhat, P.d_np, sys->d_ifoff, sys->d_relmap, F);
    }
    debug_stage<T>(sys, "extendadd", l);
    if (lp.sweep.count) {
      ProfScope ps(ctx, PC_SWEEP, lp.sweep.work);
      launch_front_sweep<T>(lp.sweep.dev(base), lp.sweep.count, lp.sweep_maxn, sys->d_err, s);
    }
    if (lp.potrf.count) {
      {
        ProfScope ps(ctx, PC_POTRF, lp.potrf.work);
        launch_potrf<T>(lp.potrf.dev(base), lp.potrf.count, lp.potrf_maxn, sys->d_err, s);
      }
      if (lp.trsm.count) {
        ProfScope ps(ctx, PC_TRSM, lp.trsm.work);
        launch_trsm<T>(lp.trsm.dev(base), lp.trsm.count, lp.trsm_maxn, s);
      }
      run_gemm<T>(sys, lp.syrk, base, PC_GEMM_FACTOR);
      {
        ProfScope ps(ctx, PC_INVERSE, lp.dinv.work);
        launch_chol_inverse<T>(lp.dinv.dev(base), lp.dinv.count, lp.potrf_maxn, s);
      }
      debug_stage<T>(sys, "dense", l);
    }
    if (lp.n_hodlr && lp.bdlr.count) {
      ProfScope ps(ctx, PC_BDLR, lp.bdlr.work);
      launch_bdlr<T>(lp.bdlr.dev(base), lp.bdlr.count, lp.bdlr_maxnh, lp.bdlr_maxcap, ctx->opts.bdlr_depth, tol,
                     sys->d_first, P.d_np, sys->d_ifoff, sys->d_iflist, sys->d_prowptr, sys->d_pcol, s);
    }
    if (lp.n_hodlr) {
      if (lp.omega.count) {
        ProfScope ps(ctx, PC_SKETCH, lp.omega.work);
        launch_omega<T>(lp.omega.dev(base), lp.omega.count, ctx->opts.seed, s);
      }
      run_gemm<T>(sys, lp.sampY, base, PC_GEMM_FACTOR);
      run_qr<T>(sys, lp.qrY, base);
      debug_stage<T>(sys, "qrY", l);
      run_gemm<T>(sys, lp.sampZ, base, PC_GEMM_FACTOR);
      run_qr<T>(sys, lp.qrZ, base);
      if (lp.svd.count) {
        ProfScope ps(ctx, PC_SVD, lp.svd.work);
        launch_svd<T>(lp.svd.dev(base), lp.svd.count, lp.svd_maxk, tol, s);
      }
      debug_stage<T>(sys, "svd", l);
      run_gemm<T>(sys, lp.formU, base, PC_GEMM_FACTOR);
      run_gemm<T>(sys, lp.formV, base, PC_GEMM_FACTOR);
      run_gemm<T>(sys, lp.ffx, base, PC_GEMM_FACTOR);  // F_ff^HODLR written back (compress_ff)
      debug_stage<T>(sys, "formUV", l);
      {
        ProfScope ps(ctx, PC_INVERSE, lp.leaf_sweep.work);
        launch_front_sweep<T>(lp.leaf_sweep.dev(base), lp.leaf_sweep.count, lp.leaf_maxn, sys->d_err, s);
      }
      run_gemm<T>(sys, lp.leaf_x, base, PC_GEMM_FACTOR);  // X = D^{-1} Bo on the leaf rows
      debug_stage<T>(sys, "leaves", l);
      for (const auto& H : lp.heights) {
        run_gemm<T>(sys, H.pre, base, PC_GEMM_FACTOR);
        debug_stage<T>(sys, "core-pre", l);
        {
          ProfScope ps(ctx, PC_CORE_LU, H.lu.work);
          launch_core_lu<T>(H.lu.dev(base), H.lu.count, H.lu_maxk, ctx->max_smem, sys->d_err, s);
        }
        debug_stage<T>(sys, "core-lu", l);
        run_gemm<T>(sys, H.sg, base, PC_GEMM_FACTOR);
        run_gemm<T>(sys, H.upd, base, PC_GEMM_FACTOR);
        run_gemm<T>(sys, H.gm, base, PC_GEMM_FACTOR);
        debug_stage<T>(sys, "core-upd", l);
      }
      run_gemm<T>(sys, lp.schurT, base, PC_GEMM_FACTOR);
      run_gemm<T>(sys, lp.schurP, base, PC_GEMM_FACTOR);
      run_gemm<T>(sys, lp.schurF, base, PC_GEMM_FACTOR);
      debug_stage<T>(sys, "schur", l);
    }
    if (lp.pack.count) {  // the level's factor out of the fronts, for the apply
      ProfScope ps(ctx, PC_PACK, lp.pack.work);
      k_copy2d<T><<<lp.pack.count, 256, 0, s>>>(lp.pack.dev(base));
    }
  }
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

int factor_impl(hm_sys_s* sys, const double* d_values, double tol) {
  host_mark("factor: enter");
  int st = sys->precision == HM_PREC_FP64 ? factor_t<double>(sys, d_values, tol)
                                          : factor_t<float>(sys, d_values, tol);
  if (st != HM_OK) return st;
  host_mark("factor: launched");
  // The apply plan depends only on the analysis, so the one for the most recent
  // right-hand-side count is built on the host while the factorization runs.
  if (sys->ctx->last_nrhs > 0) {
    SolvePlan* sp = nullptr;
    HM_TRY(get_solve_plan(sys, sys->ctx->last_nrhs, &sp));
  }
  st = check_device_error(sys, "factor");
  host_mark("factor: device done");
  return st;
}

}  // namespace hm
