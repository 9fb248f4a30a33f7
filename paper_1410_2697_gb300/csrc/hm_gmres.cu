// hm_gmres.cu -- right-preconditioned flexible GMRES(m) in FP64 (Sections 1 and 3 of the
// paper: the approximate multifrontal solve preconditions GMRES, which restores the
// accuracy).  nrhs systems run in lockstep; each keeps its own Krylov basis.
//
//   V_j  (FP64)  Krylov vectors; Z_j = M^{-1} V_j stored in the factor precision (the
//               preconditioned vectors are exactly representable there), row-major (the
//               right-hand sides of a row side by side) for the multi-RHS SpMV;
//   w = A Z_j in FP64; Arnoldi by classical Gram-Schmidt applied twice (CGS2) with
//   block partial sums reduced in a fixed order (deterministic); Givens rotations and
//   the least-squares solve on the device; x += Z y at the end of a cycle; the TRUE
//   residual ||b - A x|| / ||b|| decides convergence.
#include <algorithm>
#include <cmath>

#include "hm_internal.h"

namespace hm {

constexpr int kDotThreads = 256;

// y[r] = A x[r]  (b == nullptr)   or   y[r] = b[r] - A x[r]; rows in new numbering.
// One thread per row and up to kSpmvR right-hand sides (blockIdx.y selects the group):
// the row's column indices and values are read once and reused for every product, and
// two nonzeros are in flight per iteration.
constexpr int kSpmvR = 16;

template <typename XT>
__global__ void __launch_bounds__(256) k_spmv(const int64_t* __restrict__ rowptr,
                                              const int32_t* __restrict__ col,
                                              const double* __restrict__ val, int n, int nrhs,
                                              const XT* __restrict__ x, int64_t ldx,
                                              double* __restrict__ y, int64_t ldy,
                                              const double* __restrict__ b, int64_t ldb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r0 = blockIdx.y * kSpmvR;
  const int nr = min(kSpmvR, nrhs - r0);
  const int64_t kb = rowptr[i], ke = rowptr[i + 1];
  double s[kSpmvR];
#pragma unroll
  for (int q = 0; q < kSpmvR; ++q) s[q] = 0.0;
  const XT* x0 = x + (int64_t)r0 * ldx;
#pragma unroll 2
  for (int64_t k = kb; k < ke; ++k) {
    const int c = col[k];
    const double v = val[k];
#pragma unroll
    for (int q = 0; q < kSpmvR; ++q)
      if (q < nr) s[q] = fma(v, (double)x0[c + (int64_t)q * ldx], s[q]);
  }
#pragma unroll
  for (int q = 0; q < kSpmvR; ++q)
    if (q < nr) {
      const int r = r0 + q;
      y[i + (int64_t)r * ldy] = b ? b[i + (int64_t)r * ldb] - s[q] : s[q];
    }
}

static dim3 spmv_grid(int n, int nrhs) { return dim3((n + 255) / 256, (nrhs + kSpmvR - 1) / kSpmvR); }

// Double-float SpMV for FP32 directions: y = A z with A = a_hi + a_lo (FP32 pair, 48 bits
// of each FP64 entry) and z exact in FP32.  Every product a_hi z is split exactly into
// p + e (FMA), a_lo z is added to the error term, and the row sum is carried as an
// unevaluated FP32 pair (hi, lo) with Knuth's two-sum, so the result carries about 2^-46
// relative error per term (native FP64: 2^-53) at FP32 instruction rates: GB300 issues
// FP64 FMAs at 1/64 of the FP32 rate, and this product is the inner loop of every GMRES
// iteration.  The convergence test keeps the native FP64 residual b - A x.
constexpr int kSpmvDF = 16;

// (the _rn intrinsics keep the compiler from contracting these into FMAs, which would
// break the exactness of the error terms)
__device__ __forceinline__ void df_add(float& hi, float& lo, float p, float e) {
  const float s = __fadd_rn(hi, p);
  const float bv = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

__global__ void __launch_bounds__(256) k_spmv_df(const int64_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ col,
                                                 const float2* __restrict__ val2, int n, int nrhs,
                                                 const float* __restrict__ z, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r0 = blockIdx.y * kSpmvDF;
  const int nr = min(kSpmvDF, nrhs - r0);
  const int64_t kb = rowptr[i], ke = rowptr[i + 1];
  float hi[kSpmvDF], lo[kSpmvDF];
#pragma unroll
  for (int q = 0; q < kSpmvDF; ++q) { hi[q] = 0.f; lo[q] = 0.f; }
  const bool vec = nr == kSpmvDF && (nrhs & 3) == 0;
#pragma unroll 2
  for (int64_t k = kb; k < ke; ++k) {
    const float2 a = val2[k];
    const float* zc = z + (int64_t)col[k] * nrhs + r0;
    float zz[kSpmvDF];
    if (vec) {
#pragma unroll
      for (int q = 0; q < kSpmvDF / 4; ++q) {
        const float4 t = reinterpret_cast<const float4*>(zc)[q];
        zz[4 * q] = t.x; zz[4 * q + 1] = t.y; zz[4 * q + 2] = t.z; zz[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < kSpmvDF; ++q) zz[q] = q < nr ? zc[q] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kSpmvDF; ++q) {
      const float p = __fmul_rn(a.x, zz[q]);
      const float e = fmaf(a.y, zz[q], fmaf(a.x, zz[q], -p));
      df_add(hi[q], lo[q], p, e);
    }
  }
#pragma unroll
  for (int q = 0; q < kSpmvDF; ++q)
    if (q < nr) y[i + (int64_t)(r0 + q) * n] = (double)hi[q] + (double)lo[q];
}

// y[r] = A z[r] with z stored row-major (the nrhs values of a row contiguous, as the
// preconditioned directions Z_j are kept): one thread per row and group of kSpmvRM
// right-hand sides, so a row's column indices and values are read once per group and
// each neighbour's values arrive as one contiguous run.
constexpr int kSpmvRM = 16;

template <typename ZT>
__global__ void __launch_bounds__(256) k_spmv_rm(const int64_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ col,
                                                 const double* __restrict__ val, int n, int nrhs,
                                                 const ZT* __restrict__ z, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r0 = blockIdx.y * kSpmvRM;
  const int nr = min(kSpmvRM, nrhs - r0);
  const int64_t kb = rowptr[i], ke = rowptr[i + 1];
  double s[kSpmvRM];
#pragma unroll
  for (int q = 0; q < kSpmvRM; ++q) s[q] = 0.0;
  if (nr == kSpmvRM && (nrhs & 3) == 0 && sizeof(ZT) == 4) {
    // 16 FP32 values per neighbour as four 16-byte loads (rows are 16-byte aligned)
    for (int64_t k = kb; k < ke; ++k) {
      const double v = val[k];
      const float4* zc = reinterpret_cast<const float4*>(z + (int64_t)col[k] * nrhs + r0);
#pragma unroll
      for (int q = 0; q < kSpmvRM / 4; ++q) {
        const float4 t = zc[q];
        s[4 * q] = fma(v, (double)t.x, s[4 * q]);
        s[4 * q + 1] = fma(v, (double)t.y, s[4 * q + 1]);
        s[4 * q + 2] = fma(v, (double)t.z, s[4 * q + 2]);
        s[4 * q + 3] = fma(v, (double)t.w, s[4 * q + 3]);
      }
    }
  } else {
    for (int64_t k = kb; k < ke; ++k) {
      const double v = val[k];
      const ZT* zc = z + (int64_t)col[k] * nrhs + r0;
#pragma unroll
      for (int q = 0; q < kSpmvRM; ++q)
        if (q < nr) s[q] = fma(v, (double)zc[q], s[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < kSpmvRM; ++q)
    if (q < nr) y[i + (int64_t)(r0 + q) * n] = s[q];
}

// Row chunks: every vector kernel runs on grid (nchunks, nrhs); chunk c covers rows
// [crow[c], crow[c+1]) of one block cseg[c] (chunks never straddle blocks), so a CTA
// serves one GMRES instance inst = r * nseg + cseg[c] and caches its scalars.
// V_i[r] starts at V + (i*nrhs + r)*n.

// out[i] = d[i] summed over the CTA, i < cnt: warp shuffles, then the warps' partials
// added in a fixed order by thread i (one barrier pair for all cnt sums; deterministic).
template <int NV>
__device__ __forceinline__ void block_store_sums(const double (&d)[NV], int cnt, double* red,
                                                 double* __restrict__ out) {
  constexpr int kWarps = kDotThreads / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (i < cnt) {
      const double v = warp_sum(d[i]);
      if (lane == 0) red[wid * NV + i] = v;
    }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) t += red[q * NV + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();  // red is reused by the next group
}

// Rows a thread keeps in flight in the chunk kernels: a thread issues the loads of R rows
// (R kDotThreads apart) before it uses any, so that enough bytes are in flight per SM to
// cover the DRAM latency.  The vector count NV is a template constant and every one of the
// NV vectors is read: a load guarded by a runtime count inside an unrolled loop may be
// issued whatever the guard says, so the kernels never see more vectors than they use.
template <int NV>
struct ChunkRows {
  static constexpr int v = NV == 1 ? 8 : NV <= 4 ? 4 : 2;
};

// part[(r*nchunks + c)*stride + i0 + i] = sum over chunk c of V_{i0+i}[r] . w[r], i < NV:
// w is read once, the NV products of a row are independent loads accumulated in registers
// (rows in the plain strided order), one block reduction for the NV sums.
template <int NV>
__global__ void __launch_bounds__(kDotThreads, NV <= 4 ? 3 : 2) k_multidot(const double* __restrict__ V,
                                                                           const double* __restrict__ w,
                                                                           int n, int nrhs, int i0, int stride,
                                                                           const int* __restrict__ crow,
                                                                           double* __restrict__ part) {
  constexpr int R = ChunkRows<NV>::v;
  __shared__ double red[kDotThreads / 32 * NV];
  const int r = blockIdx.y, c = blockIdx.x;
  const int b = crow[c], e = crow[c + 1];
  const double* wr = w + (int64_t)r * n;
  const int64_t vs = (int64_t)nrhs * n;
  const double* v0 = V + (int64_t)i0 * vs + (int64_t)r * n;
  double d[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) d[i] = 0.0;
  for (int k0 = b + threadIdx.x; k0 < e; k0 += kDotThreads * R) {
    double x[R], v[R][NV];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int k = k0 + j * kDotThreads;
      const bool in = k < e;
      const int kc = in ? k : b;  // an in-range address even for a slot past the end
      x[j] = in ? wr[kc] : 0.0;
#pragma unroll
      for (int i = 0; i < NV; ++i) v[j][i] = in ? v0[i * vs + kc] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
      for (int i = 0; i < NV; ++i) d[i] = fma(v[j][i], x[j], d[i]);
  }
  block_store_sums<NV>(d, NV, red, part + ((int64_t)r * gridDim.x + c) * stride + i0);
}

// Fused Gram-Schmidt step over exactly NV basis vectors: over the chunk's rows
// w[r] -= sum_i V_i[r] coef_i, then the chunk's partial sums of the updated rows --
// V_i[r] . w[r] for i < NV (norm == 0: the next CGS pass's projections) or w[r] . w[r]
// (norm == 1: the squared norm that normalises the new basis vector) ->
// part[(r*nchunks + c)*pstride + i].
template <int NV>
__global__ void __launch_bounds__(kDotThreads, NV <= 4 ? 3 : 2) k_gs_update_dots(
    const double* __restrict__ V, double* __restrict__ w, int n, int nrhs, int stride,
    const double* __restrict__ coef, const int* __restrict__ crow, const int* __restrict__ cseg, int nseg,
    int norm, int pstride, double* __restrict__ part) {
  constexpr int R = ChunkRows<NV>::v;
  __shared__ double cs[NV];
  __shared__ double red[kDotThreads / 32 * NV];
  const int r = blockIdx.y, c = blockIdx.x;
  const int inst = r * nseg + cseg[c];
  if (threadIdx.x < NV) cs[threadIdx.x] = coef[(int64_t)inst * stride + threadIdx.x];
  __syncthreads();
  double* wr = w + (int64_t)r * n;
  const double* v0 = V + (int64_t)r * n;
  const int64_t vs = (int64_t)nrhs * n;
  const int e = crow[c + 1];
  double d[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) d[i] = 0.0;
  for (int k0 = crow[c] + threadIdx.x; k0 < e; k0 += kDotThreads * R) {
    double vk[R][NV], sv[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int k = k0 + j * kDotThreads;
      const bool in = k < e;
      const int kc = in ? k : crow[c];  // an in-range address even for a slot past the end
      sv[j] = in ? wr[kc] : 0.0;
#pragma unroll
      for (int i = 0; i < NV; ++i) vk[j][i] = in ? v0[i * vs + kc] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int k = k0 + j * kDotThreads;
      double t = sv[j];
#pragma unroll
      for (int i = 0; i < NV; ++i) t -= vk[j][i] * cs[i];
      if (k < e) wr[k] = t;
      if (norm) {
        d[0] = fma(t, t, d[0]);
      } else {
#pragma unroll
        for (int i = 0; i < NV; ++i) d[i] = fma(vk[j][i], t, d[i]);
      }
    }
  }
  block_store_sums<NV>(d, norm ? 1 : NV, red, part + ((int64_t)r * gridDim.x + c) * pstride);
}

// The fused step covers bases of up to kFusedGs vectors; wider ones take k_gs_update
// followed by k_multidot.
constexpr int kFusedGs = 8;

#define HM_NV_SWITCH(cnt, CALL) \
  switch (cnt) {                \
    case 1: CALL(1); break;     \
    case 2: CALL(2); break;     \
    case 3: CALL(3); break;     \
    case 4: CALL(4); break;     \
    case 5: CALL(5); break;     \
    case 6: CALL(6); break;     \
    case 7: CALL(7); break;     \
    default: CALL(8); break;    \
  }

// Partial dot products with all nvec basis vectors: groups of at most eight vectors,
// each group one launch of the kernel instantiated for its exact size.
static void launch_multidot(const double* V, const double* w, int n, int nrhs, int nvec, int stride,
                            const int* crow, double* part, int nchunks, cudaStream_t s) {
  const dim3 g((unsigned)nchunks, (unsigned)nrhs);
  for (int i0 = 0; i0 < nvec; i0 += 8) {
    const int cnt = std::min(8, nvec - i0);
#define HM_MD(NV) k_multidot<NV><<<g, kDotThreads, 0, s>>>(V, w, n, nrhs, i0, stride, crow, part)
    HM_NV_SWITCH(cnt, HM_MD)
#undef HM_MD
  }
}

// nvec in [1, kFusedGs]
static void launch_gs_update_dots(const double* V, double* w, int n, int nrhs, int nvec, int stride,
                                  const double* coef, const int* crow, const int* cseg, int nseg, int norm,
                                  int pstride, double* part, int nchunks, cudaStream_t s) {
  const dim3 g((unsigned)nchunks, (unsigned)nrhs);
#define HM_GSU(NV) \
  k_gs_update_dots<NV><<<g, kDotThreads, 0, s>>>(V, w, n, nrhs, stride, coef, crow, cseg, nseg, norm, pstride, part)
  HM_NV_SWITCH(nvec, HM_GSU)
#undef HM_GSU
}
#undef HM_NV_SWITCH

// h[inst*stride + i] = sum of the block's chunk partials, and h_acc[inst*stride + i] += the
// same sum when h_acc is given.  One warp per output: lane l adds chunks l, l+32, ... in
// order, then a fixed butterfly across the lanes (deterministic; the chunk loads of a
// lane are independent, so the sum costs a few L2 round trips, not one per chunk).
__global__ void k_reduce_dots(const double* __restrict__ part, int nchunks, const int* __restrict__ cptr,
                              int nseg, int ninst, int nvec, int stride, double* __restrict__ h,
                              double* __restrict__ h_acc) {
  const int e = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= ninst * nvec) return;  // uniform per warp
  const int inst = e / nvec, i = e % nvec;
  const int r = inst / nseg, sg = inst % nseg;
  double s = 0.0;
  for (int c = cptr[sg] + lane; c < cptr[sg + 1]; c += 32) s += part[((int64_t)r * nchunks + c) * stride + i];
  s = warp_sum(s);
  if (lane == 0) {
    h[(int64_t)inst * stride + i] = s;
    if (h_acc) h_acc[(int64_t)inst * stride + i] += s;
  }
}

static void launch_reduce_dots(const double* part, int nchunks, const int* cptr, int nseg, int ninst, int nvec,
                               int stride, double* h, double* h_acc, cudaStream_t s) {
  const int64_t threads = (int64_t)ninst * nvec * 32;
  k_reduce_dots<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(part, nchunks, cptr, nseg, ninst, nvec, stride,
                                                                  h, h_acc);
}

// w[r] -= sum_{i < nvec} V_i[r] * coef[inst*stride + i]
__global__ void k_gs_update(const double* __restrict__ V, double* __restrict__ w, int n, int nrhs,
                            int nvec, int stride, const double* __restrict__ coef,
                            const int* __restrict__ crow, const int* __restrict__ cseg, int nseg) {
  __shared__ double cs[256];  // nvec <= restart + 1 <= 201
  const int r = blockIdx.y, c = blockIdx.x;
  const int inst = r * nseg + cseg[c];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) cs[i] = coef[(int64_t)inst * stride + i];
  __syncthreads();
  double* wr = w + (int64_t)r * n;
  for (int k = crow[c] + threadIdx.x; k < crow[c + 1]; k += blockDim.x) {
    double s = wr[k];
    for (int i = 0; i < nvec; ++i) s -= V[((int64_t)i * nrhs + r) * n + k] * cs[i];
    wr[k] = s;
  }
}

// dst[r] = src[r] / ||.||, with ||.||^2 = ss[inst*stride] (0 if the norm is 0); the same
// values also go to cast (the factor precision: the next preconditioner input).
template <typename T>
__global__ void k_scale(const double* __restrict__ src, double* __restrict__ dst, T* __restrict__ cast, int n,
                        int nrhs, const double* __restrict__ ss, int stride, const int* __restrict__ crow,
                        const int* __restrict__ cseg, int nseg) {
  const int r = blockIdx.y, c = blockIdx.x;
  const int inst = r * nseg + cseg[c];
  const double nr = sqrt(ss[(int64_t)inst * stride]);
  const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
  const double* sr = src + (int64_t)r * n;
  double* dr = dst + (int64_t)r * n;
  T* cr = cast + (int64_t)r * n;
  const int e = crow[c + 1];
  for (int k = crow[c] + threadIdx.x; k < e; k += blockDim.x) {
    const double t = nr > 0.0 ? sr[k] * inv : 0.0;
    dr[k] = t;
    cr[k] = (T)t;
  }
}

// Givens step for column j (thread per instance): H column = h (h1 + h2), H[j+1,j] = ||w||.
__global__ void k_givens(double* __restrict__ H, const double* __restrict__ hv, int hstride,
                         const double* __restrict__ ss, int ssstride, double* __restrict__ cs,
                         double* __restrict__ sn, double* __restrict__ g, const double* __restrict__ bnorm,
                         double* __restrict__ res, int* __restrict__ len, int j, int m, int ninst,
                         double rtol) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ninst) return;
  double* Hr = H + (int64_t)r * (m + 1) * m;
  double* col = Hr + (int64_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = hv[(int64_t)r * hstride + i];
  col[j + 1] = sqrt(ss[(int64_t)r * ssstride]);
  double* c = cs + (int64_t)r * m;
  double* s = sn + (int64_t)r * m;
  double* gr = g + (int64_t)r * (m + 1);
  for (int i = 0; i < j; ++i) {
    const double t = c[i] * col[i] + s[i] * col[i + 1];
    col[i + 1] = -s[i] * col[i] + c[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  if (den > 0.0) {
    c[j] = col[j] / den;
    s[j] = col[j + 1] / den;
  } else {
    c[j] = 1.0;
    s[j] = 0.0;
  }
  col[j] = den;
  col[j + 1] = 0.0;
  gr[j + 1] = -s[j] * gr[j];
  gr[j] = c[j] * gr[j];
  const double est = bnorm[r] > 0.0 ? fabs(gr[j + 1]) / bnorm[r] : 0.0;
  res[r] = est;
  if (len[r] == 0 && est <= rtol) len[r] = j + 1;
}

// y = R^{-1} g over len[inst] (thread per instance); len == 0 -> use jend.
__global__ void k_backsolve(const double* __restrict__ H, const double* __restrict__ g,
                            double* __restrict__ y, int* __restrict__ len, int jend, int m, int ninst) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ninst) return;
  int L = len[r];
  if (L == 0 || L > jend) L = jend;
  len[r] = L;
  const double* Hr = H + (int64_t)r * (m + 1) * m;
  const double* gr = g + (int64_t)r * (m + 1);
  double* yr = y + (int64_t)r * m;
  for (int i = L - 1; i >= 0; --i) {
    double v = gr[i];
    for (int k = i + 1; k < L; ++k) v -= Hr[i + (int64_t)k * (m + 1)] * yr[k];
    const double d = Hr[i + (int64_t)i * (m + 1)];
    yr[i] = d != 0.0 ? v / d : 0.0;
  }
  for (int i = L; i < m; ++i) yr[i] = 0.0;
}

// x[r] += sum_{j < len[inst]} Z_j[r] y[inst][j]   (Z_j row-major: element (k, r) at k nrhs + r).
// A tile of rt = min(256, 1024 / nrhs) rows x every right-hand side (at most 1024 values,
// kUxVals per thread) is read along rows (coalesced) and transposed through shared memory
// into the column-major x.  A thread issues the loads of its values together (j outer),
// and reads its x values before it writes any; a chunk's tiles are spread over gridDim.y
// CTAs.
constexpr int kUxVals = 4;
template <typename ZT>
__global__ void __launch_bounds__(256) k_update_x(double* __restrict__ x, const ZT* __restrict__ Z,
                                                  const double* __restrict__ y, const int* __restrict__ len, int n,
                                                  int nrhs, int m, const int* __restrict__ crow,
                                                  const int* __restrict__ cseg, int nseg) {
  __shared__ double tile[1024 + 256];  // rt x (nrhs + 1)
  const int c = blockIdx.x, seg = cseg[c];
  const int rt = min(256, 1024 / nrhs), ld = nrhs + 1;
  const int64_t zs = (int64_t)n * nrhs;
  for (int k0 = crow[c] + rt * blockIdx.y; k0 < crow[c + 1]; k0 += rt * gridDim.y) {
    const int rows = min(rt, crow[c + 1] - k0), cnt = rows * nrhs;
    double acc[kUxVals];
    const ZT* zp[kUxVals];
    const double* yp[kUxVals];
    int L[kUxVals], lmax = 0;
#pragma unroll
    for (int q = 0; q < kUxVals; ++q) {
      const int e = threadIdx.x + q * 256;
      acc[q] = 0.0;
      L[q] = 0;
      zp[q] = Z;
      yp[q] = y;
      if (e < cnt) {
        const int kk = e / nrhs, r = e - kk * nrhs;
        const int inst = r * nseg + seg;
        L[q] = len[inst];
        zp[q] = Z + (int64_t)(k0 + kk) * nrhs + r;
        yp[q] = y + (int64_t)inst * m;
        lmax = max(lmax, L[q]);
      }
    }
    // (every address below stays inside Z and y for j < lmax <= m, whatever q)
    for (int j = 0; j < lmax; ++j) {
#pragma unroll
      for (int q = 0; q < kUxVals; ++q)
        if (j < L[q]) acc[q] = fma((double)zp[q][j * zs], yp[q][j], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kUxVals; ++q) {
      const int e = threadIdx.x + q * 256;
      if (e < cnt) {
        const int kk = e / nrhs, r = e - kk * nrhs;
        tile[kk * ld + r] = acc[q];
      }
    }
    __syncthreads();
    double xv[kUxVals];
#pragma unroll
    for (int q = 0; q < kUxVals; ++q) {
      const int e = threadIdx.x + q * 256;
      const int ec = e < cnt ? e : 0;  // an in-range address even for a slot past the end
      const int r = ec / rows, kk = ec - r * rows;
      xv[q] = e < cnt ? x[(int64_t)r * n + k0 + kk] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kUxVals; ++q) {
      const int e = threadIdx.x + q * 256;
      if (e < cnt) {
        const int r = e / rows, kk = e - r * rows;
        x[(int64_t)r * n + k0 + kk] = xv[q] + tile[kk * ld + r];
      }
    }
    __syncthreads();
  }
}

// Start of a cycle: V_0 = r / beta (inactive instances get 0), also cast to the factor
// precision (the first preconditioner input of the cycle).
template <typename T>
__global__ void k_cycle_init(const double* __restrict__ rvec, double* __restrict__ V0, T* __restrict__ cast,
                             int n, int nrhs, const double* __restrict__ ss, const int* __restrict__ active,
                             const int* __restrict__ crow, const int* __restrict__ cseg, int nseg) {
  const int r = blockIdx.y, c = blockIdx.x;
  const int inst = r * nseg + cseg[c];
  const double beta = sqrt(ss[inst]);
  const bool on = active[inst] && beta > 0.0;
  const double inv = on ? 1.0 / beta : 0.0;
  const double* rr = rvec + (int64_t)r * n;
  double* vr = V0 + (int64_t)r * n;
  T* cr = cast + (int64_t)r * n;
  const int e = crow[c + 1];
  for (int k = crow[c] + threadIdx.x; k < e; k += blockDim.x) {
    const double t = on ? rr[k] * inv : 0.0;
    vr[k] = t;
    cr[k] = (T)t;
  }
}

__global__ void k_cycle_g(double* __restrict__ g, int* __restrict__ len, const double* __restrict__ ss,
                          const int* __restrict__ active, int m, int ninst) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ninst) return;
  double* gr = g + (int64_t)r * (m + 1);
  for (int i = 0; i <= m; ++i) gr[i] = 0.0;
  gr[0] = active[r] ? sqrt(ss[r]) : 0.0;
  len[r] = 0;
}

// ------------------------------------------------------------------------------------
// Host driver
// ------------------------------------------------------------------------------------
static int gm_alloc(hm_sys_s* sys, void** p, size_t bytes) {
  return dev_alloc_ctx(sys->ctx, &sys->gm.allocs, p, bytes);
}

static int ensure_workspace(hm_sys_s* sys, int nrhs, int m) {
  auto& G = sys->gm;
  if (G.nrhs == nrhs && G.m == m) return HM_OK;
  dev_free_all(sys->ctx, &G.allocs);
  if (G.h_res) { cudaFreeHost(G.h_res); G.h_res = nullptr; }
  const int64_t n = sys->n;
  const int nseg = sys->nseg;
  const int64_t ninst = (int64_t)nrhs * nseg;
  const int es = sys->precision == HM_PREC_FP64 ? 8 : 4;
  // row chunks: about two per SM over the whole vector, never straddling a block (the
  // vector kernels run one CTA per (chunk, right-hand side))
  const int64_t L = std::max<int64_t>(1024, (n + 2 * sys->ctx->num_sms - 1) / (2 * sys->ctx->num_sms));
  std::vector<int> crow(1, 0), cseg, cptr(1, 0);
  for (int sg = 0; sg < nseg; ++sg) {
    const int b = sys->h_seg_ptr[sg], e = sys->h_seg_ptr[sg + 1];
    const int64_t nc = std::max<int64_t>(1, (e - b + L - 1) / L);
    for (int64_t c = 0; c < nc; ++c) {
      crow.push_back((int)(b + (e - b) * (c + 1) / nc));
      cseg.push_back(sg);
    }
    cptr.push_back((int)cseg.size());
  }
  G.nchunks = (int)cseg.size();
  const int stride = m + 2;
  HM_TRY(gm_alloc(sys, (void**)&G.V, sizeof(double) * (m + 1) * nrhs * n));
  HM_TRY(gm_alloc(sys, &G.Z, (size_t)es * m * nrhs * n));
  HM_TRY(gm_alloc(sys, &G.wT, (size_t)es * nrhs * n));
  HM_TRY(gm_alloc(sys, (void**)&G.w, sizeof(double) * nrhs * n));
  HM_TRY(gm_alloc(sys, (void**)&G.b, sizeof(double) * nrhs * n));
  HM_TRY(gm_alloc(sys, (void**)&G.x, sizeof(double) * nrhs * n));
  HM_TRY(gm_alloc(sys, (void**)&G.r, sizeof(double) * nrhs * n));
  HM_TRY(gm_alloc(sys, (void**)&G.H, sizeof(double) * ninst * (m + 1) * m));
  HM_TRY(gm_alloc(sys, (void**)&G.cs, sizeof(double) * ninst * m));
  HM_TRY(gm_alloc(sys, (void**)&G.sn, sizeof(double) * ninst * m));
  HM_TRY(gm_alloc(sys, (void**)&G.g, sizeof(double) * ninst * (m + 1)));
  HM_TRY(gm_alloc(sys, (void**)&G.y, sizeof(double) * ninst * m));
  HM_TRY(gm_alloc(sys, (void**)&G.bnorm, sizeof(double) * ninst));
  HM_TRY(gm_alloc(sys, (void**)&G.res, sizeof(double) * ninst * 4));
  HM_TRY(gm_alloc(sys, (void**)&G.part, sizeof(double) * (size_t)G.nchunks * nrhs * stride));
  HM_TRY(gm_alloc(sys, (void**)&G.hv, sizeof(double) * ninst * stride * 3));
  HM_TRY(gm_alloc(sys, (void**)&G.len, sizeof(int) * ninst * 2));
  HM_TRY(gm_alloc(sys, (void**)&G.crow, sizeof(int) * crow.size()));
  HM_TRY(gm_alloc(sys, (void**)&G.cseg, sizeof(int) * cseg.size()));
  HM_TRY(gm_alloc(sys, (void**)&G.cptr, sizeof(int) * cptr.size()));
  cudaStream_t s = sys->ctx->stream;
  HM_CUDA(cudaMemcpyAsync(G.crow, crow.data(), sizeof(int) * crow.size(), cudaMemcpyHostToDevice, s));
  HM_CUDA(cudaMemcpyAsync(G.cseg, cseg.data(), sizeof(int) * cseg.size(), cudaMemcpyHostToDevice, s));
  HM_CUDA(cudaMemcpyAsync(G.cptr, cptr.data(), sizeof(int) * cptr.size(), cudaMemcpyHostToDevice, s));
  HM_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  HM_CUDA(cudaMallocHost((void**)&G.h_res, sizeof(double) * ninst * 4 + sizeof(int) * ninst * 2));
  G.nrhs = nrhs;
  G.m = m;
  return HM_OK;
}

// ss[inst*stride] = ||v restricted to the instance||^2 (deterministic)
static void sqnorm(hm_sys_s* sys, const double* v, double* ss, int stride, int nrhs) {
  auto& G = sys->gm;
  cudaStream_t s = sys->ctx->stream;
  const int ninst = nrhs * sys->nseg;
  ProfScope ps(sys->ctx, PC_DOTS, Work{2.0 * sys->n * nrhs, 8.0 * sys->n * nrhs}, 2);
  // with V = v and nvec = 1 the "basis" is v itself
  launch_multidot(v, v, sys->n, nrhs, 1, stride, G.crow, G.part, G.nchunks, s);
  launch_reduce_dots(G.part, G.nchunks, G.cptr, sys->nseg, ninst, 1, stride, ss, nullptr, s);
}

// One restart cycle of GMRES(m) over the instances with active[inst] = 1 (right
// preconditioning, flexible form): V_0 = r / ||r||, then at most min(m, budget) Arnoldi
// steps, each the preconditioner apply, the double-float Krylov product, CGS2 and a
// Givens rotation, stopping early once every active instance's rotated residual
// estimate is at or below rtol; then x += Z y and the true FP64 residual r = b - A x.
// *its = the Arnoldi steps run.
template <typename T>
static int gm_cycle(hm_sys_s* sys, int nrhs, double rtol, int budget, const std::vector<int>& active, int* its) {
  const int m = std::max(1, sys->ctx->opts.restart);
  auto& G = sys->gm;
  cudaStream_t s = sys->ctx->stream;
  const int n = sys->n;
  const int64_t nn = (int64_t)n * nrhs;
  const int stride = m + 2;
  const int nseg = sys->nseg, ninst = nrhs * nseg;
  const dim3 vgrid((unsigned)G.nchunks, (unsigned)nrhs);
  int* d_active = G.len + ninst;
  double* rss = G.hv + 2 * (int64_t)ninst * stride + ninst;  // squared residual norms
  T* Z = (T*)G.Z;
  const int max_iters = budget;
  int iters = 0;
  HM_CUDA(cudaMemcpyAsync(d_active, active.data(), sizeof(int) * ninst, cudaMemcpyHostToDevice, s));
  {
    ProfScope ps(sys->ctx, PC_VECTOR, Work{(double)nn, (16.0 + sizeof(T)) * nn}, 2);
    k_cycle_init<T><<<vgrid, 256, 0, s>>>(G.r, G.V, (T*)G.wT, n, nrhs, rss, d_active, G.crow, G.cseg, nseg);
    k_cycle_g<<<(ninst + 63) / 64, 64, 0, s>>>(G.g, G.len, rss, d_active, m, ninst);
  }
  int j = 0;
  for (; j < m && iters < max_iters; ++j) {
    T* Zj = Z + (int64_t)j * nrhs * n;
    // G.wT holds V_j in the factor precision (written with V_j by k_cycle_init / k_scale)
    HM_TRY(apply_impl_rowmajor(sys, nrhs, G.wT, Zj));  // Z_j row-major
    {
      ProfScope ps(sys->ctx, PC_SPMV, Work{2.0 * sys->nnz * nrhs,
                                           12.0 * sys->nnz + 8.0 * n + (8.0 + sizeof(T)) * nn});
      if (sizeof(T) == 4)
        k_spmv_df<<<dim3((n + 255) / 256, (nrhs + kSpmvDF - 1) / kSpmvDF), 256, 0, s>>>(
            sys->d_prowptr, sys->d_pcol, sys->d_pvals2, n, nrhs, (const float*)Zj, G.w);
      else
        k_spmv_rm<T><<<dim3((n + 255) / 256, (nrhs + kSpmvRM - 1) / kSpmvRM), 256, 0, s>>>(
            sys->d_prowptr, sys->d_pcol, sys->d_pvals, n, nrhs, Zj, G.w);
    }
    // CGS2: h1 = V^T w, w -= V h1, h2 = V^T w, w -= V h2, ||w||^2
    double* h1 = G.hv;
    double* h2 = G.hv + (int64_t)ninst * stride;
    double* wss = G.hv + 2 * (int64_t)ninst * stride + 2 * ninst;  // ||w||^2 per instance
    const int nvec = j + 1;
    {
      ProfScope ps(sys->ctx, PC_DOTS, Work{2.0 * nvec * nn, 8.0 * (nvec + 1) * nn}, 2);
      launch_multidot(G.V, G.w, n, nrhs, nvec, stride, G.crow, G.part, G.nchunks, s);
      launch_reduce_dots(G.part, G.nchunks, G.cptr, nseg, ninst, nvec, stride, h1, nullptr, s);
    }
    if (nvec <= kFusedGs) {
      {
        ProfScope ps(sys->ctx, PC_GS_UPDATE, Work{4.0 * nvec * nn, 8.0 * (nvec + 2) * nn}, 2);
        launch_gs_update_dots(G.V, G.w, n, nrhs, nvec, stride, h1, G.crow, G.cseg, nseg, 0, stride, G.part,
                              G.nchunks, s);
        launch_reduce_dots(G.part, G.nchunks, G.cptr, nseg, ninst, nvec, stride, h2, h1, s);  // h1 += h2
      }
      {
        ProfScope ps(sys->ctx, PC_GS_UPDATE, Work{2.0 * (nvec + 1) * nn, 8.0 * (nvec + 2) * nn}, 2);
        launch_gs_update_dots(G.V, G.w, n, nrhs, nvec, stride, h2, G.crow, G.cseg, nseg, 1, 1, G.part,
                              G.nchunks, s);
        launch_reduce_dots(G.part, G.nchunks, G.cptr, nseg, ninst, 1, 1, wss, nullptr, s);
      }
    } else {
      {
        ProfScope ps(sys->ctx, PC_GS_UPDATE, Work{2.0 * nvec * nn, 8.0 * (nvec + 2) * nn});
        k_gs_update<<<vgrid, 256, 0, s>>>(G.V, G.w, n, nrhs, nvec, stride, h1, G.crow, G.cseg, nseg);
      }
      {
        ProfScope ps(sys->ctx, PC_DOTS, Work{2.0 * nvec * nn, 8.0 * (nvec + 1) * nn}, 2);
        launch_multidot(G.V, G.w, n, nrhs, nvec, stride, G.crow, G.part, G.nchunks, s);
        launch_reduce_dots(G.part, G.nchunks, G.cptr, nseg, ninst, nvec, stride, h2, h1, s);  // h1 += h2
      }
      {
        ProfScope ps(sys->ctx, PC_GS_UPDATE, Work{2.0 * nvec * nn, 8.0 * (nvec + 2) * nn});
        k_gs_update<<<vgrid, 256, 0, s>>>(G.V, G.w, n, nrhs, nvec, stride, h2, G.crow, G.cseg, nseg);
      }
      sqnorm(sys, G.w, wss, 1, nrhs);
    }
    {
      ProfScope ps(sys->ctx, PC_VECTOR, Work{(double)nn, (16.0 + sizeof(T)) * nn});
      k_scale<T><<<vgrid, 256, 0, s>>>(G.w, G.V + (int64_t)(j + 1) * nrhs * n, (T*)G.wT, n, nrhs, wss, 1,
                                       G.crow, G.cseg, nseg);
    }
    {
      ProfScope ps(sys->ctx, PC_GMRES_SMALL, Work{});
      k_givens<<<(ninst + 63) / 64, 64, 0, s>>>(G.H, h1, stride, wss, 1, G.cs, G.sn, G.g, G.bnorm,
                                                G.res, G.len, j, m, ninst, rtol);
    }
    ++iters;
    HM_CUDA(cudaMemcpyAsync(G.h_res, G.res, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    host_mark("gmres: iteration");
    bool all = true;
    for (int r = 0; r < ninst; ++r)
      if (active[r] && !(G.h_res[r] <= rtol)) all = false;
    if (all) { ++j; break; }
  }
  const int jend = std::min(j, m);
  {
    ProfScope ps(sys->ctx, PC_GMRES_SMALL, Work{});
    k_backsolve<<<(ninst + 63) / 64, 64, 0, s>>>(G.H, G.g, G.y, G.len, jend, m, ninst);
  }
  {
    ProfScope ps(sys->ctx, PC_VECTOR, Work{2.0 * jend * nn, (16.0 + sizeof(T) * jend) * nn});
    const int split = std::max(1, (6 * sys->ctx->num_sms + G.nchunks - 1) / G.nchunks);
    k_update_x<T><<<dim3(G.nchunks, split), 256, 0, s>>>(G.x, Z, G.y, G.len, n, nrhs, m, G.crow, G.cseg, nseg);
  }
  {
    ProfScope ps(sys->ctx, PC_SPMV, Work{2.0 * sys->nnz * nrhs, 12.0 * sys->nnz + 8.0 * n + 24.0 * nn});
    k_spmv<double><<<spmv_grid(n, nrhs), 256, 0, s>>>(sys->d_prowptr, sys->d_pcol, sys->d_pvals, n, nrhs,
                                                   G.x, n, G.r, n, G.b, n);
  }
  sqnorm(sys, G.r, rss, 1, nrhs);
  *its = iters;
  return HM_OK;
}

template <typename T>
static int gmres_t(hm_sys_s* sys, int nrhs, const double* d_b, double rtol, int max_iters,
                   double* d_x, hm_solve_info* info) {
  host_mark("gmres: enter");
  const int m = std::max(1, sys->ctx->opts.restart);
  HM_TRY(ensure_workspace(sys, nrhs, m));
  host_mark("gmres: workspace");
  auto& G = sys->gm;
  cudaStream_t s = sys->ctx->stream;
  const int n = sys->n;
  const int64_t nn = (int64_t)n * nrhs;
  const int stride = m + 2;
  const int nseg = sys->nseg, ninst = nrhs * nseg;  // instance = r * nseg + block
  {
    ProfScope ps(sys->ctx, PC_VECTOR, Work{0.0, 20.0 * nn});
    launch_permute_in(d_b, G.b, sys->d_perm, n, nrhs, s);
    HM_CUDA(cudaMemsetAsync(G.x, 0, sizeof(double) * nn, s));
  }
  // ||b|| per instance
  double* bn2 = G.hv + 2 * (int64_t)ninst * stride;  // scratch: squared norms (stride 1)
  sqnorm(sys, G.b, bn2, 1, nrhs);
  std::vector<double> hb(ninst);
  HM_CUDA(cudaMemcpyAsync(hb.data(), bn2, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  std::vector<double> bnorm(ninst);
  for (int r = 0; r < ninst; ++r) bnorm[r] = std::sqrt(hb[r]);
  HM_CUDA(cudaMemcpyAsync(G.bnorm, bnorm.data(), sizeof(double) * ninst, cudaMemcpyHostToDevice, s));
  // r = b (x0 = 0)
  HM_CUDA(cudaMemcpyAsync(G.r, G.b, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  std::vector<double> relres(ninst);
  std::vector<int> active(ninst);
  for (int r = 0; r < ninst; ++r) relres[r] = bnorm[r] > 0 ? 1.0 : 0.0;
  int iters = 0, cycles = 0;
  double* rss = G.hv + 2 * (int64_t)ninst * stride + ninst;  // squared residual norms
  HM_CUDA(cudaMemcpyAsync(rss, bn2, sizeof(double) * ninst, cudaMemcpyDeviceToDevice, s));
  bool done = true;
  for (int r = 0; r < ninst; ++r) done = done && relres[r] <= rtol;
  while (!done && iters < max_iters) {
    for (int r = 0; r < ninst; ++r) active[r] = relres[r] > rtol ? 1 : 0;
    int j = 0;
    HM_TRY(gm_cycle<T>(sys, nrhs, rtol, max_iters - iters, active, &j));
    iters += j;
    std::vector<double> hr(ninst);
    HM_CUDA(cudaMemcpyAsync(hr.data(), rss, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    ++cycles;
    done = true;
    for (int r = 0; r < ninst; ++r) {
      relres[r] = bnorm[r] > 0 ? std::sqrt(hr[r]) / bnorm[r] : 0.0;
      if (!(relres[r] <= rtol)) done = false;
    }
  }
  {
    ProfScope ps(sys->ctx, PC_VECTOR, Work{0.0, 20.0 * nn});
    launch_permute_out(G.x, d_x, sys->d_perm, n, nrhs, s);
  }
  HM_CUDA(cudaStreamSynchronize(s));
  host_mark("gmres: done");
  HM_CUDA(cudaGetLastError());
  if (info) {
    info->iters = iters;
    info->restarts = cycles;
    double mx = 0;
    for (double v : relres) mx = std::max(mx, v);
    info->relres = mx;
    info->converged = done ? 1 : 0;
  }
  HM_TRY(check_device_error(sys, "solve"));
  return done ? HM_OK : HM_ERR_NO_CONVERGENCE;
}

// x += z (z in the factor's precision), column-major n x nrhs.
template <typename T>
__global__ void k_add_cast(double* __restrict__ x, const T* __restrict__ z, int64_t nn) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x)
    x[e] += (double)z[e];
}

// Direct mode: x = M^{-1} b, then `refine` steps x += M^{-1} (b - A x) with the FP64
// residual; the relative residual of every instance is reported.
template <typename T>
static int direct_t(hm_sys_s* sys, int nrhs, const double* d_b, int refine, double* d_x, hm_solve_info* info) {
  const int m = std::max(1, sys->ctx->opts.restart);
  HM_TRY(ensure_workspace(sys, nrhs, m));  // the GMRES workspace: b, x, r, staging, norms
  auto& G = sys->gm;
  cudaStream_t s = sys->ctx->stream;
  const int n = sys->n;
  const int64_t nn = (int64_t)n * nrhs;
  const int stride = m + 2;
  const int ninst = nrhs * sys->nseg;
  T* zT = (T*)G.Z;  // first Krylov block as the apply's output
  const unsigned eg = (unsigned)std::min<int64_t>((nn + 255) / 256, 4096);
  {
    ProfScope ps(sys->ctx, PC_VECTOR, Work{0.0, 20.0 * nn});
    launch_permute_in(d_b, G.b, sys->d_perm, n, nrhs, s);
    HM_CUDA(cudaMemsetAsync(G.x, 0, sizeof(double) * nn, s));
    HM_CUDA(cudaMemcpyAsync(G.r, G.b, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  }
  for (int it = 0; it <= refine; ++it) {
    {
      ProfScope ps(sys->ctx, PC_VECTOR, Work{0.0, (8.0 + sizeof(T)) * nn});
      launch_cast_to<T>(G.r, (T*)G.wT, nn, s);
    }
    HM_TRY(apply_impl(sys, nrhs, G.wT, zT));
    {
      ProfScope ps(sys->ctx, PC_VECTOR, Work{(double)nn, (16.0 + sizeof(T)) * nn});
      k_add_cast<T><<<eg, 256, 0, s>>>(G.x, zT, nn);
    }
    {
      ProfScope ps(sys->ctx, PC_SPMV, Work{2.0 * sys->nnz * nrhs, 12.0 * sys->nnz + 8.0 * n + 24.0 * nn});
      k_spmv<double><<<spmv_grid(n, nrhs), 256, 0, s>>>(sys->d_prowptr, sys->d_pcol, sys->d_pvals, n, nrhs,
                                                        G.x, n, G.r, n, G.b, n);
    }
  }
  double* bn2 = G.hv + 2 * (int64_t)ninst * stride;
  double* rss = bn2 + ninst;
  sqnorm(sys, G.b, bn2, 1, nrhs);
  sqnorm(sys, G.r, rss, 1, nrhs);
  std::vector<double> hb(ninst), hr(ninst);
  HM_CUDA(cudaMemcpyAsync(hb.data(), bn2, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaMemcpyAsync(hr.data(), rss, sizeof(double) * ninst, cudaMemcpyDeviceToHost, s));
  {
    ProfScope ps(sys->ctx, PC_VECTOR, Work{0.0, 20.0 * nn});
    launch_permute_out(G.x, d_x, sys->d_perm, n, nrhs, s);
  }
  HM_CUDA(cudaStreamSynchronize(s));
  HM_CUDA(cudaGetLastError());
  if (info) {
    double mx = 0;
    for (int r = 0; r < ninst; ++r) mx = std::max(mx, hb[r] > 0 ? std::sqrt(hr[r] / hb[r]) : 0.0);
    info->iters = refine + 1;
    info->restarts = 0;
    info->relres = mx;
    info->converged = 1;
  }
  return check_device_error(sys, "direct solve");
}

int direct_impl(hm_sys_s* sys, int nrhs, const double* d_b, int refine, double* d_x, hm_solve_info* info) {
  if (sys->precision == HM_PREC_FP64) return direct_t<double>(sys, nrhs, d_b, refine, d_x, info);
  return direct_t<float>(sys, nrhs, d_b, refine, d_x, info);
}

int gmres_impl(hm_sys_s* sys, int nrhs, const double* d_b, double rtol, int max_iters, double* d_x,
               hm_solve_info* info) {
  if (sys->precision == HM_PREC_FP64) return gmres_t<double>(sys, nrhs, d_b, rtol, max_iters, d_x, info);
  return gmres_t<float>(sys, nrhs, d_b, rtol, max_iters, d_x, info);
}

// ------------------------------------------------------------------------------------
// Slot sessions.  Between cycles the columns are independent instances: a slot's b, x
// and r are (re)set without touching the others, and the next cycle's V_0 = r / ||r|| is
// formed per column, so a right-hand side that joins a running session is solved by the
// same iteration as alone (GMRES runs each column on its own Krylov space).
// ------------------------------------------------------------------------------------
int gm_session_begin(hm_sys_s* sys, int nslots) {
  if (sys->nseg != 1) {
    set_last_error("solve sessions serve one mesh per system");
    return HM_ERR_INVALID_ARG;
  }
  const int m = std::max(1, sys->ctx->opts.restart);
  HM_TRY(ensure_workspace(sys, nslots, m));
  auto& G = sys->gm;
  cudaStream_t s = sys->ctx->stream;
  const int64_t nn = (int64_t)sys->n * nslots;
  HM_CUDA(cudaMemsetAsync(G.b, 0, sizeof(double) * nn, s));
  HM_CUDA(cudaMemsetAsync(G.x, 0, sizeof(double) * nn, s));
  HM_CUDA(cudaMemsetAsync(G.r, 0, sizeof(double) * nn, s));
  G.on.assign(nslots, 0);
  G.fresh.assign(nslots, 0);
  G.rtol.assign(nslots, 1e-10);
  G.bnorm_h.assign(nslots, 0.0);
  G.relres.assign(nslots, 0.0);
  G.iters.assign(nslots, 0);
  G.cap.assign(nslots, 0);
  return HM_OK;
}

int gm_session_put(hm_sys_s* sys, int slot, const double* b_host, double rtol, int max_iters) {
  auto& G = sys->gm;
  if (slot < 0 || slot >= (int)G.on.size() || G.on[slot]) return HM_ERR_INVALID_ARG;
  cudaStream_t s = sys->ctx->stream;
  const int n = sys->n;
  double* stage = G.w + (int64_t)slot * n;  // the Arnoldi scratch is free between cycles
  HM_CUDA(cudaMemcpyAsync(stage, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  launch_permute_in(stage, G.b + (int64_t)slot * n, sys->d_perm, n, 1, s);
  HM_CUDA(cudaMemsetAsync(G.x + (int64_t)slot * n, 0, sizeof(double) * n, s));
  HM_CUDA(cudaMemcpyAsync(G.r + (int64_t)slot * n, G.b + (int64_t)slot * n, sizeof(double) * n,
                          cudaMemcpyDeviceToDevice, s));
  G.on[slot] = 1;
  G.fresh[slot] = 1;
  G.rtol[slot] = rtol;
  G.iters[slot] = 0;
  G.cap[slot] = max_iters;
  G.relres[slot] = 1.0;
  HM_CUDA(cudaStreamSynchronize(s));  // the host array may go away after the call
  return HM_OK;
}

template <typename T>
static int session_cycle_t(hm_sys_s* sys, int* its) {
  auto& G = sys->gm;
  cudaStream_t s = sys->ctx->stream;
  const int nslots = G.nrhs, m = G.m, stride = m + 2;
  double* bn2 = G.hv + 2 * (int64_t)nslots * stride;
  double* rss = bn2 + nslots;
  *its = 0;
  bool fresh = false;
  for (int k = 0; k < nslots; ++k) fresh = fresh || G.fresh[k];
  if (fresh) {  // ||b|| of the slots that joined; their squared residual is ||b||^2 (x = 0)
    std::vector<double> hb(nslots), hr(nslots);
    sqnorm(sys, G.b, bn2, 1, nslots);
    HM_CUDA(cudaMemcpyAsync(hb.data(), bn2, sizeof(double) * nslots, cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(hr.data(), rss, sizeof(double) * nslots, cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nslots; ++k)
      if (G.fresh[k]) {
        G.bnorm_h[k] = std::sqrt(hb[k]);
        G.relres[k] = G.bnorm_h[k] > 0 ? 1.0 : 0.0;
        hr[k] = hb[k];
        G.fresh[k] = 0;
      }
    HM_CUDA(cudaMemcpyAsync(G.bnorm, G.bnorm_h.data(), sizeof(double) * nslots, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyAsync(rss, hr.data(), sizeof(double) * nslots, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int> active(nslots, 0);
  double rtol = 1.0;
  int budget = 0;
  bool any = false;
  for (int k = 0; k < nslots; ++k)
    if (G.on[k] && !(G.relres[k] <= G.rtol[k]) && G.iters[k] < G.cap[k]) {  // NaN: runs to its cap
      active[k] = 1;
      any = true;
      rtol = std::min(rtol, G.rtol[k]);
      budget = std::max(budget, G.cap[k] - G.iters[k]);
    }
  if (!any) return HM_OK;
  HM_TRY(gm_cycle<T>(sys, nslots, rtol, budget, active, its));
  std::vector<double> hr(nslots);
  HM_CUDA(cudaMemcpyAsync(hr.data(), rss, sizeof(double) * nslots, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < nslots; ++k)
    if (active[k]) {
      G.iters[k] += *its;
      G.relres[k] = G.bnorm_h[k] > 0 ? std::sqrt(hr[k]) / G.bnorm_h[k] : 0.0;
    }
  return check_device_error(sys, "solve session");
}

int gm_session_cycle(hm_sys_s* sys, int* its) {
  if (sys->precision == HM_PREC_FP64) return session_cycle_t<double>(sys, its);
  return session_cycle_t<float>(sys, its);
}

int gm_session_state(const hm_sys_s* sys, int slot, double* relres, int* iters) {
  const auto& G = sys->gm;
  if (relres) *relres = G.relres[slot];
  if (iters) *iters = G.iters[slot];
  if (G.relres[slot] <= G.rtol[slot]) return 1;
  return G.iters[slot] >= G.cap[slot] ? -1 : 0;
}

int gm_session_take(hm_sys_s* sys, int slot, double* x_host) {
  auto& G = sys->gm;
  if (slot < 0 || slot >= (int)G.on.size() || !G.on[slot]) return HM_ERR_INVALID_ARG;
  cudaStream_t s = sys->ctx->stream;
  const int n = sys->n;
  double* stage = G.w + (int64_t)slot * n;
  launch_permute_out(G.x + (int64_t)slot * n, stage, sys->d_perm, n, 1, s);
  HM_CUDA(cudaMemcpyAsync(x_host, stage, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  G.on[slot] = 0;
  return HM_OK;
}

}  // namespace hm
