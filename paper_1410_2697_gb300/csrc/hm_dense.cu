// hm_dense.cu -- batched dense kernels (FP32/FP64 SIMT) used by factor and apply.
#include <algorithm>

#include "hm_dense.cuh"

namespace hm {

// =====================================================================================
// Batched GEMM: 64 x BN output tiles (BN = 64 or 16), 256 threads; a thread owns rows
// ty + 16 i (i < 4) and columns tx + 16 j (j < BN / 16).  Operand tiles are staged
// through shared memory with the next k-slice prefetched into registers while the
// current one is consumed.  The narrow variant serves products with few columns (one
// right-hand side block of the preconditioner apply).  Each width comes with a shallow
// k-slice (16: few registers, more resident CTAs) and a deep one (64 for the narrow
// tiles, 32 for the wide: fewer memory round trips along k); a batch's variant is its
// GemmBatch::bk, set by the autotuner.
// =====================================================================================
constexpr int BM = kGemmBM;

template <typename T>
__device__ __forceinline__ T load_op(const T* __restrict__ X, int op, int ld, int r, int c,
                                     int nr, int nc) {
  // element (r, c) of op(X), with op(X) of size nr x nc; zero outside
  if (r >= nr || c >= nc) return T(0);
  return op == 0 ? X[(size_t)r + (size_t)c * ld] : X[(size_t)c + (size_t)r * ld];
}

// C = alpha acc + beta C on the valid entries of a thread's NI x NJ outputs (rows
// r0 + 16 i, columns c0 + 16 j).  Every old C value is read before the first store: the
// compiler must assume a store may alias a later load, so interleaved read-modify-writes
// would each wait a full memory round trip.
template <typename T, int NI, int NJ>
__device__ __forceinline__ void store_tile(const GemmTask& t, T* __restrict__ C, const T (&acc)[NI][NJ], int r0,
                                           int c0) {
  const T alpha = (T)t.alpha, beta = (T)t.beta;
  T old[NI][NJ];
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int r = r0 + 16 * i, c = c0 + 16 * j;
      const bool ok = r < t.m && c < t.n && !(t.lower && r < c);
      old[i][j] = (ok && beta != T(0)) ? C[(size_t)r + (size_t)c * t.ldc] : T(0);
    }
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int r = r0 + 16 * i, c = c0 + 16 * j;
      if (r < t.m && c < t.n && !(t.lower && r < c)) {
        const T v = alpha * acc[i][j];
        C[(size_t)r + (size_t)c * t.ldc] = (beta == T(0)) ? v : fma(beta, old[i][j], v);
      }
    }
}

template <typename T, int BN, int BK>
__global__ void __launch_bounds__(256, BK == 16 ? 4 : 3) k_gemm(const GemmTask* __restrict__ tasks,
                                                                const GemmTile* __restrict__ tiles,
                                                                T* __restrict__ split_ws,
                                                                unsigned* __restrict__ split_cnt) {
  constexpr int TN = BN / 16;        // columns per thread
  constexpr int NA = BK * BM / 256;  // A elements loaded per thread
  constexpr int NB = BK * BN / 256;  // B elements loaded per thread
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  const int m0 = (tl.mn >> 16) * BM, n0 = (tl.mn & 0xffff) * BN;
  const T* __restrict__ A = (const T*)t.A;
  const T* __restrict__ B = (const T*)t.B;
  T* __restrict__ C = (T*)t.C;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  // k beyond this tile's part [k0, k1) reads as zero, so a part need not be a whole
  // number of k-slices
  const int kend = tl.k1;
  T ra[NA], rb[NB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + 256 * q;
      int r, p;
      if (t.opA == 0) { r = e % BM; p = e / BM; } else { p = e % BK; r = e / BK; }
      ra[q] = load_op(A, t.opA, t.lda, m0 + r, k0 + p, t.m, kend);
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + 256 * q;
      int c, pb;
      if (t.opB == 0) { pb = e % BK; c = e / BK; } else { c = e % BN; pb = e / BN; }
      rb[q] = load_op(B, t.opB, t.ldb, k0 + pb, n0 + c, kend, t.n);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + 256 * q;
      int r, p;
      if (t.opA == 0) { r = e % BM; p = e / BM; } else { p = e % BK; r = e / BK; }
      As[p][r] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + 256 * q;
      int c, pb;
      if (t.opB == 0) { pb = e % BK; c = e / BK; } else { c = e % BN; pb = e / BN; }
      Bs[pb][c] = rb[q];
    }
  };

  if (tl.k0 < kend) fetch(tl.k0);
  for (int k0 = tl.k0; k0 < kend; k0 += BK) {
    __syncthreads();
    stash();
    __syncthreads();
    if (k0 + BK < kend) fetch(k0 + BK);
#pragma unroll
    for (int p = 0; p < BK; ++p) {
      T a[4], b[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[p][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[p][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  if (tl.slot >= 0) {
    // split k: publish this part, and let the last part to arrive reduce in fixed order
    __shared__ int last;
    T* ws = split_ws + tl.woff;
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        ws[(size_t)tl.part * BM * BN + (ty + 16 * i) + (tx + 16 * j) * BM] = acc[i][j];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(split_cnt + tl.slot, 1u) == (unsigned)(tl.nsplit - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        T v = T(0);
        for (int p = 0; p < tl.nsplit; ++p)
          v += __ldcg(ws + (size_t)p * BM * BN + (ty + 16 * i) + (tx + 16 * j) * BM);
        acc[i][j] = v;
      }
    if (tid == 0) split_cnt[tl.slot] = 0u;  // ready for the next launch
  }
  store_tile<T, 4, TN>(t, C, acc, m0 + ty, n0 + tx);
}

// =====================================================================================
// Pipelined variant: the same 64 x BN tiles and thread layout, with the operand slices
// (32 deep) copied global -> shared by cp.async (4- or 8-byte copies, zero-filled
// outside the operands) kGemmStages slices ahead, so a tile waits on about one memory
// round trip instead of one per slice.  Dynamic shared memory: kGemmStages x
// (32 x (64 + 4) + 32 x (BN + 4)) elements.
// =====================================================================================
constexpr int kGemmStages = 4, kAsyncBK = 32;

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(T) : 0;
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T, int BN>
__host__ __device__ constexpr int gemm_async_stage_elems() { return kAsyncBK * (BM + 4) + kAsyncBK * (BN + 4); }

template <typename T, int BN>
__global__ void __launch_bounds__(256, BN == 16 ? 4 : 3) k_gemm_async(const GemmTask* __restrict__ tasks,
                                                    const GemmTile* __restrict__ tiles, T* __restrict__ split_ws,
                                                    unsigned* __restrict__ split_cnt) {
  constexpr int BK = kAsyncBK, TN = BN / 16, NA = BK * BM / 256, NB = BK * BN / 256;
  constexpr int SE = gemm_async_stage_elems<T, BN>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  const int m0 = (tl.mn >> 16) * BM, n0 = (tl.mn & 0xffff) * BN;
  const T* __restrict__ A = (const T*)t.A;
  const T* __restrict__ B = (const T*)t.B;
  T* __restrict__ C = (T*)t.C;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int kbeg = tl.k0, kend = tl.k1;
  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  auto issue = [&](int kt) {
    T* As = smem + (kt % kGemmStages) * SE;
    T* Bs = As + BK * (BM + 4);
    const int k0 = kbeg + kt * BK;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + 256 * q;
      int r, pp;
      if (t.opA == 0) { r = e % BM; pp = e / BM; } else { pp = e % BK; r = e / BK; }
      const int gr = m0 + r, gk = k0 + pp;
      const bool ok = gr < t.m && gk < kend;
      const T* src = ok ? (t.opA == 0 ? A + (size_t)gr + (size_t)gk * t.lda : A + (size_t)gk + (size_t)gr * t.lda) : A;
      cp_async_elem(As + pp * (BM + 4) + r, src, ok);
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + 256 * q;
      int c, pb;
      if (t.opB == 0) { pb = e % BK; c = e / BK; } else { c = e % BN; pb = e / BN; }
      const int gc = n0 + c, gk = k0 + pb;
      const bool ok = gc < t.n && gk < kend;
      const T* src = ok ? (t.opB == 0 ? B + (size_t)gk + (size_t)gc * t.ldb : B + (size_t)gc + (size_t)gk * t.ldb) : B;
      cp_async_elem(Bs + pb * (BN + 4) + c, src, ok);
    }
  };
  T acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
#pragma unroll
  for (int s = 0; s < kGemmStages - 1; ++s) {
    if (s < nk) issue(s);
    cp_async_commit();
  }
  for (int kt = 0; kt < nk; ++kt) {
    cp_async_wait<kGemmStages - 2>();
    __syncthreads();  // slice kt visible to all; slice kt - 1's buffer free
    if (kt + kGemmStages - 1 < nk) issue(kt + kGemmStages - 1);
    cp_async_commit();
    const T* As = smem + (kt % kGemmStages) * SE;
    const T* Bs = As + BK * (BM + 4);
#pragma unroll
    for (int p = 0; p < BK; ++p) {
      T a[4], b[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[p * (BM + 4) + ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[p * (BN + 4) + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  cp_async_wait<0>();
  if (tl.slot >= 0) {
    __shared__ int last;
    T* ws = split_ws + tl.woff;
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        ws[(size_t)tl.part * BM * BN + (ty + 16 * i) + (tx + 16 * j) * BM] = acc[i][j];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(split_cnt + tl.slot, 1u) == (unsigned)(tl.nsplit - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        T v = T(0);
        for (int p = 0; p < tl.nsplit; ++p)
          v += __ldcg(ws + (size_t)p * BM * BN + (ty + 16 * i) + (tx + 16 * j) * BM);
        acc[i][j] = v;
      }
    if (tid == 0) split_cnt[tl.slot] = 0u;
  }
  store_tile<T, 4, TN>(t, C, acc, m0 + ty, n0 + tx);
}

int gemm_async_setup(int max_smem) {
  (void)max_smem;
  HM_CUDA(cudaFuncSetAttribute(k_gemm_async<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kGemmStages * gemm_async_stage_elems<float, 16>() * sizeof(float))));
  HM_CUDA(cudaFuncSetAttribute(k_gemm_async<float, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kGemmStages * gemm_async_stage_elems<float, 64>() * sizeof(float))));
  HM_CUDA(cudaFuncSetAttribute(k_gemm_async<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kGemmStages * gemm_async_stage_elems<double, 16>() * sizeof(double))));
  HM_CUDA(cudaFuncSetAttribute(k_gemm_async<double, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kGemmStages * gemm_async_stage_elems<double, 64>() * sizeof(double))));
  return HM_OK;
}

// =====================================================================================
// Large-tile variant (FP32): 128 x 128 output tiles, 256 threads, each thread an 8 x 8
// register block (rows ty*4 + {0..3, 64..67}, columns tx*4 + {0..3, 64..67}), so one
// k step reads 2 + 2 float4 from shared memory for 64 FMAs.  k-slices of 8, staged
// k-major in double-buffered shared memory with the next slice prefetched into
// registers.  Same tile/split contract as k_gemm with 128 x 128 tiles; each output adds
// its products in increasing k, as the other variants do.
// =====================================================================================
constexpr int kBigBM = 128, kBigBK = 8;

__global__ void __launch_bounds__(256, 2) k_gemm_big(const GemmTask* __restrict__ tasks,
                                                     const GemmTile* __restrict__ tiles,
                                                     float* __restrict__ split_ws, unsigned* __restrict__ split_cnt) {
  constexpr int BM = kBigBM, BN = kBigBM, BK = kBigBK;
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  const int m0 = (tl.mn >> 16) * BM, n0 = (tl.mn & 0xffff) * BN;
  const float* __restrict__ A = (const float*)t.A;
  const float* __restrict__ B = (const float*)t.B;
  float* __restrict__ C = (float*)t.C;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int kend = tl.k1;
  float ra[4], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int r, p;
      if (t.opA == 0) { r = e % BM; p = e / BM; } else { p = e % BK; r = e / BK; }
      const int gr = m0 + r, gk = k0 + p;
      ra[q] = (gr < t.m && gk < kend) ? (t.opA == 0 ? A[(size_t)gr + (size_t)gk * t.lda]
                                                     : A[(size_t)gk + (size_t)gr * t.lda]) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int c, p;
      if (t.opB == 0) { p = e % BK; c = e / BK; } else { c = e % BN; p = e / BN; }
      const int gc = n0 + c, gk = k0 + p;
      rb[q] = (gc < t.n && gk < kend) ? (t.opB == 0 ? B[(size_t)gk + (size_t)gc * t.ldb]
                                                     : B[(size_t)gc + (size_t)gk * t.ldb]) : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int r, p;
      if (t.opA == 0) { r = e % BM; p = e / BM; } else { p = e % BK; r = e / BK; }
      As[buf][p][r] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int c, p;
      if (t.opB == 0) { p = e % BK; c = e / BK; } else { c = e % BN; p = e / BN; }
      Bs[buf][p][c] = rb[q];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  int buf = 0;
  if (tl.k0 < kend) {
    fetch(tl.k0);
    stash(0);
  }
  __syncthreads();
  for (int k0 = tl.k0; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int p = 0; p < BK; ++p) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][p][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][p][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][p][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][p][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  auto row_of = [&](int i) { return (i < 4 ? 0 : 64) + ty * 4 + (i & 3); };
  auto col_of = [&](int j) { return (j < 4 ? 0 : 64) + tx * 4 + (j & 3); };
  if (tl.slot >= 0) {
    __shared__ int last;
    float* ws = split_ws + tl.woff;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) ws[(size_t)tl.part * BM * BN + row_of(i) + col_of(j) * BM] = acc[i][j];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(split_cnt + tl.slot, 1u) == (unsigned)(tl.nsplit - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float v = 0.f;
        for (int q = 0; q < tl.nsplit; ++q) v += __ldcg(ws + (size_t)q * BM * BN + row_of(i) + col_of(j) * BM);
        acc[i][j] = v;
      }
    if (tid == 0) split_cnt[tl.slot] = 0u;
  }
  // C = alpha acc + beta C, two columns at a time with their old values read before the
  // first store (see store_tile)
  const float alpha = (float)t.alpha, beta = (float)t.beta;
#pragma unroll
  for (int j0 = 0; j0 < 8; j0 += 2) {
    float old[2][8];
#pragma unroll
    for (int jj = 0; jj < 2; ++jj)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = m0 + row_of(i), c = n0 + col_of(j0 + jj);
        const bool ok = r < t.m && c < t.n && !(t.lower && r < c);
        old[jj][i] = (ok && beta != 0.f) ? C[(size_t)r + (size_t)c * t.ldc] : 0.f;
      }
#pragma unroll
    for (int jj = 0; jj < 2; ++jj)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = m0 + row_of(i), c = n0 + col_of(j0 + jj);
        if (r < t.m && c < t.n && !(t.lower && r < c)) {
          const float v = alpha * acc[i][j0 + jj];
          C[(size_t)r + (size_t)c * t.ldc] = (beta == 0.f) ? v : fmaf(beta, old[jj][i], v);
        }
      }
  }
}

void launch_gemm_big(const GemmTask* tasks, const GemmTile* tiles, int ntiles, float* split_ws,
                     unsigned* split_cnt, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_gemm_big<<<ntiles, 256, 0, s>>>(tasks, tiles, split_ws, split_cnt);
}

int gemm_bn_for(const std::vector<GemmTask>& t) {
  int nmax = 0;
  for (const auto& x : t) nmax = std::max(nmax, x.n);
  return nmax <= 16 ? 16 : 64;
}

int gemm_tile_count(const GemmTask& t, int bm, int bn) {
  if (t.m <= 0 || t.n <= 0) return 0;
  const int tm = (t.m + bm - 1) / bm, tn = (t.n + bn - 1) / bn;
  int c = 0;
  for (int a = 0; a < tm; ++a)
    for (int b = 0; b < tn; ++b) c += (t.lower && (a + 1) * bm - 1 < b * bn) ? 0 : 1;
  return c;
}

void gemm_tiles_for(const GemmTask& t, int task_index, int bm, int bn, int nsplit, std::vector<GemmTile>* out,
                    int* slots, int64_t* ws) {
  if (t.m <= 0 || t.n <= 0) return;
  const int tm = (t.m + bm - 1) / bm, tn = (t.n + bn - 1) / bn;
  // k chunks are whole multiples of 16 (every kernel masks k beyond its part's end)
  const int kc = nsplit > 1 ? ((t.k + nsplit - 1) / nsplit + 15) / 16 * 16 : t.k;
  const int parts = nsplit > 1 ? (t.k + kc - 1) / kc : 1;
  for (int a = 0; a < tm; ++a)
    for (int b = 0; b < tn; ++b) {
      if (t.lower && (a + 1) * bm - 1 < b * bn) continue;  // tile strictly above diagonal
      if (parts <= 1) {
        out->push_back(GemmTile{task_index, (a << 16) | b, 0, t.k, -1, 0, 1, 0, 0});
        continue;
      }
      const int slot = (*slots)++;
      const int64_t woff = *ws;
      *ws += (int64_t)parts * bm * bn;
      for (int p = 0; p < parts; ++p)
        out->push_back(GemmTile{task_index, (a << 16) | b, p * kc, std::min(t.k, (p + 1) * kc), slot, p,
                                parts, 0, woff});
    }
}

template <typename T>
void launch_gemm(const GemmTask* tasks, const GemmTile* tiles, int ntiles, int bn, int deep, T* split_ws,
                 unsigned* split_cnt, cudaStream_t s) {
  if (ntiles <= 0) return;
  if (deep == 2) {
    if (bn == 16)
      k_gemm_async<T, 16><<<ntiles, 256, kGemmStages * gemm_async_stage_elems<T, 16>() * sizeof(T), s>>>(
          tasks, tiles, split_ws, split_cnt);
    else
      k_gemm_async<T, 64><<<ntiles, 256, kGemmStages * gemm_async_stage_elems<T, 64>() * sizeof(T), s>>>(
          tasks, tiles, split_ws, split_cnt);
    return;
  }
  if (bn == 16) {
    if (deep) k_gemm<T, 16, 64><<<ntiles, 256, 0, s>>>(tasks, tiles, split_ws, split_cnt);
    else k_gemm<T, 16, 16><<<ntiles, 256, 0, s>>>(tasks, tiles, split_ws, split_cnt);
  } else {
    if (deep) k_gemm<T, 64, 32><<<ntiles, 256, 0, s>>>(tasks, tiles, split_ws, split_cnt);
    else k_gemm<T, 64, 16><<<ntiles, 256, 0, s>>>(tasks, tiles, split_ws, split_cnt);
  }
}

template void launch_gemm<float>(const GemmTask*, const GemmTile*, int, int, int, float*, unsigned*,
                                 cudaStream_t);
template void launch_gemm<double>(const GemmTask*, const GemmTile*, int, int, int, double*, unsigned*,
                                  cudaStream_t);

}  // namespace hm
