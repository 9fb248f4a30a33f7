// hm_dense_tc.cu -- batched GEMM on the 5th-generation tensor cores (tcgen05), BF16
// operands with FP32 accumulation in tensor memory, for the randomized range finder's
// sampling products Y = B Omega and Z = B^T Q (the BF16 range-finder precision mode).
//
// One CTA (256 threads) per 128 x 64 output tile (or per k part of a split tile, with
// the same fixed-order reduction as the SIMT GEMM).  Per 64-deep k slice the threads
// read the FP32 operands from HBM (coalesced for either transpose), round them to BF16
// and store them in shared memory in the K-major core-matrix layout (8 rows x 16 bytes
// per 128-byte core matrix; K-adjacent core matrices 16 * rows bytes apart, row-group
// adjacent ones 128 bytes apart).  One elected thread issues four
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 64, K = 16) on the slice and commits
// them to the slice's mbarrier; the next slice is staged into the other buffer while the
// tensor core runs.  The accumulator (128 lanes x 64 FP32 columns of tensor memory) is
// read back with tcgen05.ld (warp w: lanes 32 (w % 4) .., columns 32 (w / 4) ..) for the
// alpha / beta epilogue.  Every mbarrier wait is bounded (wait_limit polls); a wait that
// runs out sets the device error word (HM_ERR_DEVICE_TIMEOUT) and skips the rest of the
// tile, but first waits, with the default limit, for the last MMA group it committed
// (tcgen05.commit tracks every MMA issued before it), so the tensor memory is freed only
// once no MMA can still write it.
//
// The same kernel in its second mode computes FP32 products at FP32 accuracy on the
// tensor cores (kind::tf32): every operand x is split while it is staged into
// hi = x rounded to TF32 (10 mantissa bits, round to nearest) and lo = x - hi (exact in
// FP32), and each k slice runs three MMAs per 8-deep step, hi*hi + hi*lo + lo*hi, into
// the same FP32 accumulator (the lo*lo term is below FP32 rounding).  32-deep slices of
// FP32 take the same 128 bytes per row as the 64-deep BF16 slices, so the core-matrix
// layout and descriptors are shared; the stage holds four buffers (A and B, hi and lo).
#include <cuda_bf16.h>

#include "hm_dense.cuh"

namespace hm {

namespace {

constexpr int TM = 128, TN = 64;                           // output tile
constexpr int kSliceBytes = 128;                             // bytes of one row of a k slice
constexpr int kStageA = TM * kSliceBytes, kStageB = TN * kSliceBytes;  // one operand copy
constexpr int kTcSmem = 2 * (kStageA + kStageB);             // BF16: double-buffered A, B
constexpr int kTf32Smem = 2 * 2 * (kStageA + kStageB);       // TF32x3: A, B in hi and lo, double-buffered
constexpr int kWaitLimit = 1 << 22;                          // default mbarrier polls before giving up
enum TcMode { kModeBf16 = 0, kModeTf32x3 = 1 };
// k elements per slice (128 bytes per row) and per MMA instruction (32 bytes)
template <int MODE> struct TcShape;
template <> struct TcShape<kModeBf16> { static constexpr int TK = 64, KI = 16; };
template <> struct TcShape<kModeTf32x3> { static constexpr int TK = 32, KI = 8; };


// Shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (row-group direction) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptors: FP32 accumulator (bits 4-5 = 1), A and B K-major, N >> 3 at
// bit 17, M >> 4 at bit 24; operand types at bits 7-9 and 10-12: kind::f16 with BF16
// (1), kind::tf32 with TF32 (2).
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                                ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                                ((uint32_t)(TM >> 4) << 24);

// byte offset of element (row, kk) of a K-major slice with `rows` rows: core matrices of
// 8 rows x 16 bytes (8 BF16 or 4 FP32 elements along k), K-adjacent ones 16 * rows bytes
// apart, row-group adjacent ones 128 bytes apart
template <int MODE>
__device__ __forceinline__ uint32_t kmaj(int row, int kk, int rows) {
  if (MODE == kModeBf16)
    return (uint32_t)((kk >> 3) * rows * 16 + (row >> 3) * 128 + (row & 7) * 16 + (kk & 7) * 2);
  return (uint32_t)((kk >> 2) * rows * 16 + (row >> 3) * 128 + (row & 7) * 16 + (kk & 3) * 4);
}

// x rounded to TF32 (round to nearest, ties away from zero): low 13 bits of the result zero
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}


// Stages rows row0 .. row0+R-1 and k indices k0 .. k0+TK-1 of an operand (FP32 in
// memory, zero outside rows < nrows and k < kend) into a K-major slice of R rows: as BF16
// (BF16 mode), or as its TF32 split, hi into sl and lo into sl_lo (TF32x3 mode).
// rows_fast: element (row, k) sits at X[row + k ld] (consecutive threads take consecutive
// rows), else at X[k + row ld] (consecutive threads take consecutive k).  A thread issues
// all its loads before converting and storing, so they are in flight together.
template <int MODE, int R>
__device__ __forceinline__ void stage_slice(unsigned char* __restrict__ sl, unsigned char* __restrict__ sl_lo,
                                            const float* __restrict__ X, bool rows_fast, int ld, int row0,
                                            int nrows, int k0, int kend, int tid) {
  constexpr int TK = TcShape<MODE>::TK;
  constexpr int PER = R * TK / 256;
  float v[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = tid + 256 * q;
    const int r = rows_fast ? e % R : e / TK, c = rows_fast ? e / R : e % TK;
    const int gr = row0 + r, gk = k0 + c;
    v[q] = (gr < nrows && gk < kend) ? (rows_fast ? X[(size_t)gr + (size_t)gk * ld] : X[(size_t)gk + (size_t)gr * ld])
                                     : 0.f;
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = tid + 256 * q;
    const int r = rows_fast ? e % R : e / TK, c = rows_fast ? e / R : e % TK;
    const uint32_t off = kmaj<MODE>(r, c, R);
    if (MODE == kModeBf16) {
      *(__nv_bfloat16*)(sl + off) = __float2bfloat16(v[q]);
    } else {
      const float hi = tf32_hi(v[q]);
      *(float*)(sl + off) = hi;
      *(float*)(sl_lo + off) = v[q] - hi;
    }
  }
}

}  // namespace

template <int MODE>
__global__ void __launch_bounds__(256) k_gemm_tc(const GemmTask* __restrict__ tasks,
                                                 const GemmTile* __restrict__ tiles, float* __restrict__ split_ws,
                                                 unsigned* __restrict__ split_cnt, int* __restrict__ err,
                                                 int wait_limit, int inject_timeout) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t mbar_never;  // fault injection: nothing ever arrives on it
  __shared__ uint32_t tmem_slot;
  __shared__ int s_ok, s_last, s_committed;
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  const int m0 = (tl.mn >> 16) * TM, n0 = (tl.mn & 0xffff) * TN;
  const float* __restrict__ A = (const float*)t.A;
  const float* __restrict__ B = (const float*)t.B;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar_never)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
    s_committed = 0;  // k slices whose MMAs have been committed
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(TN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  constexpr int TK = TcShape<MODE>::TK, KI = TcShape<MODE>::KI;
  constexpr int kStage = MODE == kModeBf16 ? kStageA + kStageB : 2 * (kStageA + kStageB);
  const int nk = (tl.k1 - tl.k0 + TK - 1) / TK;
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (kt >= 2) {  // the MMAs that read this buffer two slices ago must be done
      if (tid == 0 && !mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((kt >> 1) - 1) & 1), wait_limit)) s_ok = 0;
      __syncthreads();
      if (!s_ok) break;
    }
    unsigned char* sA = smem + s * kStage;
    unsigned char* sB = sA + kStageA;
    unsigned char* sAlo = sB + kStageB;  // TF32x3 mode only
    unsigned char* sBlo = sAlo + kStageA;
    const int kb = tl.k0 + kt * TK;
    // A slice: op(A)[m0 .., kb ..]; B slice as N x K (row n = column n of op(B))
    stage_slice<MODE, TM>(sA, sAlo, A, t.opA == 0, t.lda, m0, t.m, kb, tl.k1, tid);
    stage_slice<MODE, TN>(sB, sBlo, B, t.opB != 0, t.ldb, n0, t.n, kb, tl.k1, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // one MMA instruction per KI-deep step: 32 bytes = two core matrices along k
      constexpr int nterm = MODE == kModeBf16 ? 1 : 3;  // hi*hi, hi*lo, lo*hi
#pragma unroll
      for (int j = 0; j < TK / KI; ++j)
#pragma unroll
        for (int term = 0; term < nterm; ++term) {
          const uint32_t a0 = smem_u32(term == 2 ? sAlo : sA), b0 = smem_u32(term == 1 ? sBlo : sB);
          const uint64_t da = umma_desc(a0 + (uint32_t)(2 * j * TM * 16), TM * 16, 128);
          const uint64_t db = umma_desc(b0 + (uint32_t)(2 * j * TN * 16), TN * 16, 128);
          const uint32_t acc = (kt > 0 || j > 0 || term > 0) ? 1u : 0u;
          if (MODE == kModeBf16)
            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                         :: "r"(tmem), "l"(da), "l"(db), "r"(kIdescBf16), "r"(acc)
                         : "memory");
          else
            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                         :: "r"(tmem), "l"(da), "l"(db), "r"(kIdescTf32), "r"(acc)
                         : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mbar[s])) : "memory");
      s_committed = kt + 1;
    }
  }
  if (nk > 0 && s_ok) {
    const int s = (nk - 1) & 1;
    if (tid == 0 && !mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((nk - 1) >> 1) & 1), wait_limit)) s_ok = 0;
  }
  // fault injection: one more bounded wait, on a barrier that no MMA commit arrives on,
  // so it runs out (right after the last commit, with MMAs possibly still in flight)
  if (inject_timeout && tid == 0 && s_ok && !mbar_wait(smem_u32(&mbar_never), 0u, wait_limit)) s_ok = 0;
  __syncthreads();
  const bool ok = s_ok != 0;
  if (!ok && tid == 0) {
    raise_error(err, HM_ERR_DEVICE_TIMEOUT, 20, blockIdx.x);
    // Drain before the tensor memory is released: slice c = s_committed - 1 was the last
    // one committed, to buffer c & 1, as that buffer's (c >> 1)-th use; its commit
    // completes once every MMA issued before it has.  The default limit applies here.
    const int c = s_committed - 1;
    if (c >= 0) (void)mbar_wait(smem_u32(&mbar[c & 1]), (uint32_t)((c >> 1) & 1), kWaitLimit);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // accumulator -> registers: row = lane quarter of the warp, 32 columns per warp half
  const int row = 32 * (warp & 3) + lane, c0 = 32 * (warp >> 2);
  float acc[32];
  if (ok && nk > 0) {
    uint32_t v[32];
    const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                   "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                   "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                   "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = __uint_as_float(v[j]);
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TN) : "memory");
  if (!ok) return;
  if (tl.slot >= 0) {  // split k: same fixed-order reduction as the SIMT GEMM
    float* ws = split_ws + tl.woff;
#pragma unroll
    for (int j = 0; j < 32; ++j) ws[(size_t)tl.part * TM * TN + row + (size_t)(c0 + j) * TM] = acc[j];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(split_cnt + tl.slot, 1u) == (unsigned)(tl.nsplit - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float v = 0.f;
      for (int p = 0; p < tl.nsplit; ++p) v += __ldcg(ws + (size_t)p * TM * TN + row + (size_t)(c0 + j) * TM);
      acc[j] = v;
    }
    if (tid == 0) split_cnt[tl.slot] = 0u;
  }
  float* C = (float*)t.C;
  const float alpha = (float)t.alpha, beta = (float)t.beta;
  const int r = m0 + row;
  if (r >= t.m) return;
  // eight columns at a time, their old values read before the first store (a store may
  // alias a later load as far as the compiler knows)
#pragma unroll
  for (int j0 = 0; j0 < 32; j0 += 8) {
    float old[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = n0 + c0 + j0 + j;
      const bool ok = c < t.n && !(t.lower && r < c);
      old[j] = (ok && beta != 0.f) ? C[(size_t)r + (size_t)c * t.ldc] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = n0 + c0 + j0 + j;
      if (c >= t.n || (t.lower && r < c)) continue;
      const float v = alpha * acc[j0 + j];
      C[(size_t)r + (size_t)c * t.ldc] = (beta == 0.f) ? v : fmaf(beta, old[j], v);
    }
  }
}

void launch_gemm_tc(const GemmTask* tasks, const GemmTile* tiles, int ntiles, float* split_ws,
                    unsigned* split_cnt, int* err, int wait_limit, int inject_timeout, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_gemm_tc<kModeBf16><<<ntiles, 256, kTcSmem, s>>>(tasks, tiles, split_ws, split_cnt, err,
                                                     wait_limit > 0 ? wait_limit : kWaitLimit, inject_timeout);
}

void launch_gemm_tf32x3(const GemmTask* tasks, const GemmTile* tiles, int ntiles, float* split_ws,
                        unsigned* split_cnt, int* err, int wait_limit, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_gemm_tc<kModeTf32x3><<<ntiles, 256, kTf32Smem, s>>>(tasks, tiles, split_ws, split_cnt, err,
                                                         wait_limit > 0 ? wait_limit : kWaitLimit, 0);
}

int dense_tc_setup(int max_smem) {
  (void)max_smem;
  HM_CUDA(cudaFuncSetAttribute(k_gemm_tc<kModeBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
  HM_CUDA(cudaFuncSetAttribute(k_gemm_tc<kModeTf32x3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTf32Smem));
  return HM_OK;
}

}  // namespace hm
