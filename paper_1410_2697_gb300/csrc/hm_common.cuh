// hm_common.cuh -- shared device/host helpers of the HODLR multifrontal library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/hodlr_mf.h"

namespace hm {

// ------------------------------------------------------------------------------------
// Host error reporting: the last failure message of the calling thread.
// ------------------------------------------------------------------------------------
void set_last_error(const std::string& msg);
// Host-side phase trace (environment HM_TRACE_HOST=1): prints to stderr the host wall
// time since the previous mark of the same thread.  Off by default.
void host_mark(const char* what);

#define HM_CUDA(call)                                                               \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::hm::set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_) +     \
                           " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
      return HM_ERR_CUDA;                                                           \
    }                                                                               \
  } while (0)

#define HM_TRY(expr)                 \
  do {                               \
    int s_ = (expr);                 \
    if (s_ != HM_OK) return s_;      \
  } while (0)

// ------------------------------------------------------------------------------------
// Device error word: err[0] = first status code raised, err[1], err[2] = detail.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void raise_error(int* err, int code, int a = 0, int b = 0) {
  if (atomicCAS(err, 0, code) == 0) {
    err[1] = a;
    err[2] = b;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// 1/x correctly rounded (the value of the IEEE division 1/x) by the reciprocal intrinsic.
__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_rn(double x) { return __drcp_rn(x); }

// Block-wide sum in fixed order (deterministic). `red` holds >= 32 entries.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = T(0);
  if (wid == 0) {
    s = lane < nw ? red[lane] : T(0);
    s = warp_sum(s);
    if (lane == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published definition:
// ten rounds of (hi0,lo0)=mulhilo(M0,c0), (hi1,lo1)=mulhilo(M1,c2),
// c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0); key += (W0, W1) between rounds.
// ------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t p0 = (uint64_t)M0 * c[0];
    const uint64_t p1 = (uint64_t)M1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Sketch entry (i, c) of block `blk`: ((w >> 8) - 2^23) / 2^23 with w = Philox word 0,
// a 24-bit uniform grid on [-1, 1), exact in FP32 and FP64.
__host__ __device__ __forceinline__ float sketch_entry(uint32_t i, uint32_t col, uint64_t blk,
                                                      uint64_t seed) {
  uint32_t c[4] = {i, col, (uint32_t)blk, (uint32_t)(blk >> 32)};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return (float)((int)(c[0] >> 8) - 8388608) * (1.0f / 8388608.0f);
}

// 64-bit id of a compressed block: kind 0 = off-diagonal block (level, node) of the
// pivot block's HODLR tree, kind 1 = the coupling block F_fp.
__host__ __device__ __forceinline__ uint64_t block_id(int front, int kind, int level, int node) {
  return ((uint64_t)front << 24) | ((uint64_t)kind << 20) | ((uint64_t)level << 16) |
         (uint64_t)node;
}

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Packed dense-front factor: [F_pp^-1 | K^T] (np x nhat, ld np) then K (nu x np, ld nu),
// each part starting on a 16-byte boundary (whole 16-byte units for vector or bulk copies).
__host__ __device__ __forceinline__ int64_t packed_k_offset(int np, int nhat, int es) {
  const int64_t a = 16 / es;
  return ((int64_t)np * nhat + a - 1) / a * a;
}
__host__ __device__ __forceinline__ int64_t packed_size(int np, int nhat, int es) {
  const int64_t a = 16 / es;
  return packed_k_offset(np, nhat, es) + ((int64_t)(nhat - np) * np + a - 1) / a * a;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Waits for the phase of parity `parity` of the mbarrier to complete, `limit` polls at
// most: the first poll is mbarrier.test_wait (it never suspends the thread), the later
// ones mbarrier.try_wait (which may suspend it for a while).  Returns false if the phase
// did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t ok;
    if (it == 0)
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(bar), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(bar), "r"(parity)
          : "memory");
    if (ok) return true;
  }
  return false;
}

#endif

// Opt a kernel into the largest dynamic shared memory the device allows per block
// (the per-block opt-in limit minus the kernel's static shared memory).
template <typename F>
inline cudaError_t allow_max_dyn_smem(F* func, int max_smem) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, func);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_smem - (int)a.sharedSizeBytes);
}

}  // namespace hm
