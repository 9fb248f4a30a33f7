// hm_dense_comp.cu -- kernels of the randomized low-rank compression (the randomized
// alternative to BDLR that Section 2.2 of the paper cites): sketch generation,
// Householder QR with explicit Q, and the small SVD by one-sided Jacobi.
#include "hm_dense.cuh"

namespace hm {

// =====================================================================================
// Sketch Omega[i, c] from Philox4x32-10 (counter (i, c, blk), key seed): 24-bit uniform.
// =====================================================================================
template <typename T>
__global__ void k_omega(const OmegaTask* __restrict__ tasks, uint64_t seed) {
  const OmegaTask t = tasks[blockIdx.y];
  T* out = (T*)t.out;
  const int total = t.rows * t.cols;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e % t.rows, c = e / t.rows;
    out[(size_t)i + (size_t)c * t.ld] = (T)sketch_entry((uint32_t)i, (uint32_t)c, t.blk, seed);
  }
}

template <typename T>
void launch_omega(const OmegaTask* tasks, int ntasks, uint64_t seed, cudaStream_t s) {
  if (ntasks <= 0) return;
  dim3 grid(32, ntasks);
  k_omega<T><<<grid, 256, 0, s>>>(tasks, seed);
}

// =====================================================================================
// Householder QR of a tall m x k panel (k <= m), one CTA per panel, in global memory.
// Reflector j in the scale-safe form: beta = -sign(x0) ||x||, tau = (beta - x0) / beta in
// [1, 2], v = [1; x_tail / (x0 - beta)] with |v_i| <= 1, H_j = I - tau v v^T; a column
// whose tail is exactly zero is left alone (tau = 0).  No quantity is divided by a sum of
// squares, so columns that have shrunk to rounding level (rank-deficient sketches) cannot
// overflow in FP32.  R (upper k x k) is copied out if requested, then Q is formed in place
// by backward accumulation Q = H_0 (H_1 (... H_{k-1} [I; 0])).
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) k_qr(const QrTask* __restrict__ tasks) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T red[32];
  const QrTask t = tasks[blockIdx.x];
  const int m = t.m, k = t.k, ld = t.ld;
  T* tau = reinterpret_cast<T*>(smem_raw);
  T* Y = (T*)t.Y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    T* yj = Y + (size_t)j * ld;
    T s = T(0);
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) s += yj[i] * yj[i];
    s = block_sum(s, red);
    const T x0 = yj[j];
    T tj = T(0), beta = x0, scale = T(1);
    if (s > T(0)) {
      const T nrm = sqrt(x0 * x0 + s);
      beta = x0 >= T(0) ? -nrm : nrm;
      tj = (beta - x0) / beta;
      scale = T(1) / (x0 - beta);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) yj[i] *= scale;
    if (threadIdx.x == 0) {
      yj[j] = beta;
      tau[j] = tj;
    }
    __syncthreads();
    if (tj != T(0)) {
      for (int c = j + 1 + wid; c < k; c += nw) {
        T* yc = Y + (size_t)c * ld;
        T w = T(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += yj[i] * yc[i];
        w = warp_sum(w) + yc[j];
        const T f = tj * w;
        __syncwarp();
        if (lane == 0) yc[j] -= f;
        for (int i = j + 1 + lane; i < m; i += 32) yc[i] -= f * yj[i];
      }
    }
    __syncthreads();
  }
  if (t.R) {
    T* R = (T*)t.R;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int i = e % k, c = e / k;
      R[i + (size_t)c * k] = (i <= c) ? Y[(size_t)i + (size_t)c * ld] : T(0);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, c = e / k;
    if (i < c) Y[(size_t)i + (size_t)c * ld] = T(0);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const T tj = tau[j];
    T* yj = Y + (size_t)j * ld;
    for (int c = j + 1 + wid; c < k; c += nw) {
      T* yc = Y + (size_t)c * ld;
      T w = T(0);
      for (int i = j + 1 + lane; i < m; i += 32) w += yj[i] * yc[i];
      w = warp_sum(w);  // Q[j, c] is still zero here
      const T f = tj * w;
      if (lane == 0) yc[j] = -f;
      for (int i = j + 1 + lane; i < m; i += 32) yc[i] -= f * yj[i];
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) yj[i] *= -tj;
    if (threadIdx.x == 0) yj[j] = T(1) - tj;
    __syncthreads();
  }
}

// =====================================================================================
// Blocked Householder QR of a tall m x k panel (k <= m), one CTA per panel, in global
// memory: panels of kQrNB columns are factored column by column (the updates stay inside
// the panel), then their product H_p0 ... H_p0+nb-1 = I - V T V^T (compact WY form, T upper
// triangular, built from V^T V) is applied to the trailing columns in one pass
// (a -= V T^T V^T a).  Q is formed backwards panel by panel from [I; 0]: trailing
// columns get (I - V T V^T) q, the panel's own columns e_j - V T V^T e_j.  Same
// scale-safe reflectors as the unblocked kernel.  V of the current panel is staged in
// shared memory (m x nb); T of every panel is kept for the Q pass.
// =====================================================================================
constexpr int kQrNB = 8;

template <typename T>
__device__ __forceinline__ T warp_sum_all(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reflector of column j (rows j.. of a, global): tail scaled in place, a[j] = beta.
// Returns tau; every thread of warp 0 calls it.
template <typename T>
__device__ __forceinline__ T make_reflector_warp(T* __restrict__ aj, int j, int m) {
  const int lane = threadIdx.x & 31;
  T s = T(0);
  for (int i = j + 1 + lane; i < m; i += 32) s += aj[i] * aj[i];
  s = warp_sum_all(s);
  const T x0 = aj[j];
  T tj = T(0), beta = x0, scale = T(1);
  if (s > T(0)) {
    const T nrm = sqrt(x0 * x0 + s);
    beta = x0 >= T(0) ? -nrm : nrm;
    tj = (beta - x0) / beta;
    scale = T(1) / (x0 - beta);
  }
  for (int i = j + 1 + lane; i < m; i += 32) aj[i] *= scale;
  __syncwarp();
  if (lane == 0) aj[j] = beta;
  return tj;
}

template <typename T>
__global__ void __launch_bounds__(512) k_qr_blocked(const QrTask* __restrict__ tasks) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T tau[256];
  __shared__ T Tall[256 / kQrNB][kQrNB][kQrNB];  // T of every panel (upper triangular)
  __shared__ T G[kQrNB][kQrNB];
  const QrTask t = tasks[blockIdx.x];
  const int m = t.m, k = t.k, ld = t.ld;
  T* Y = (T*)t.Y;
  T* Vs = reinterpret_cast<T*>(smem_raw);  // (m - p0) x nb of the current panel, ld m
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int npanels = (k + kQrNB - 1) / kQrNB;
  for (int pi = 0; pi < npanels; ++pi) {
    const int p0 = pi * kQrNB, pw = min(kQrNB, k - p0), mv = m - p0;
    // --- panel columns (rows p0..) into shared memory, factored there: reflector j by
    //     warp 0, updates of the panel's later columns by one warp each; then written back
    for (int e = threadIdx.x; e < mv * pw; e += blockDim.x) {
      const int i = e % mv, c = e / mv;
      Vs[i + (size_t)c * mv] = Y[(size_t)(p0 + i) + (size_t)(p0 + c) * ld];
    }
    __syncthreads();
    for (int tt = 0; tt < pw; ++tt) {
      T* vj = Vs + (size_t)tt * mv;  // column p0 + tt, local row index i <-> row p0 + i
      if (wid == 0) {
        const T tj = make_reflector_warp<T>(vj, tt, mv);
        if (lane == 0) tau[p0 + tt] = tj;
      }
      __syncthreads();
      const T tj = tau[p0 + tt];
      if (tj != T(0))
        for (int c = tt + 1 + wid; c < pw; c += nw) {
          T* vc = Vs + (size_t)c * mv;
          T w = T(0);
          for (int i = tt + 1 + lane; i < mv; i += 32) w += vj[i] * vc[i];
          w = warp_sum_all(w) + vc[tt];
          const T f = tj * w;
          __syncwarp();
          if (lane == 0) vc[tt] -= f;
          for (int i = tt + 1 + lane; i < mv; i += 32) vc[i] -= f * vj[i];
        }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < mv * pw; e += blockDim.x) {
      const int i = e % mv, c = e / mv;
      Y[(size_t)(p0 + i) + (size_t)(p0 + c) * ld] = Vs[i + (size_t)c * mv];
    }
    __syncthreads();
    // --- V (unit diagonal, zero above) in place
    for (int e = threadIdx.x; e < mv * pw; e += blockDim.x) {
      const int i = e % mv, c = e / mv;
      if (i <= c) Vs[i + (size_t)c * mv] = i == c ? T(1) : T(0);
    }
    __syncthreads();
    // --- G = V^T V (upper part), then T: T[s][s] = tau_s, T[0:s, s] = -tau_s T[0:s,0:s] G[0:s, s]
    for (int e = wid; e < pw * pw; e += nw) {
      const int a = e % pw, b = e / pw;
      if (a >= b) continue;
      T g = T(0);
      for (int i = lane; i < mv; i += 32) g += Vs[i + (size_t)a * mv] * Vs[i + (size_t)b * mv];
      g = warp_sum_all(g);
      if (lane == 0) G[a][b] = g;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      T (*Tp)[kQrNB] = Tall[pi];
      for (int s = 0; s < kQrNB; ++s)
        for (int r = 0; r < kQrNB; ++r) Tp[r][s] = T(0);
      for (int s = 0; s < pw; ++s) {
        const T ts = tau[p0 + s];
        for (int r = 0; r < s; ++r) {
          T acc = T(0);
          for (int q = r; q < s; ++q) acc += Tp[r][q] * G[q][s];
          Tp[r][s] = -ts * acc;
        }
        Tp[s][s] = ts;
      }
    }
    __syncthreads();
    // --- trailing columns: a -= V (T^T (V^T a)), rows p0..m-1
    const T (*Tp)[kQrNB] = Tall[pi];
    for (int c = p0 + pw + wid; c < k; c += nw) {
      T* ac = Y + (size_t)c * ld + p0;
      T w[kQrNB];
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) w[s] = T(0);
#pragma unroll 8
      for (int i = lane; i < mv; i += 32) {
        const T a = ac[i];
#pragma unroll
        for (int s = 0; s < kQrNB; ++s)
          if (s < pw) w[s] += Vs[i + (size_t)s * mv] * a;
      }
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) w[s] = warp_sum_all(w[s]);
      T u[kQrNB];
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) {
        T acc = T(0);
#pragma unroll
        for (int r = 0; r < kQrNB; ++r)
          if (r <= s) acc += Tp[r][s] * w[r];  // (T^T w)_s = sum_{r <= s} T[r][s] w[r]
        u[s] = acc;
      }
#pragma unroll 8
      for (int i = lane; i < mv; i += 32) {
        T a = ac[i];
#pragma unroll
        for (int s = 0; s < kQrNB; ++s)
          if (s < pw) a -= Vs[i + (size_t)s * mv] * u[s];
        ac[i] = a;
      }
    }
    __syncthreads();
  }
  if (t.R) {
    T* R = (T*)t.R;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int i = e % k, c = e / k;
      R[i + (size_t)c * k] = (i <= c) ? Y[(size_t)i + (size_t)c * ld] : T(0);
    }
  }
  __syncthreads();
  // --- Q = H_0 ... H_{k-1} [I; 0], panels backwards
  for (int pi = npanels - 1; pi >= 0; --pi) {
    const int p0 = pi * kQrNB, pw = min(kQrNB, k - p0), mv = m - p0;
    for (int e = threadIdx.x; e < mv * pw; e += blockDim.x) {
      const int i = e % mv, s = e / mv;
      const T v = i < s ? T(0) : (i == s ? T(1) : Y[(size_t)(p0 + i) + (size_t)(p0 + s) * ld]);
      Vs[i + (size_t)s * mv] = v;
    }
    __syncthreads();
    const T (*Tp)[kQrNB] = Tall[pi];
    // trailing Q columns c >= p0 + pw over rows p0..: rows p0 .. p0+pw-1 still hold R and
    // are read as the zeros they are in Q at this stage (rows above p0 are handled by the
    // earlier panels, processed after this one)
    for (int c = p0 + pw + wid; c < k; c += nw) {
      T* qc = Y + (size_t)c * ld + p0;
      T w[kQrNB];
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) w[s] = T(0);
#pragma unroll 8
      for (int i = lane; i < mv; i += 32) {
        const T q = i < pw ? T(0) : qc[i];
#pragma unroll
        for (int s = 0; s < kQrNB; ++s)
          if (s < pw) w[s] += Vs[i + (size_t)s * mv] * q;
      }
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) w[s] = warp_sum_all(w[s]);
      T u[kQrNB];
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) {
        T acc = T(0);
#pragma unroll
        for (int r = 0; r < kQrNB; ++r)
          if (r >= s) acc += Tp[s][r] * w[r];  // (T w)_s = sum_{r >= s} T[s][r] w[r]
        u[s] = acc;
      }
#pragma unroll 8
      for (int i = lane; i < mv; i += 32) {
        T q = i < pw ? T(0) : qc[i];
#pragma unroll
        for (int s = 0; s < kQrNB; ++s)
          if (s < pw) q -= Vs[i + (size_t)s * mv] * u[s];
        qc[i] = q;
      }
    }
    // the panel's own columns: e_j - V (T (V^T e_j)), V^T e_j = row j - p0 of V
    for (int tt = wid; tt < pw; tt += nw) {
      T* qc = Y + (size_t)(p0 + tt) * ld + p0;
      T u[kQrNB];
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) {
        T acc = T(0);
#pragma unroll
        for (int r = 0; r < kQrNB; ++r)
          if (r >= s && r < pw) acc += Tp[s][r] * Vs[tt + (size_t)r * mv];
        u[s] = acc;
      }
      for (int i = lane; i < mv; i += 32) {
        T q = (i == tt) ? T(1) : T(0);
#pragma unroll
        for (int s = 0; s < kQrNB; ++s)
          if (s < pw) q -= Vs[i + (size_t)s * mv] * u[s];
        qc[i] = q;
      }
    }
    __syncthreads();
  }
}

// =====================================================================================
// Panel QR with the whole panel resident in shared memory (m k elements) plus a
// row-major copy of the current block of reflectors (m x 8).  Same blocked compact-WY
// Householder algorithm as k_qr_blocked, but every trailing update and the backward
// formation of Q run on shared memory instead of round trips to global memory, and a
// row of V (unit diagonal and zeros above it written out) is two 16-byte loads.  The
// trailing columns go to warps in groups of four (two in FP64).
// =====================================================================================
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

// V of the current panel at local row i, reflector s (reflector tails in place below
// the diagonal of S).
template <typename T>
__device__ __forceinline__ T vget(const T* __restrict__ Vp, int m, int i, int s) {
  return i > s ? Vp[i + (size_t)s * m] : (i == s ? T(1) : T(0));
}

// Row-major reflector block: plane p (m rows of 16 bytes) holds reflectors p NV .. p NV + NV - 1.
template <typename T>
__device__ __forceinline__ T& vr_at(T* __restrict__ Vr, int m, int i, int s) {
  constexpr int NV = 16 / sizeof(T);
  return Vr[(size_t)(s / NV) * NV * m + (size_t)i * NV + s % NV];
}
template <typename T>
__device__ __forceinline__ void vr_row(const T* __restrict__ Vr, int m, int i, T (&v)[kQrNB]) {
  using V = typename Vec16<T>::type;
  constexpr int NV = 16 / sizeof(T);
#pragma unroll
  for (int p = 0; p < kQrNB / NV; ++p) {
    const V x = reinterpret_cast<const V*>(Vr + (size_t)p * NV * m)[i];
    const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int q = 0; q < NV; ++q) v[p * NV + q] = e[q];
  }
}

// Reflector of column j (rows j.. of aj in shared memory): tail scaled in place,
// aj[j] = beta; returns tau.  Every lane of one warp calls it; four partial sums per
// lane keep several loads in flight.
template <typename T>
__device__ __forceinline__ T reflector_warp_ilp(T* __restrict__ aj, int j, int m) {
  const int lane = threadIdx.x & 31;
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int i = j + 1 + lane;
  for (; i + 96 < m; i += 128) {
    const T a0 = aj[i], a1 = aj[i + 32], a2 = aj[i + 64], a3 = aj[i + 96];
    s0 += a0 * a0; s1 += a1 * a1; s2 += a2 * a2; s3 += a3 * a3;
  }
  for (; i < m; i += 32) s0 += aj[i] * aj[i];
  const T s = warp_sum_all((s0 + s1) + (s2 + s3));
  const T x0 = aj[j];
  T tj = T(0), beta = x0, scale = T(1);
  if (s > T(0)) {
    const T nrm = sqrt(x0 * x0 + s);
    beta = x0 >= T(0) ? -nrm : nrm;
    tj = (beta - x0) / beta;
    scale = T(1) / (x0 - beta);
  }
  for (int r = j + 1 + lane; r < m; r += 32) aj[r] *= scale;
  __syncwarp();
  if (lane == 0) aj[j] = beta;
  return tj;
}

template <typename T>
__device__ __forceinline__ void cp_async_4or8(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}

// Trailing update of one reflector block (rows p0.., columns p0 + pw ..), CW columns per
// warp pass so that a row of V is read once per pass: the factorization applies
// (I - V T V^T)^T (u = T^T w), the backward formation of Q applies I - V T V^T
// (u = T w) and reads the block's own rows 0..pw-1 of those columns as zero.  Groups
// narrow as the trailing part shrinks, so all warps stay busy.
template <typename T, int CW, bool QFORM>
__device__ __forceinline__ void qr_trail(T* __restrict__ S, const T* __restrict__ Vr, const T (*Tp)[kQrNB], int m,
                                         int k, int p0, int pw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int mv = m - p0, c0 = p0 + pw, ngroups = (k - c0 + CW - 1) / CW;
  for (int g = wid; g < ngroups; g += nw) {
    const int cb = c0 + g * CW, ncol = min(CW, k - cb);
    T* A0 = S + (size_t)cb * m + p0;
    T w[CW][kQrNB];
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) w[c][s] = T(0);
    for (int i = (QFORM ? pw : 0) + lane; i < mv; i += 32) {
      T v[kQrNB];
      vr_row(Vr, m, i, v);
#pragma unroll
      for (int c = 0; c < CW; ++c)
        if (c < ncol) {
          const T a = A0[i + (size_t)c * m];
#pragma unroll
          for (int s = 0; s < kQrNB; ++s) w[c][s] += v[s] * a;
        }
    }
    T u[CW][kQrNB];
#pragma unroll
    for (int c = 0; c < CW; ++c) {
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) w[c][s] = warp_sum_all(w[c][s]);
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) {
        T acc = T(0);
        if (QFORM) {
#pragma unroll
          for (int r = s; r < kQrNB; ++r) acc += Tp[s][r] * w[c][r];  // (T w)_s
        } else {
#pragma unroll
          for (int r = 0; r <= s; ++r) acc += Tp[r][s] * w[c][r];  // (T^T w)_s
        }
        u[c][s] = acc;
      }
    }
    for (int i = lane; i < mv; i += 32) {
      T v[kQrNB], a[CW];
      vr_row(Vr, m, i, v);
#pragma unroll
      for (int c = 0; c < CW; ++c) a[c] = c < ncol && (!QFORM || i >= pw) ? A0[i + (size_t)c * m] : T(0);
#pragma unroll
      for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int s = 0; s < kQrNB; ++s) a[c] -= v[s] * u[c][s];
#pragma unroll
      for (int c = 0; c < CW; ++c)
        if (c < ncol) A0[i + (size_t)c * m] = a[c];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_qr_smem(const QrTask* __restrict__ tasks, int64_t vr_off) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T tau[256];
  __shared__ T vscale[256];
  __shared__ T Tall[256 / kQrNB][kQrNB][kQrNB];
  __shared__ T Gred[16][kQrNB * (kQrNB - 1) / 2];
  __shared__ T U8[kQrNB][kQrNB];
  constexpr int CWMAX = sizeof(T) == 8 ? 2 : 4;  // widest trailing column group
  const QrTask t = tasks[blockIdx.x];
  const int m = t.m, k = t.k, ld = t.ld;
  T* __restrict__ Y = (T*)t.Y;
  T* __restrict__ S = reinterpret_cast<T*>(smem_raw);  // the panel, m x k, ld m
  T* __restrict__ Vr = S + vr_off;                     // current reflector block, row-major
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < k; c += nw)  // all copies in flight at once
    for (int i = lane; i < m; i += 32) cp_async_4or8(S + i + (size_t)c * m, Y + i + (size_t)c * ld);
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  const int npanels = (k + kQrNB - 1) / kQrNB;
  for (int pi = 0; pi < npanels; ++pi) {
    const int p0 = pi * kQrNB, pw = min(kQrNB, k - p0), mv = m - p0;
    T* Vp = S + (size_t)p0 * m + p0;
    // --- panel, with look-ahead: after reflector tt is known, warp 0 applies it to
    //     column tt + 1 and at once forms reflector tt + 1 (its norm accumulated while
    //     updating), while warps 1.. apply it to the panel's later columns; one barrier
    //     per column
    //     A reflector's tail stays unscaled in S (v_i = sc_j x_i, sc_j in vscale) until
    //     the row-major copy is built, which saves a pass over the column.
    if (wid == 0) {
      T s0 = T(0), s1 = T(0);
      for (int r = 1 + lane; r < mv; r += 32) {
        const T v = Vp[r];
        if (r & 32) s1 += v * v; else s0 += v * v;
      }
      const T s = warp_sum_all(s0 + s1);
      const T x0 = Vp[0];
      T tn = T(0), beta = x0, scale = T(1);
      if (s > T(0)) {
        const T nrm = sqrt(x0 * x0 + s);
        beta = x0 >= T(0) ? -nrm : nrm;
        tn = (beta - x0) / beta;
        scale = T(1) / (x0 - beta);
      }
      __syncwarp();
      if (lane == 0) {
        Vp[0] = beta;
        tau[p0] = tn;
        vscale[p0] = scale;
      }
    }
    __syncthreads();
    for (int tt = 0; tt + 1 < pw; ++tt) {
      const T* vj = Vp + (size_t)tt * m;
      const T tj = tau[p0 + tt], sj = vscale[p0 + tt];
      for (int c = tt + 1 + wid; c < pw; c += nw) {
        T* vc = Vp + (size_t)c * m;
        T f = T(0);  // the update is vc -= f v_j = (f sc_j) x
        if (tj != T(0)) {
          T w0 = T(0), w1 = T(0), w2 = T(0), w3 = T(0);
          int i = tt + 1 + lane;
          for (; i + 96 < mv; i += 128) {
            w0 += vj[i] * vc[i];
            w1 += vj[i + 32] * vc[i + 32];
            w2 += vj[i + 64] * vc[i + 64];
            w3 += vj[i + 96] * vc[i + 96];
          }
          for (; i < mv; i += 32) w0 += vj[i] * vc[i];
          const T ft = tj * (sj * warp_sum_all((w0 + w1) + (w2 + w3)) + vc[tt]);
          __syncwarp();
          if (lane == 0) vc[tt] -= ft;
          f = ft * sj;
        }
        T s0 = T(0), s1 = T(0);
        int r = tt + 1 + lane;
        for (; r + 96 < mv; r += 128) {  // loads first: the stores cannot alias them
          T a0 = vc[r], a1 = vc[r + 32], a2 = vc[r + 64], a3 = vc[r + 96];
          const T b0 = vj[r], b1 = vj[r + 32], b2 = vj[r + 64], b3 = vj[r + 96];
          a0 -= f * b0; a1 -= f * b1; a2 -= f * b2; a3 -= f * b3;
          vc[r] = a0; vc[r + 32] = a1; vc[r + 64] = a2; vc[r + 96] = a3;
          if (r > c) s0 += a0 * a0;
          s1 += a1 * a1 + a2 * a2;
          s0 += a3 * a3;
        }
        for (; r < mv; r += 32) {
          const T a = vc[r] - f * vj[r];
          vc[r] = a;
          if (r > c) s1 += a * a;
        }
        if (c == tt + 1) {  // warp 0: the next reflector, from the column just updated
          const T s = warp_sum_all(s0 + s1);
          __syncwarp();
          const T x0 = vc[c];
          T tn = T(0), beta = x0, scale = T(1);
          if (s > T(0)) {
            const T nrm = sqrt(x0 * x0 + s);
            beta = x0 >= T(0) ? -nrm : nrm;
            tn = (beta - x0) / beta;
            scale = T(1) / (x0 - beta);
          }
          __syncwarp();
          if (lane == 0) {
            vc[c] = beta;
            tau[p0 + c] = tn;
            vscale[p0 + c] = scale;
          }
        }
      }
      __syncthreads();
    }
    // --- the block's V, row-major, unit diagonal and zeros above written out
    for (int i = threadIdx.x; i < mv; i += blockDim.x)
#pragma unroll
      for (int s = 0; s < kQrNB; ++s)
        vr_at(Vr, m, i, s) = s < pw ? (i > s ? vscale[p0 + s] * Vp[i + (size_t)s * m] : (i == s ? T(1) : T(0))) : T(0);
    __syncthreads();
    // --- G = V^T V (strict upper part) in one pass over the rows, then the panel's T
    //     column by column (lane r of warp 0 holds row r of T)
    {
      T gacc[kQrNB * (kQrNB - 1) / 2];
#pragma unroll
      for (int e = 0; e < kQrNB * (kQrNB - 1) / 2; ++e) gacc[e] = T(0);
      for (int i = threadIdx.x; i < mv; i += blockDim.x) {
        T v[kQrNB];
        vr_row(Vr, m, i, v);
        int e = 0;
#pragma unroll
        for (int b = 1; b < kQrNB; ++b)
#pragma unroll
          for (int a = 0; a < b; ++a) gacc[e++] += v[a] * v[b];
      }
#pragma unroll
      for (int e = 0; e < kQrNB * (kQrNB - 1) / 2; ++e) {
        const T g = warp_sum_all(gacc[e]);
        if (lane == 0) Gred[wid][e] = g;
      }
    }
    __syncthreads();
    if (threadIdx.x < kQrNB * (kQrNB - 1) / 2) {
      T g = T(0);
      for (int w = 0; w < nw; ++w) g += Gred[w][threadIdx.x];
      Gred[0][threadIdx.x] = g;  // packed: pair (a, b), a < b, at b (b - 1) / 2 + a
    }
    __syncthreads();
    if (wid == 0) {
      T trow[kQrNB];
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) trow[s] = T(0);
#pragma unroll
      for (int s = 0; s < kQrNB; ++s) {
        if (s < pw) {
          const T ts = tau[p0 + s];
          T acc = T(0);
#pragma unroll
          for (int q = 0; q < s; ++q)
            if (q >= lane) acc += trow[q] * Gred[0][s * (s - 1) / 2 + q];
          trow[s] = lane < s ? -ts * acc : (lane == s ? ts : T(0));
        }
      }
      if (lane < kQrNB)
#pragma unroll
        for (int s = 0; s < kQrNB; ++s) Tall[pi][lane][s] = trow[s];
    }
    __syncthreads();
    // --- trailing columns: a -= V (T^T (V^T a)), local rows 0..mv-1
    {
      const int ntr = k - (p0 + pw);
      if (CWMAX >= 4 && ntr > 32) qr_trail<T, 4, false>(S, Vr, Tall[pi], m, k, p0, pw);
      else if (ntr > 16) qr_trail<T, 2, false>(S, Vr, Tall[pi], m, k, p0, pw);
      else qr_trail<T, 1, false>(S, Vr, Tall[pi], m, k, p0, pw);
    }
    __syncthreads();
  }
  if (t.R) {
    T* R = (T*)t.R;
    const int ldr = t.ldr > 0 ? t.ldr : k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int i = e % k, c = e / k;
      R[i + (size_t)c * ldr] = (i <= c) ? S[i + (size_t)c * m] : T(0);
    }
  }
  __syncthreads();
  // --- Q = H_0 ... H_{k-1} [I; 0], panels backwards
  for (int pi = npanels - 1; pi >= 0; --pi) {
    const int p0 = pi * kQrNB, pw = min(kQrNB, k - p0), mv = m - p0;
    T* Vp = S + (size_t)p0 * m + p0;
    const T (*Tp)[kQrNB] = Tall[pi];
    for (int i = threadIdx.x; i < mv; i += blockDim.x)
#pragma unroll
      for (int s = 0; s < kQrNB; ++s)
        vr_at(Vr, m, i, s) = s < pw ? (i > s ? vscale[p0 + s] * Vp[i + (size_t)s * m] : (i == s ? T(1) : T(0))) : T(0);
    __syncthreads();
    if (threadIdx.x < kQrNB * kQrNB) {  // U8[j] = T V^T e_j for the panel's own columns
      const int j = threadIdx.x / kQrNB, s = threadIdx.x % kQrNB;
      T acc = T(0);
      if (j < pw && s < pw)
        for (int r = s; r < pw; ++r) acc += Tp[s][r] * vr_at(Vr, m, j, r);
      U8[j][s] = acc;
    }
    __syncthreads();
    // trailing Q columns c >= p0 + pw: local rows 0..pw-1 still hold R and are read as
    // the zeros they are in Q at this stage (rows above p0 belong to earlier panels,
    // which run after this one and write them)
    {
      const int ntr = k - (p0 + pw);
      if (CWMAX >= 4 && ntr > 32) qr_trail<T, 4, true>(S, Vr, Tall[pi], m, k, p0, pw);
      else if (ntr > 16) qr_trail<T, 2, true>(S, Vr, Tall[pi], m, k, p0, pw);
      else qr_trail<T, 1, true>(S, Vr, Tall[pi], m, k, p0, pw);
    }
    // the panel's own columns: Q(i, j) = delta_ij - sum_s V(i, s) (T V^T e_j)_s
    for (int i = threadIdx.x; i < mv; i += blockDim.x) {
      T v[kQrNB];
      vr_row(Vr, m, i, v);
#pragma unroll
      for (int j = 0; j < kQrNB; ++j)
        if (j < pw) {
          T q = i == j ? T(1) : T(0);
#pragma unroll
          for (int s = 0; s < kQrNB; ++s) q -= v[s] * U8[j][s];
          Vp[i + (size_t)j * m] = q;
        }
    }
    __syncthreads();
  }
  T* __restrict__ Qo = t.Q ? (T*)t.Q : Y;
  const int ldo = t.Q ? t.ldq : ld;
  for (int c = wid; c < k; c += nw)
    for (int i = lane; i < m; i += 32) Qo[i + (size_t)c * ldo] = S[i + (size_t)c * m];
}

// Static shared memory of k_qr_smem (tau, every panel's T, the G partial sums, U8).
template <typename T>
constexpr size_t qr_smem_static() {
  return (512 + 256 / kQrNB * kQrNB * kQrNB + 16 * kQrNB * (kQrNB - 1) / 2 + kQrNB * kQrNB) * sizeof(T);
}

size_t qr_smem_overhead(int es) {
  return (es == 8 ? qr_smem_static<double>() : qr_smem_static<float>()) + 1024;
}

template <typename T>
void launch_qr(const QrTask* tasks, int ntasks, int maxm, int64_t maxmk, int max_smem, cudaStream_t s) {
  if (ntasks <= 0) return;
  // the panels, then (16-byte aligned) the row-major reflector block of the largest panel
  const int64_t vr_off = (maxmk + 15) / 16 * 16;
  const size_t whole = (size_t)(vr_off + (int64_t)kQrNB * maxm) * sizeof(T);
  if (whole + qr_smem_static<T>() + 1024 <= (size_t)max_smem) {
    k_qr_smem<T><<<ntasks, 512, whole, s>>>(tasks, vr_off);
    return;
  }
  const size_t vs = (size_t)maxm * kQrNB * sizeof(T);
  static const size_t blocked_static = [] {  // the kernel's own static shared memory
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, k_qr_blocked<T>) == cudaSuccess ? (size_t)a.sharedSizeBytes : (size_t)32768;
  }();
  if (vs + blocked_static + 1024 <= (size_t)max_smem) {
    k_qr_blocked<T><<<ntasks, 512, vs, s>>>(tasks);
    return;
  }
  // dynamic shared memory: tau for up to 256 reflectors
  k_qr<T><<<ntasks, 256, 256 * sizeof(T), s>>>(tasks);
}

// =====================================================================================
// Tall-skinny QR (TSQR) for the range finder's panels.  A panel's m rows are split into
// nb balanced blocks (each at least k rows).  (1) every block is factored by Householder
// in shared memory, its reflectors stay in the panel and its R_b goes to rows b k of a
// stacked matrix S (nb k x k); (2) S is factored the same way, giving the panel's R, and
// its explicit Q_S replaces S; (3) every block forms its rows of Q = diag(Q_b) Q_S as
// H_0 ... H_{k-1} [S_b; 0] from its reflectors and the rows b k .. b k + k - 1 of Q_S.
// Blocks of all panels of a level run in parallel; panels too large for shared memory
// use the single-CTA kernel above.  Reflectors are the scale-safe ones of that kernel.
// =====================================================================================

// Householder factorization of A (m x k, ld, shared memory, m >= k) in place: R on and
// above the diagonal, reflector tails below it, tau[j] per column.
template <typename T>
__device__ void hh_factor_smem(T* __restrict__ A, int m, int k, int ld, T* __restrict__ tau,
                               T* __restrict__ red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    T* aj = A + (size_t)j * ld;
    T s = T(0);
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) s += aj[i] * aj[i];
    s = block_sum(s, red);
    const T x0 = aj[j];
    T tj = T(0), beta = x0, scale = T(1);
    if (s > T(0)) {
      const T nrm = sqrt(x0 * x0 + s);
      beta = x0 >= T(0) ? -nrm : nrm;
      tj = (beta - x0) / beta;
      scale = T(1) / (x0 - beta);
    }
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) aj[i] *= scale;
    if (threadIdx.x == 0) {
      aj[j] = beta;
      tau[j] = tj;
    }
    __syncthreads();
    if (tj != T(0)) {
      for (int c = j + 1 + wid; c < k; c += nw) {
        T* ac = A + (size_t)c * ld;
        T w = T(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += aj[i] * ac[i];
        w = warp_sum(w) + ac[j];
        const T f = tj * w;
        __syncwarp();
        if (lane == 0) ac[j] -= f;
        for (int i = j + 1 + lane; i < m; i += 32) ac[i] -= f * aj[i];
      }
    }
    __syncthreads();
  }
}

// B (m x k, ld, shared memory) <- H_0 H_1 ... H_{k-1} B for reflectors with tails V
// (column j: rows j+1 .. m-1 of V, implicit 1 at row j; any memory) and scalars tau.
template <typename T>
__device__ void hh_apply_backward(const T* __restrict__ V, int ldv, const T* __restrict__ tau,
                                  T* __restrict__ B, int m, int k, int ldb) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = k - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj != T(0)) {
      const T* vj = V + (size_t)j * ldv;
      for (int c = wid; c < k; c += nw) {
        T* bc = B + (size_t)c * ldb;
        T w = T(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += vj[i] * bc[i];
        w = warp_sum(w) + bc[j];
        const T f = tj * w;
        __syncwarp();
        if (lane == 0) bc[j] -= f;
        for (int i = j + 1 + lane; i < m; i += 32) bc[i] -= f * vj[i];
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_tsqr_blocks(const TsqrTask* __restrict__ tasks,
                                                     const TsqrBlock* __restrict__ blocks, T* __restrict__ scratch) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T red[32];
  const TsqrBlock bl = blocks[blockIdx.x];
  const TsqrTask t = tasks[bl.task];
  const int k = t.k, nb = t.nb;
  const int r0 = (int)((int64_t)bl.block * t.m / nb), r1 = (int)((int64_t)(bl.block + 1) * t.m / nb);
  const int mb = r1 - r0;
  T* A = reinterpret_cast<T*>(smem_raw);  // mb x k, ld mb
  T* Y = (T*)t.Y + r0;
  for (int e = threadIdx.x; e < mb * k; e += blockDim.x) {
    const int i = e % mb, c = e / mb;
    A[e] = Y[(size_t)i + (size_t)c * t.ld];
  }
  __syncthreads();
  T* tau = scratch + t.soff + (int64_t)nb * k * k + (int64_t)bl.block * k;
  hh_factor_smem<T>(A, mb, k, mb, tau, red);
  T* S = scratch + t.soff;  // nb k x k, ld nb k
  const int lds = nb * k;
  for (int e = threadIdx.x; e < mb * k; e += blockDim.x) {
    const int i = e % mb, c = e / mb;
    Y[(size_t)i + (size_t)c * t.ld] = A[e];
    if (i < k) S[(size_t)(bl.block * k + i) + (size_t)c * lds] = i <= c ? A[e] : T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_tsqr_stack(const TsqrTask* __restrict__ tasks, T* __restrict__ scratch) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T red[32];
  const TsqrTask t = tasks[blockIdx.x];
  const int k = t.k, ms = t.nb * k;
  T* A = reinterpret_cast<T*>(smem_raw);  // ms x k, ld ms
  T* tau = A + (size_t)ms * k;            // k
  T* S = scratch + t.soff;
  for (int e = threadIdx.x; e < ms * k; e += blockDim.x) A[e] = S[e];
  __syncthreads();
  hh_factor_smem<T>(A, ms, k, ms, tau, red);
  if (t.R) {
    T* R = (T*)t.R;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int i = e % k, c = e / k;
      R[i + (size_t)c * k] = i <= c ? A[(size_t)i + (size_t)c * ms] : T(0);
    }
  }
  // explicit Q_S = H_0 ... H_{k-1} [I; 0], formed in place (column j's reflector is
  // consumed at step j, after which the column holds Q_S's column j)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, c = e / k;
    if (i < c) A[(size_t)i + (size_t)c * ms] = T(0);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const T tj = tau[j];
    T* aj = A + (size_t)j * ms;
    for (int c = j + 1 + wid; c < k; c += nw) {
      T* ac = A + (size_t)c * ms;
      T w = T(0);
      for (int i = j + 1 + lane; i < ms; i += 32) w += aj[i] * ac[i];
      w = warp_sum(w);  // Q_S[j, c] is still zero here
      const T f = tj * w;
      if (lane == 0) ac[j] = -f;
      for (int i = j + 1 + lane; i < ms; i += 32) ac[i] -= f * aj[i];
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < ms; i += blockDim.x) aj[i] *= -tj;
    if (threadIdx.x == 0) aj[j] = T(1) - tj;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < ms * k; e += blockDim.x) S[e] = A[e];
}

template <typename T>
__global__ void __launch_bounds__(256) k_tsqr_q(const TsqrTask* __restrict__ tasks,
                                                const TsqrBlock* __restrict__ blocks, T* __restrict__ scratch) {
  extern __shared__ unsigned char smem_raw[];
  const TsqrBlock bl = blocks[blockIdx.x];
  const TsqrTask t = tasks[bl.task];
  const int k = t.k, nb = t.nb, lds = nb * k;
  const int r0 = (int)((int64_t)bl.block * t.m / nb), r1 = (int)((int64_t)(bl.block + 1) * t.m / nb);
  const int mb = r1 - r0;
  T* B = reinterpret_cast<T*>(smem_raw);  // mb x k, ld mb
  const T* S = scratch + t.soff;
  for (int e = threadIdx.x; e < mb * k; e += blockDim.x) {
    const int i = e % mb, c = e / mb;
    B[e] = i < k ? S[(size_t)(bl.block * k + i) + (size_t)c * lds] : T(0);
  }
  __syncthreads();
  T* Y = (T*)t.Y + r0;
  const T* tau = scratch + t.soff + (int64_t)nb * k * k + (int64_t)bl.block * k;
  hh_apply_backward<T>(Y, t.ld, tau, B, mb, k, mb);
  for (int e = threadIdx.x; e < mb * k; e += blockDim.x) {
    const int i = e % mb, c = e / mb;
    Y[(size_t)i + (size_t)c * t.ld] = B[e];
  }
}

template <typename T>
void launch_tsqr(const TsqrTask* tasks, int ntasks, const TsqrBlock* blocks, int nblocks, size_t smem_block,
                 size_t smem_stack, T* scratch, cudaStream_t s) {
  if (ntasks <= 0) return;
  k_tsqr_blocks<T><<<nblocks, 256, smem_block, s>>>(tasks, blocks, scratch);
  k_tsqr_stack<T><<<ntasks, 256, smem_stack, s>>>(tasks, scratch);
  k_tsqr_q<T><<<nblocks, 256, smem_block, s>>>(tasks, blocks, scratch);
}

// =====================================================================================
// SVD of M = R^T (k x k) by one-sided Jacobi (Hestenes) with the round-robin pair order;
// a warp rotates one column pair at a time.  Sorted output, truncation at tol*sigma_1.
// =====================================================================================
template <typename T>
struct JacobiEps;
// Rotation threshold |gamma| > eps sqrt(alpha beta): a few units of rounding of the
// precision (singular values come out with that relative accuracy, far below any
// truncation tolerance); sweeps are capped at kJacobiSweeps (convergence is quadratic).
template <>
struct JacobiEps<float> {
  static constexpr float v = 4e-7f * 8;
};
template <>
struct JacobiEps<double> {
  static constexpr double v = 2.3e-16 * 8;
};
constexpr int kJacobiSweeps = 12;

template <typename T>
__global__ void __launch_bounds__(512) k_svd(const SvdTask* __restrict__ tasks, double tol) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int rotated, nlive;
  __shared__ int live[256];
  const SvdTask t = tasks[blockIdx.x];
  const int k = t.k, ls = k + 1;
  T* M = reinterpret_cast<T*>(smem_raw);
  T* V = M + (size_t)k * ls;
  T* sig = V + (size_t)k * ls;
  const T* R = (const T*)t.R;
  __shared__ T red[32];
  T f2 = T(0);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, c = e / k;
    const T v = R[c + (size_t)i * k];
    M[i + c * ls] = v;  // M = R^T
    V[i + c * ls] = (i == c) ? T(1) : T(0);
    f2 += v * v;
  }
  // A column at rounding level of ||M||_F carries no information (its singular value
  // falls far below any truncation tolerance): pairs involving one are left alone, so
  // such columns are compacted away and the sweeps run over the other columns only.
  const T floor2 = block_sum(f2, red) * JacobiEps<T>::v * JacobiEps<T>::v;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < k; c += nw) {
    T s2 = T(0);
    for (int i = lane; i < k; i += 32) s2 += M[i + c * ls] * M[i + c * ls];
    s2 = warp_sum(s2);
    if (lane == 0) sig[c] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int c = 0; c < k; ++c)
      if (sig[c] > floor2) live[n++] = c;
    nlive = n;
  }
  __syncthreads();
  const int kl = nlive, kk = kl + (kl & 1), npairs = kk / 2;
  // one 16-lane group per column pair; every group runs the same number of passes so
  // the width-16 shuffles are always executed by full warps
  const int gl = threadIdx.x & 15, gid = threadIdx.x >> 4, ng = blockDim.x >> 4;
  const T eps2 = JacobiEps<T>::v * JacobiEps<T>::v;
  for (int sweep = 0; sweep < kJacobiSweeps && kk > 1; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < kk - 1; ++r) {
      for (int base = 0; base < npairs; base += ng) {
        // round-robin order over the live columns (position 0 fixed, the others rotate)
        const int pi = base + gid;
        int x = pi - 1 + r, y = kk - 2 - pi + r;
        if (x >= kk - 1) x -= kk - 1;
        if (y >= kk - 1) y -= kk - 1;
        const int a = pi == 0 ? 0 : 1 + x, b = 1 + y;
        const bool valid = pi < npairs && a < kl && b < kl;
        const int p = valid ? min(live[a], live[b]) : 0, q = valid ? max(live[a], live[b]) : 0;
        T al = T(0), be = T(0), ga = T(0);
        if (valid)
          for (int i = gl; i < k; i += 16) {
            const T mp = M[i + p * ls], mq = M[i + q * ls];
            al += mp * mp;
            be += mq * mq;
            ga += mp * mq;
          }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o, 16);
          be += __shfl_xor_sync(0xffffffffu, be, o, 16);
          ga += __shfl_xor_sync(0xffffffffu, ga, o, 16);
        }
        if (valid && ga != T(0) && ga * ga > eps2 * (al * be)) {
          const T zeta = (be - al) / (T(2) * ga);
          const T tt = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T c = T(1) / sqrt(T(1) + tt * tt), sn = c * tt;
          for (int i = gl; i < k; i += 16) {
            const T mp = M[i + p * ls], mq = M[i + q * ls];
            M[i + p * ls] = c * mp - sn * mq;
            M[i + q * ls] = sn * mp + c * mq;
            const T vp = V[i + p * ls], vq = V[i + q * ls];
            V[i + p * ls] = c * vp - sn * vq;
            V[i + q * ls] = sn * vp + c * vq;
          }
          if (gl == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  for (int c = wid; c < k; c += nw) {
    T s2 = T(0);
    for (int i = lane; i < k; i += 32) s2 += M[i + c * ls] * M[i + c * ls];
    s2 = warp_sum(s2);
    if (lane == 0) sig[c] = sqrt(s2);
  }
  __syncthreads();
  T smax = T(0);
  for (int c = 0; c < k; ++c) smax = sig[c] > smax ? sig[c] : smax;
  const T thr = tol > 0.0 ? (T)tol * smax : T(0);
  int rank = 0;
  for (int c = 0; c < k; ++c) rank += (sig[c] > thr) ? 1 : 0;
  T* UhS = (T*)t.UhS;
  T* Vh = (T*)t.Vh;
  for (int c = wid; c < k; c += nw) {
    int pos = 0;
    for (int j = 0; j < k; ++j) pos += (sig[j] > sig[c] || (sig[j] == sig[c] && j < c)) ? 1 : 0;
    const bool keep = pos < rank;
    for (int i = lane; i < k; i += 32) {
      UhS[i + (size_t)pos * k] = keep ? M[i + c * ls] : T(0);
      Vh[i + (size_t)pos * k] = keep ? V[i + c * ls] : T(0);
    }
  }
  if (threadIdx.x == 0 && t.rank) *t.rank = rank;
}

// =====================================================================================
// BDLR (Section 2.2, Eq. Bhat): one block of 256 threads per off-diagonal block.
// (1) Breadth-first distances (up to depth) from Y and from X over the graph of A
//     restricted to the front's unknowns [I_p, I_p^f] (local position p <-> global new
//     index first[q] + p for p < np, else the sorted I_p^f list, found by bisection).
// (2) I = rows of X with distance <= depth from Y, J likewise, nearer first then lower
//     position, at most cap each (warp-ballot compaction in position order).
// (3) Complete-pivoting LU of B^ = B(I, J) in shared memory (argmax of |entry|, ties to
//     the lower (i, j) in selection order), stopping at the first pivot below tol |u_11|.
// (4) U rows = B(x, J_q) U_r^{-1} (one row of X per thread), V rows = L_r^{-1} B(I_p, y)
//     (one column of Y per thread).
// =====================================================================================
constexpr unsigned char kBdlrFar = 255;

__device__ __forceinline__ int bdlr_local(int u, int b0, int np, const int32_t* __restrict__ If, int nu) {
  if (u >= b0 && u < b0 + np) return u - b0;
  int lo = 0, hi = nu;  // first position with If[pos] >= u
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (If[mid] < u) lo = mid + 1; else hi = mid;
  }
  return (lo < nu && If[lo] == u) ? np + lo : -1;
}

template <typename T>
__global__ void __launch_bounds__(256) k_bdlr(const BdlrTask* __restrict__ tasks, int depth, double tol,
                                              const int32_t* __restrict__ first, const int* __restrict__ npiv,
                                              const int64_t* __restrict__ ifoff, const int32_t* __restrict__ iflist,
                                              const int64_t* __restrict__ prowptr, const int32_t* __restrict__ pcol,
                                              int maxcap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BdlrTask t = tasks[blockIdx.x];
  const int nh = t.nh, cap = t.cap, q = t.q;
  const int np = npiv[q], nu = nh - np, b0 = first[q];
  const int32_t* If = iflist + ifoff[q];
  // shared memory: Bh (maxcap^2 T), row/col lists, pivot orders, then the two distance arrays
  T* Bh = reinterpret_cast<T*>(smem_raw);
  int* Il = reinterpret_cast<int*>(Bh + (size_t)maxcap * maxcap);
  int* Jl = Il + maxcap;
  int* pr = Jl + maxcap;
  int* pc = pr + maxcap;
  unsigned char* rowUsed = reinterpret_cast<unsigned char*>(pc + maxcap);
  unsigned char* colUsed = rowUsed + maxcap;
  unsigned char* dY = colUsed + maxcap;
  unsigned char* dX = dY + nh;
  __shared__ int s_n[2], s_rank, s_stop;
  __shared__ T s_val[8];
  __shared__ int s_idx[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v = threadIdx.x; v < nh; v += blockDim.x) {
    dY[v] = (v >= t.y0 && v < t.y0 + t.my) ? 0 : kBdlrFar;
    dX[v] = (v >= t.x0 && v < t.x0 + t.mx) ? 0 : kBdlrFar;
  }
  __syncthreads();
  for (int l = 0; l < depth; ++l) {
    for (int v = threadIdx.x; v < nh; v += blockDim.x) {
      const bool fy = dY[v] == l, fx = dX[v] == l;
      if (!fy && !fx) continue;
      const int g = v < np ? b0 + v : If[v - np];
      for (int64_t e = prowptr[g]; e < prowptr[g + 1]; ++e) {
        const int p = bdlr_local(pcol[e], b0, np, If, nu);
        if (p < 0) continue;
        if (fy && dY[p] == kBdlrFar) dY[p] = (unsigned char)(l + 1);
        if (fx && dX[p] == kBdlrFar) dX[p] = (unsigned char)(l + 1);
      }
    }
    __syncthreads();
  }
  // selection in (distance, position) order
  if (wid < 2) {
    const unsigned char* d = wid == 0 ? dY : dX;
    const int lo = wid == 0 ? t.x0 : t.y0, m = wid == 0 ? t.mx : t.my;
    int* out = wid == 0 ? Il : Jl;
    int cnt = 0;
    for (int l = 1; l <= depth && cnt < cap; ++l)
      for (int base = 0; base < m && cnt < cap; base += 32) {
        const int i = base + lane;
        const bool sel = i < m && d[lo + i] == l;
        const unsigned bal = __ballot_sync(0xffffffffu, sel);
        const int before = __popc(bal & ((1u << lane) - 1u));
        if (sel && cnt + before < cap) out[cnt + before] = i;
        cnt = min(cap, cnt + __popc(bal));
      }
    if (lane == 0) s_n[wid] = cnt;
  }
  __syncthreads();
  const int nI = s_n[0], nJ = s_n[1];
  auto Bel = [&](int i, int j) -> T {  // B(i, j), i in X, j in Y (block-relative)
    const T* F = (const T*)t.F;
    return t.trans ? F[(size_t)(t.y0 + j) + (size_t)(t.x0 + i) * nh] : F[(size_t)(t.x0 + i) + (size_t)(t.y0 + j) * nh];
  };
  for (int e = threadIdx.x; e < nI * nJ; e += blockDim.x) {
    const int i = e / nJ, j = e % nJ;
    Bh[i * maxcap + j] = Bel(Il[i], Jl[j]);
  }
  for (int a = threadIdx.x; a < maxcap; a += blockDim.x) { rowUsed[a] = 0; colUsed[a] = 0; }
  if (threadIdx.x == 0) { s_rank = 0; s_stop = 0; }
  __syncthreads();
  // complete-pivoting LU; rows/columns already pivoted are marked by pr/pc entries
  T u11 = T(0);
  const int rmax = min(nI, nJ);
  for (int s = 0; s < rmax; ++s) {
    T best = T(-1);
    int bidx = INT_MAX;
    for (int e = threadIdx.x; e < nI * nJ; e += blockDim.x) {
      const int i = e / nJ, j = e % nJ;
      if (rowUsed[i] || colUsed[j]) continue;
      const T v = fabs(Bh[i * maxcap + j]);
      if (v > best || (v == best && e < bidx)) { best = v; bidx = e; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
    }
    if (lane == 0) { s_val[wid] = best; s_idx[wid] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      T bv = s_val[0];
      int bi = s_idx[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bi)) { bv = s_val[w]; bi = s_idx[w]; }
      if (s == 0) u11 = bv;
      const T u1 = s == 0 ? bv : fabs(Bh[pr[0] * maxcap + pc[0]]);
      if (bv <= T(0) || (s > 0 && tol > 0.0 && bv < (T)tol * u1)) s_stop = 1;
      else {
        pr[s] = bi / nJ;
        pc[s] = bi % nJ;
        s_rank = s + 1;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int ip = pr[s], jp = pc[s];
    const T piv = Bh[ip * maxcap + jp];
    // eliminate: multipliers into column jp of the remaining rows, update the rest
    for (int e = threadIdx.x; e < nI * nJ; e += blockDim.x) {
      const int i = e / nJ, j = e % nJ;
      if (i == ip || j == jp || rowUsed[i] || colUsed[j]) continue;
      const T l = Bh[i * maxcap + jp] / piv;
      Bh[i * maxcap + j] -= l * Bh[ip * maxcap + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nI; i += blockDim.x)
      if (i != ip && !rowUsed[i]) Bh[i * maxcap + jp] /= piv;
    __syncthreads();
    if (threadIdx.x == 0) {
      rowUsed[ip] = 1;
      colUsed[jp] = 1;
    }
    __syncthreads();
  }
  (void)u11;
  const int r = s_rank;
  // L_r(a, b) = Bh[pr[a], pc[b]] (a > b), U_r(a, b) = Bh[pr[a], pc[b]] (a <= b)
  T* U = (T*)t.U;
  T* V = (T*)t.V;
  for (int x = threadIdx.x; x < t.mx; x += blockDim.x) {
    // c~ U_r = B(x, J_q): c~_b = (B(x, J[pc[b]]) - sum_{a < b} c~_a U_r(a, b)) / U_r(b, b)
    for (int b = 0; b < r; ++b) {
      T v = Bel(x, Jl[pc[b]]);
      for (int a = 0; a < b; ++a) v -= U[x + (size_t)a * t.ldu] * Bh[pr[a] * maxcap + pc[b]];
      U[x + (size_t)b * t.ldu] = v / Bh[pr[b] * maxcap + pc[b]];
    }
  }
  for (int y = threadIdx.x; y < t.my; y += blockDim.x) {
    // L_r w~ = B(I_p, y): w~_a = B(I[pr[a]], y) - sum_{b < a} L_r(a, b) w~_b
    for (int a = 0; a < r; ++a) {
      T v = Bel(Il[pr[a]], y);
      for (int b = 0; b < a; ++b) v -= Bh[pr[a] * maxcap + pc[b]] * V[y + (size_t)b * t.ldv];
      V[y + (size_t)a * t.ldv] = v;
    }
  }
  if (threadIdx.x == 0 && t.rank) *t.rank = r;
}

template <typename T>
void launch_bdlr(const BdlrTask* tasks, int ntasks, int maxnh, int maxcap, int depth, double tol,
                 const int32_t* first, const int* npiv, const int64_t* ifoff, const int32_t* iflist,
                 const int64_t* prowptr, const int32_t* pcol, cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t smem = (size_t)maxcap * maxcap * sizeof(T) + 4 * sizeof(int) * maxcap + 2 * (size_t)maxcap +
                      2 * (size_t)maxnh;
  k_bdlr<T><<<ntasks, 256, smem, s>>>(tasks, depth, tol, first, npiv, ifoff, iflist, prowptr, pcol, maxcap);
}

template <typename T>
void launch_svd(const SvdTask* tasks, int ntasks, int maxk, double tol, cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t smem = ((size_t)2 * maxk * (maxk + 1) + maxk) * sizeof(T);
  k_svd<T><<<ntasks, 512, smem, s>>>(tasks, tol);
}

int dense_comp_setup(int max_smem) {
  HM_CUDA(allow_max_dyn_smem(k_bdlr<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_bdlr<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_qr_smem<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_qr_smem<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_qr_blocked<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_qr_blocked<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_tsqr_blocks<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_tsqr_blocks<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_tsqr_stack<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_tsqr_stack<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_tsqr_q<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_tsqr_q<double>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_svd<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_svd<double>, max_smem));
  return HM_OK;
}

template void launch_omega<float>(const OmegaTask*, int, uint64_t, cudaStream_t);
template void launch_omega<double>(const OmegaTask*, int, uint64_t, cudaStream_t);
template void launch_qr<float>(const QrTask*, int, int, int64_t, int, cudaStream_t);
template void launch_qr<double>(const QrTask*, int, int, int64_t, int, cudaStream_t);
template void launch_tsqr<float>(const TsqrTask*, int, const TsqrBlock*, int, size_t, size_t, float*,
                                 cudaStream_t);
template void launch_tsqr<double>(const TsqrTask*, int, const TsqrBlock*, int, size_t, size_t, double*,
                                  cudaStream_t);
template void launch_svd<float>(const SvdTask*, int, int, double, cudaStream_t);
template void launch_bdlr<float>(const BdlrTask*, int, int, int, int, double, const int32_t*, const int*,
                                 const int64_t*, const int32_t*, const int64_t*, const int32_t*, cudaStream_t);
template void launch_bdlr<double>(const BdlrTask*, int, int, int, int, double, const int32_t*, const int*,
                                  const int64_t*, const int32_t*, const int64_t*, const int32_t*, cudaStream_t);
template void launch_svd<double>(const SvdTask*, int, int, double, cudaStream_t);

}  // namespace hm
