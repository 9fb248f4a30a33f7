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

template <typename T>
void launch_qr(const QrTask* tasks, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  // dynamic shared memory: tau for up to 256 reflectors
  k_qr<T><<<ntasks, 256, 256 * sizeof(T), s>>>(tasks);
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
  __shared__ int rotated;
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
  // Pairs of columns that are both at rounding level of ||M||_F carry no information
  // (their singular values fall far below any truncation tolerance) and are left alone;
  // rotating them only shuffles rounding noise and keeps the sweeps from converging.
  const T floor2 = block_sum(f2, red) * JacobiEps<T>::v * JacobiEps<T>::v;
  // one 16-lane group per column pair; every group runs the same number of passes so
  // the width-16 shuffles are always executed by full warps
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gl = threadIdx.x & 15, gid = threadIdx.x >> 4, ng = blockDim.x >> 4;
  const int kk = k + (k & 1);
  const int npairs = kk / 2;
  const T eps = JacobiEps<T>::v;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < kk - 1; ++r) {
      for (int base = 0; base < npairs; base += ng) {
        const int pi = base + gid;
        int a = 0, b = 0;
        bool valid = pi < npairs;
        if (valid) {
          a = (pi == 0) ? 0 : 1 + ((pi - 1 + r) % (kk - 1));
          b = 1 + ((kk - 2 - pi + r) % (kk - 1));
          valid = a < k && b < k;
        }
        const int p = min(a, b), q = max(a, b);
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
        if (valid && ga != T(0) && fabs(ga) > eps * sqrt(al * be) && (al > floor2 || be > floor2)) {
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

template <typename T>
void launch_svd(const SvdTask* tasks, int ntasks, int maxk, double tol, cudaStream_t s) {
  if (ntasks <= 0) return;
  const size_t smem = ((size_t)2 * maxk * (maxk + 1) + maxk) * sizeof(T);
  k_svd<T><<<ntasks, 512, smem, s>>>(tasks, tol);
}

int dense_comp_setup(int max_smem) {
  HM_CUDA(allow_max_dyn_smem(k_svd<float>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_svd<double>, max_smem));
  return HM_OK;
}

template void launch_omega<float>(const OmegaTask*, int, uint64_t, cudaStream_t);
template void launch_omega<double>(const OmegaTask*, int, uint64_t, cudaStream_t);
template void launch_qr<float>(const QrTask*, int, cudaStream_t);
template void launch_qr<double>(const QrTask*, int, cudaStream_t);
template void launch_svd<float>(const SvdTask*, int, int, double, cudaStream_t);
template void launch_svd<double>(const SvdTask*, int, int, double, cudaStream_t);

}  // namespace hm
