// hm_hodlr_apply.cu -- the preconditioner apply of the HODLR fronts of one tree level in
// one launch per pass (Section 4.2.2: the conventional upward / downward passes with the
// pivot solve replaced by the HODLR solve and F_fp, F_pf by their low-rank forms).
//
// One thread-block cluster of C CTAs (C = 1, 2, 4 or 8) per (front, group of RB
// right-hand sides).  CTA c of the cluster owns the pivot rows of node (lc, c) of the
// front's HODLR tree (lc = log2 C; the tree halves every index range, so the rows of a
// node at depth >= lc never straddle two CTAs) and the update rows [c nu / C,
// (c + 1) nu / C).  Its vectors stay in shared memory for the whole pass; the only
// exchanges are the sums over rows that a node spanning several CTAs needs (t = Z^T y
// in the Woodbury steps, tf = Vtilde^T b_p, tf = W^T x_f): every CTA writes its partial
// sum to its own shared memory, the cluster synchronises, and every CTA adds the
// partials of the node's CTAs in cluster-rank order through distributed shared memory
// (a fixed order, so the result does not depend on timing).
//
//   upward:   fv_q = [r(I_q); 0] (+) children's update parts (relative maps, children
//             in order);  b_f -= W (Vtilde^T b_p)         (Vf^T F_pp^{-1} = Vtilde^T)
//   downward: y = K_leaf^{-1} b_p on the leaves; for depth l = L-1 .. 0 and each node:
//             t = [U^T y_a; V^T y_b], y -= G t  (G = Zhat C^{-1}, formed by the factor);
//             x_p = y + Vtilde (W^T (-x_f))
//
// Every product reads each factor entry once per right-hand-side group, one row per
// thread (consecutive threads, consecutive rows of a column-major block: coalesced),
// or one column per warp for the sums over rows (lanes over rows, then a butterfly of
// shuffles over the warp).
#include <cooperative_groups.h>

#include "hm_internal.h"

namespace cg = cooperative_groups;

namespace hm {

namespace {

constexpr int kHaThreads = 256;  // threads per CTA (an autotuner variant takes 512)

__device__ __forceinline__ int ilog2i(int v) { return 31 - __clz(v); }

// Shared-memory layout (elements of T) of the two kernels; RP = RB + 1 (padded rows).
struct HaLayout {
  int bp, ys, xf, ts, part, part2, tf, total;
};
__host__ __device__ inline HaLayout ha_layout(const HaDims& d, int RB, bool down) {
  const int RP = RB + 1;
  HaLayout L;
  int o = 0;
  L.bp = o; o += d.rowsP * RP;
  L.ys = o; o += down ? d.rowsP * RP : 0;
  L.xf = o; o += d.rowsU * RP;                          // up: f rows; down: -x_f rows
  L.ts = o; o += down ? d.tstore : 0;                    // t of the nodes being processed
  L.part = o; o += down ? 2 * d.kmax * RB : 0;           // cross-CTA partials, two buffers
  L.part2 = o; o += d.kf * RB;                           // this CTA's partial of tf
  L.tf = o; o += d.kf * RB;                              // tf summed over the cluster
  L.total = o;
  return L;
}

// acc[r] = sum over rows rr in [0, cnt) of M[rr] * S[(s0 + rr) * RP + r], one column of M
// per warp (lanes over rows, eight rows per lane in flight), reduced over the warp by a
// butterfly (every lane ends with the sums).  Rows past cnt read row cnt - 1 of S (a
// finite value) against a zero of M.
template <typename T, int RB>
__device__ __forceinline__ void warp_col_dot(const T* __restrict__ M, int cnt, const T* __restrict__ S, int s0,
                                             T (&acc)[RB]) {
  constexpr int RP = RB + 1, U = 8;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < RB; ++r) acc[r] = T(0);
  for (int b = lane; b < cnt; b += 32 * U) {
    T m[U];
#pragma unroll
    for (int u = 0; u < U; ++u) m[u] = b + 32 * u < cnt ? M[b + 32 * u] : T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const T* s = S + (s0 + min(b + 32 * u, cnt - 1)) * RP;
#pragma unroll
      for (int r = 0; r < RB; ++r) acc[r] = fma(m[u], s[r], acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < RB; ++r) acc[r] = warp_sum(acc[r]);
}

// Y[i * RP + r] += sign * sum_{c < ncols} M[i + c ld] * Tsrc(i)[c * RB + r] for the rows i
// of [0, rows) (one row per thread; M's rows start at the CTA's first row; Tsrc(i) is
// the coefficient block of row i's node).
template <typename T, int RB, int NT, typename TSrc>
__device__ __forceinline__ void rows_update(const T* __restrict__ M, int64_t ld, int rows, int ncols, TSrc tsrc,
                                            T* __restrict__ Y, T sign) {
  constexpr int RP = RB + 1, U = 16;  // sixteen loads of M in flight per thread
  for (int i = threadIdx.x; i < rows; i += NT) {
    const T* __restrict__ Tsrc = tsrc(i);
    T acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = T(0);
    int c = 0;
    for (; c + U <= ncols; c += U) {
      T m[U];
#pragma unroll
      for (int u = 0; u < U; ++u) m[u] = M[i + (int64_t)(c + u) * ld];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = fma(m[u], Tsrc[(c + u) * RB + r], acc[r]);
    }
    for (; c < ncols; ++c) {
      const T m = M[i + (int64_t)c * ld];
#pragma unroll
      for (int r = 0; r < RB; ++r) acc[r] = fma(m, Tsrc[c * RB + r], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) Y[i * RP + r] = fma(sign, acc[r], Y[i * RP + r]);
  }
}

// The leaf in [j0, j1) holding row `row` (lb: leaf boundaries, increasing).
__device__ __forceinline__ int leaf_of(const int* __restrict__ lb, int j0, int j1, int row) {
  int lo = j0, hi = j1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (lb[mid] <= row) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// First t in [0, n) with a[t] >= v (a increasing).
__device__ __forceinline__ int lower_bound_i32(const int32_t* __restrict__ a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

}  // namespace

// ------------------------------------------------------------------------------------
// Upward pass of the HODLR fronts of one level.
// ------------------------------------------------------------------------------------
template <typename T, int RB, int NT>
__global__ void __launch_bounds__(NT) k_hodlr_up(
    const HApplyTask* __restrict__ tasks, int C, int nrhs, int n, const T* __restrict__ win,
    const int* __restrict__ npiv, const int* __restrict__ nhat, const int64_t* __restrict__ fvoff,
    const int32_t* __restrict__ child_ptr, const int32_t* __restrict__ child_list,
    const int64_t* __restrict__ ifoff, const int32_t* __restrict__ relmap, const int* __restrict__ leafb,
    const int4* __restrict__ ea, T* __restrict__ FV, HaDims dm) {
  constexpr int RP = RB + 1;
  extern __shared__ __align__(16) unsigned char ha_smem[];
  T* sm = reinterpret_cast<T*>(ha_smem);
  const HaLayout lay = ha_layout(dm, RB, false);
  T* Bp = sm + lay.bp;
  T* Fs = sm + lay.xf;
  T* Part = sm + lay.part2;
  T* tf = sm + lay.tf;
  const int c = (int)(blockIdx.x % (unsigned)C);
  const HApplyTask& tk = tasks[blockIdx.x / C];
  const int r0 = blockIdx.y * RB, nr = min(RB, nrhs - r0);
  const int lc = ilog2i(C);
  const int* lb = leafb + tk.leaf_off;
  const int span = 1 << (tk.L - lc);
  const int P0 = lb[c * span], P1 = lb[(c + 1) * span], nP = P1 - P0;
  const int U0 = (int)((int64_t)tk.nu * c / C), U1 = (int)((int64_t)tk.nu * (c + 1) / C), nU = U1 - U0;
  const int np = tk.np, nh = tk.nhat;
  // [r(I_q); 0] on this CTA's rows
  for (int e = threadIdx.x; e < nP * RB; e += NT) {
    const int i = e % nP, r = e / nP;
    Bp[i * RP + r] = r < nr ? win[tk.first + P0 + i + (int64_t)(r0 + r) * n] : T(0);
  }
  for (int e = threadIdx.x; e < nU * RP; e += NT) Fs[e] = T(0);
  // the children's update parts through the relative maps, one child after another; a
  // relative map is increasing, so the entries that land on this CTA's rows are two
  // contiguous ranges of it
  const int cp0 = child_ptr[tk.q], nch = child_ptr[tk.q + 1] - cp0;
  for (int ci = cp0; ci < cp0 + nch; ++ci) {
    __syncthreads();
    const int ch = child_list[ci];
    const int npc = npiv[ch], nhc = nhat[ch];
    const T* fc = FV + fvoff[ch] + npc;
    const int32_t* rm = relmap + ifoff[ch];
    const int4 rg = ea[tk.ea_off + c * nch + (ci - cp0)];  // formed once per plan
    const int ta = rg.x, tb = rg.y, tc = rg.z, td = rg.w;
    const int na = tb - ta, nb = td - tc;
    const int tot = (na + nb) * nr;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * NT) {  // eight entries per thread in flight
      int d[8], t[8];
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = min(e0 + u * NT, tot - 1), r = e / (na + nb), j = e - r * (na + nb);
        t[u] = j < na ? ta + j : tc + (j - na);
        d[u] = rm[t[u]];
        v[u] = fc[t[u] + (int64_t)(r0 + r) * nhc];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * NT;
        if (e >= tot) continue;
        const int r = e / (na + nb), j = e - r * (na + nb);
        if (j < na) Bp[(d[u] - P0) * RP + r] += v[u];
        else Fs[(d[u] - np - U0) * RP + r] += v[u];
      }
    }
  }
  __syncthreads();
  cg::cluster_group cluster = cg::this_cluster();
  if (tk.kf > 0) {
    // partial tf = Vtilde(rows)^T b_p(rows), one column of Vtilde per warp
    const T* Vt = (const T*)tk.X + P0;
    for (int col = threadIdx.x >> 5; col < tk.kf; col += (NT / 32)) {
      T acc[RB];
      warp_col_dot<T, RB>(Vt + (int64_t)col * np, nP, Bp, 0, acc);
      if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int r = 0; r < RB; ++r) Part[col * RB + r] = acc[r];
      }
    }
    if (C > 1) cluster.sync(); else __syncthreads();
    for (int e = threadIdx.x; e < tk.kf * RB; e += NT) {
      T s = T(0);
      for (int cc = 0; cc < C; ++cc) s += cluster.map_shared_rank(Part, cc)[e];
      tf[e] = s;
    }
    __syncthreads();
    // b_f -= W(rows) tf
    rows_update<T, RB, NT>((const T*)tk.W + U0, tk.nu, nU, tk.kf, [&](int) { return (const T*)tf; }, Fs, T(-1));
    __syncthreads();
  }
  T* fv = FV + tk.fv_off;
  for (int e = threadIdx.x; e < nP * nr; e += NT) {
    const int i = e % nP, r = e / nP;
    fv[P0 + i + (int64_t)(r0 + r) * nh] = Bp[i * RP + r];
  }
  for (int e = threadIdx.x; e < nU * nr; e += NT) {
    const int i = e % nU, r = e / nU;
    fv[np + U0 + i + (int64_t)(r0 + r) * nh] = Fs[i * RP + r];
  }
  if (C > 1 && tk.kf > 0) cluster.sync();  // no CTA leaves while a peer reads its partials
}

// ------------------------------------------------------------------------------------
// Downward pass of the HODLR fronts of one level.
// ------------------------------------------------------------------------------------
template <typename T, int RB, int NT>
__global__ void __launch_bounds__(NT) k_hodlr_down(
    const HApplyTask* __restrict__ tasks, int C, int nrhs, int n, T* __restrict__ xv,
    const int64_t* __restrict__ ifoff, const int32_t* __restrict__ iflist, const int* __restrict__ leafb,
    const T* __restrict__ FV, HaDims dm) {
  constexpr int RP = RB + 1;
  extern __shared__ __align__(16) unsigned char ha_smem[];
  T* sm = reinterpret_cast<T*>(ha_smem);
  const HaLayout lay = ha_layout(dm, RB, true);
  T* Bp = sm + lay.bp;
  T* Ys = sm + lay.ys;
  T* Xf = sm + lay.xf;
  T* Ts = sm + lay.ts;
  T* Part = sm + lay.part;
  T* Part2 = sm + lay.part2;
  T* tf2 = sm + lay.tf;
  const int c = (int)(blockIdx.x % (unsigned)C);
  const HApplyTask& tk = tasks[blockIdx.x / C];
  const int r0 = blockIdx.y * RB, nr = min(RB, nrhs - r0);
  const int lc = ilog2i(C), L = tk.L;
  const int* lb = leafb + tk.leaf_off;
  const int span = 1 << (L - lc);
  const int P0 = lb[c * span], P1 = lb[(c + 1) * span], nP = P1 - P0;
  const int U0 = (int)((int64_t)tk.nu * c / C), U1 = (int)((int64_t)tk.nu * (c + 1) / C), nU = U1 - U0;
  const int np = tk.np, nh = tk.nhat;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // b_p (left by the upward pass) and -x(I_q^f) on this CTA's rows
  const T* fv = FV + tk.fv_off;
  for (int e = threadIdx.x; e < nP * RB; e += NT) {
    const int i = e % nP, r = e / nP;
    Bp[i * RP + r] = r < nr ? fv[P0 + i + (int64_t)(r0 + r) * nh] : T(0);
  }
  // -x(I_q^f): eight indices per thread loaded, then the eight values
  const int32_t* If = iflist + ifoff[tk.q];
  for (int e0 = threadIdx.x; e0 < nU * RB; e0 += 8 * NT) {
    int g[8];
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = min(e0 + u * NT, nU * RB - 1), i = e % nU;
      g[u] = If[U0 + i];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = min(e0 + u * NT, nU * RB - 1), r = e / nU;
      v[u] = r < nr ? -xv[g[u] + (int64_t)(r0 + r) * n] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * NT;
      if (e < nU * RB) Xf[(e % nU) * RP + e / nU] = v[u];
    }
  }
  __syncthreads();
  // this CTA's partial of tf = W^T (-x_f)
  if (tk.kf > 0) {
    const T* Wr = (const T*)tk.W + U0;
    for (int col = warp; col < tk.kf; col += (NT / 32)) {
      T acc[RB];
      warp_col_dot<T, RB>(Wr + (int64_t)col * tk.nu, nU, Xf, 0, acc);
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < RB; ++r) Part2[col * RB + r] = acc[r];
      }
    }
  }
  // leaves: y = K_leaf^{-1} b_p, one row per thread (the leaf's inverse, symmetric, is
  // read by columns: consecutive threads read consecutive rows; packed, ld np)
  const T* F = (const T*)tk.F;
  for (int i = threadIdx.x; i < nP; i += NT) {
    const int j = leaf_of(lb, c * span, (c + 1) * span, P0 + i);
    const int lo = lb[j], nl = lb[j + 1] - lo, ii = P0 + i - lo;
    T acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = T(0);
    const T* K = F + (lo + ii);
    const T* b = Bp + (lo - P0) * RP;
    int jj = 0;
    for (; jj + 16 <= nl; jj += 16) {  // sixteen loads in flight per thread
      T m[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) m[u] = K[(int64_t)(jj + u) * np];
#pragma unroll
      for (int u = 0; u < 16; ++u)
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = fma(m[u], b[(jj + u) * RP + r], acc[r]);
    }
    for (; jj < nl; ++jj) {
      const T m = K[(int64_t)jj * np];
#pragma unroll
      for (int r = 0; r < RB; ++r) acc[r] = fma(m, b[jj * RP + r], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) Ys[i * RP + r] = acc[r];
  }
  __syncthreads();
  cg::cluster_group cluster = cg::this_cluster();
  bool tf_ready = false;
  int buf = 0;
  for (int l = L - 1; l >= 0; --l) {
    const int k = tk.kl[l];
    const T* Bo = (const T*)tk.Bo + (int64_t)tk.col[l] * np;          // U on rows a, V on rows b
    const T* Gl = (const T*)tk.G + (int64_t)2 * (tk.col[l] - tk.kf) * np;
    const int nspan = 1 << (L - l);                                    // leaves per node
    if (l >= lc) {
      // nodes inside this CTA: t = [U^T y_a; V^T y_b] for each, then y -= G t
      const int nn = 1 << (l - lc), n0 = c << (l - lc);
      for (int it = warp; it < nn * 2 * k; it += (NT / 32)) {
        const int ni = it / (2 * k), cc = it - ni * 2 * k;
        const int nd = n0 + ni;
        const int lo = lb[nd * nspan], mid = lb[nd * nspan + nspan / 2], hi = lb[(nd + 1) * nspan];
        const int a = cc < k ? lo : mid, cnt = cc < k ? mid - lo : hi - mid, col = cc < k ? cc : cc - k;
        T acc[RB];
        warp_col_dot<T, RB>(Bo + a + (int64_t)col * np, cnt, Ys, a - P0, acc);
        if (lane == 0) {
#pragma unroll
          for (int r = 0; r < RB; ++r) Ts[(ni * 2 * k + cc) * RB + r] = acc[r];
        }
      }
      __syncthreads();
      const int sh = L - l;
      rows_update<T, RB, NT>(Gl + P0, np, nP, 2 * k,
                         [&](int i) {
                           const int ni = (leaf_of(lb, c * span, (c + 1) * span, P0 + i) >> sh) - n0;
                           return (const T*)(Ts + ni * 2 * k * RB);
                         },
                         Ys, T(-1));
      __syncthreads();
    } else {
      // the node spans 2^(lc - l) CTAs; this CTA's rows lie on one side of its split
      const int g = lc - l, nd = c >> g;
      T* pb = Part + buf * dm.kmax * RB;
      for (int col = warp; col < k; col += (NT / 32)) {
        T acc[RB];
        warp_col_dot<T, RB>(Bo + P0 + (int64_t)col * np, nP, Ys, 0, acc);
        if (lane == 0) {
#pragma unroll
          for (int r = 0; r < RB; ++r) pb[col * RB + r] = acc[r];
        }
      }
      cluster.sync();
      const int cfirst = nd << g, half = 1 << (g - 1);
      for (int e = threadIdx.x; e < 2 * k * RB; e += NT) {
        const int cc = e / RB, r = e - cc * RB, sd = cc < k ? 0 : 1, col = cc - sd * k;
        T s = T(0);
        for (int p = 0; p < half; ++p) s += cluster.map_shared_rank(pb, cfirst + sd * half + p)[col * RB + r];
        Ts[e] = s;
      }
      if (!tf_ready && tk.kf > 0) {
        for (int e = threadIdx.x; e < tk.kf * RB; e += NT) {
          T s = T(0);
          for (int cc = 0; cc < C; ++cc) s += cluster.map_shared_rank(Part2, cc)[e];
          tf2[e] = s;
        }
      }
      tf_ready = true;
      __syncthreads();
      rows_update<T, RB, NT>(Gl + P0, np, nP, 2 * k, [&](int) { return (const T*)Ts; }, Ys, T(-1));
      __syncthreads();
      buf ^= 1;
    }
  }
  if (tk.kf > 0) {
    if (!tf_ready) {  // one CTA per front (or no level spans several): the partial is the sum
      for (int e = threadIdx.x; e < tk.kf * RB; e += NT) tf2[e] = Part2[e];
      __syncthreads();
    }
    // x_p = y + Vtilde tf,  tf = W^T (-x_f)
    rows_update<T, RB, NT>((const T*)tk.X + P0, np, nP, tk.kf, [&](int) { return (const T*)tf2; }, Ys, T(1));
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nP * nr; e += NT) {
    const int i = e % nP, r = e / nP;
    xv[tk.first + P0 + i + (int64_t)(r0 + r) * n] = Ys[i * RP + r];
  }
  if (C > 1) cluster.sync();  // no CTA leaves while a peer reads its partials
}

// The relative map of a child is increasing, so the entries that land on CTA c's pivot
// rows [P0, P1) and update rows np + [U0, U1) are two contiguous ranges of it: found by
// binary search once per plan (one thread per (task, CTA, child)), not in every apply.
__global__ void k_hodlr_child_ranges(const HApplyTask* __restrict__ tasks, int C,
                                     const int32_t* __restrict__ child_ptr, const int32_t* __restrict__ child_list,
                                     const int* __restrict__ npiv, const int* __restrict__ nhat,
                                     const int64_t* __restrict__ ifoff, const int32_t* __restrict__ relmap,
                                     const int* __restrict__ leafb, int4* __restrict__ ea) {
  const HApplyTask& tk = tasks[blockIdx.x];
  const int cp0 = child_ptr[tk.q], nch = child_ptr[tk.q + 1] - cp0;
  const int lc = ilog2i(C);
  const int* lb = leafb + tk.leaf_off;
  const int span = 1 << (tk.L - lc);
  for (int e = threadIdx.x; e < C * nch; e += blockDim.x) {
    const int c = e / nch, ci = e - c * nch;
    const int P0 = lb[c * span], P1 = lb[(c + 1) * span];
    const int U0 = (int)((int64_t)tk.nu * c / C), U1 = (int)((int64_t)tk.nu * (c + 1) / C);
    const int ch = child_list[cp0 + ci];
    const int nuc = nhat[ch] - npiv[ch];
    const int32_t* rm = relmap + ifoff[ch];
    ea[tk.ea_off + e] = make_int4(lower_bound_i32(rm, nuc, P0), lower_bound_i32(rm, nuc, P1),
                                  lower_bound_i32(rm, nuc, tk.np + U0), lower_bound_i32(rm, nuc, tk.np + U1));
  }
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
int hodlr_child_ranges(const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys, SolvePlan* sp) {
  if (!lp.ha_ok || lp.ha_tasks.count == 0) return HM_OK;
  const Plan& P = sys->plan;
  k_hodlr_child_ranges<<<lp.ha_tasks.count, 64, 0, sys->ctx->stream>>>(
      lp.ha_tasks.dev(base), lp.ha_C, sys->d_child_ptr, sys->d_child_list, P.d_np, P.d_nhat, sys->d_ifoff,
      sys->d_relmap, lp.ha_leaf.dev(base), sp->d_ea);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}
size_t hodlr_apply_smem(const HaDims& d, int RB, bool down, int es) {
  return (size_t)ha_layout(d, RB, down).total * es;
}

template <typename T, int RB, int NT>
static cudaError_t launch_rb(bool down, const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys,
                             SolvePlan* sp, int nrhs, const T* win, T* xv, cudaStream_t s) {
  const Plan& P = sys->plan;
  const HaDims& dm = lp.ha_dims;
  const int C = lp.ha_C;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(lp.ha_tasks.count * C), (unsigned)((nrhs + RB - 1) / RB), 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = hodlr_apply_smem(dm, RB, down, (int)sizeof(T));
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const HApplyTask* tasks = lp.ha_tasks.dev(base);
  const int* leafb = lp.ha_leaf.dev(base);
  if (!down)
    return cudaLaunchKernelEx(&cfg, k_hodlr_up<T, RB, NT>, tasks, C, nrhs, sys->n, win, (const int*)P.d_np,
                              (const int*)P.d_nhat, (const int64_t*)sp->d_fvoff, (const int32_t*)sys->d_child_ptr,
                              (const int32_t*)sys->d_child_list, (const int64_t*)sys->d_ifoff,
                              (const int32_t*)sys->d_relmap, leafb, (const int4*)sp->d_ea, (T*)sp->d_fv, dm);
  return cudaLaunchKernelEx(&cfg, k_hodlr_down<T, RB, NT>, tasks, C, nrhs, sys->n, xv, (const int64_t*)sys->d_ifoff,
                            (const int32_t*)sys->d_iflist, leafb, (const T*)sp->d_fv, dm);
}

// nt: threads per CTA, 256, or 512 (for groups of at most four right-hand sides: more
// loads in flight on the few clusters of the top levels)
template <typename T>
int launch_hodlr_apply(bool down, const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys,
                       SolvePlan* sp, int nrhs, const T* win, T* xv, int rb, int nt) {
  cudaStream_t s = sys->ctx->stream;
  cudaError_t e;
  if (nt == 512 && rb <= 4) {
    switch (rb) {
      case 1: e = launch_rb<T, 1, 512>(down, lp, base, sys, sp, nrhs, win, xv, s); break;
      case 2: e = launch_rb<T, 2, 512>(down, lp, base, sys, sp, nrhs, win, xv, s); break;
      default: e = launch_rb<T, 4, 512>(down, lp, base, sys, sp, nrhs, win, xv, s); break;
    }
  } else {
    switch (rb) {
      case 1: e = launch_rb<T, 1, kHaThreads>(down, lp, base, sys, sp, nrhs, win, xv, s); break;
      case 2: e = launch_rb<T, 2, kHaThreads>(down, lp, base, sys, sp, nrhs, win, xv, s); break;
      case 4: e = launch_rb<T, 4, kHaThreads>(down, lp, base, sys, sp, nrhs, win, xv, s); break;
      case 8: e = launch_rb<T, 8, kHaThreads>(down, lp, base, sys, sp, nrhs, win, xv, s); break;
      default: e = launch_rb<T, 16, kHaThreads>(down, lp, base, sys, sp, nrhs, win, xv, s); break;
    }
  }
  HM_CUDA(e);
  return HM_OK;
}
template int launch_hodlr_apply<float>(bool, const LevelSolvePlan&, const unsigned char*, hm_sys_s*, SolvePlan*,
                                       int, const float*, float*, int, int);
template int launch_hodlr_apply<double>(bool, const LevelSolvePlan&, const unsigned char*, hm_sys_s*, SolvePlan*,
                                        int, const double*, double*, int, int);

template <typename T, int RB, int NT>
static int setup_rb(int max_smem) {
  HM_CUDA(allow_max_dyn_smem(k_hodlr_up<T, RB, NT>, max_smem));
  HM_CUDA(allow_max_dyn_smem(k_hodlr_down<T, RB, NT>, max_smem));
  return HM_OK;
}
template <typename T>
static int setup_t(int max_smem) {
  HM_TRY((setup_rb<T, 1, kHaThreads>(max_smem)));
  HM_TRY((setup_rb<T, 2, kHaThreads>(max_smem)));
  HM_TRY((setup_rb<T, 4, kHaThreads>(max_smem)));
  HM_TRY((setup_rb<T, 8, kHaThreads>(max_smem)));
  HM_TRY((setup_rb<T, 16, kHaThreads>(max_smem)));
  HM_TRY((setup_rb<T, 1, 512>(max_smem)));
  HM_TRY((setup_rb<T, 2, 512>(max_smem)));
  HM_TRY((setup_rb<T, 4, 512>(max_smem)));
  return HM_OK;
}
int hodlr_apply_setup(int max_smem) {
  HM_TRY(setup_t<float>(max_smem));
  HM_TRY(setup_t<double>(max_smem));
  return HM_OK;
}

}  // namespace hm
