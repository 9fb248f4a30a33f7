// hm_analyze.cu -- symbolic analysis on the GPU (Section 4.1.1 of the paper):
// nested-dissection ordering and elimination tree, coupling sets S_p (Eq. couplingSet),
// frontal index sets I_p^f and the child-to-parent relative index maps.
#include <algorithm>
#include <climits>

#include "hm_internal.h"

namespace hm {

// One independent block (mesh) of a batched analysis: its lattice box and where its
// unknowns, its tree scratch and its nodes in the forest start.  A single system is one
// block.
struct NdBlock {
  int lo0[3], ext[3];
  int unk_off, n;         // unknowns [unk_off, unk_off + n)
  int node_off, cap;      // tree scratch nodes [node_off, node_off + cap)
  int forest_off, nodes;  // the block's nodes in the forest (set after the tree kernel)
};

// ------------------------------------------------------------------------------------
// Validation of the CSR pattern: monotone row pointers, columns in range, strictly
// increasing within a row.
// ------------------------------------------------------------------------------------
// Block of unknown i: largest b with bp[b] <= i.
__device__ __forceinline__ int block_of(const int32_t* __restrict__ bp, int nblocks, int i) {
  int lo = 0, hi = nblocks;
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (bp[m] <= i) lo = m; else hi = m;
  }
  return lo;
}

// Sorted, in-range column indices; with blocks, every coupling stays inside its block.
__global__ void k_csr_check(const int64_t* rowptr, const int32_t* colidx, int n, const int32_t* bp,
                            int nblocks, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int blk = block_of(bp, nblocks, i);
  const int lo = bp[blk], hi = bp[blk + 1];
  const int64_t b = rowptr[i], e = rowptr[i + 1];
  if (e < b) { raise_error(err, HM_ERR_INVALID_ARG, 1, i); return; }
  int prev = -1;
  for (int64_t k = b; k < e; ++k) {
    const int c = colidx[k];
    if (c < 0 || c >= n || c <= prev) { raise_error(err, HM_ERR_INVALID_ARG, 2, i); return; }
    if (c < lo || c >= hi) { raise_error(err, HM_ERR_INVALID_ARG, 6, i); return; }
    prev = c;
  }
}

// Bounding box of every block: CTA (b, c) reduces chunk c of block b's unknowns.
__global__ void k_bbox(const int32_t* coords, int dim, const int32_t* bp, int chunk, int* bb) {
  const int blk = blockIdx.x;
  const int i0 = bp[blk] + blockIdx.y * chunk, i1 = min(bp[blk + 1], i0 + chunk);
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
    for (int d = 0; d < dim; ++d) {
      const int v = coords[(size_t)i * dim + d];
      lo[d] = min(lo[d], v);
      hi[d] = max(hi[d], v);
    }
  for (int d = 0; d < dim; ++d) {
    lo[d] = -warp_max(-lo[d]);
    hi[d] = warp_max(hi[d]);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&bb[6 * blk + d], lo[d]);
      atomicMax(&bb[6 * blk + 3 + d], hi[d]);
    }
  }
}

// Vector problems: node k's coordinates (those of its first unknown b k); every one of
// its b unknowns must carry the same ones.
__global__ void k_node_coords(const int32_t* coords, int npts, int b, int dim, int32_t* pc, int* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npts) return;
  for (int d = 0; d < dim; ++d) {
    const int32_t v = coords[((size_t)k * b) * dim + d];
    pc[(size_t)k * dim + d] = v;
    for (int c = 1; c < b; ++c)
      if (coords[((size_t)k * b + c) * dim + d] != v) raise_error(err, HM_ERR_INVALID_ARG, 7, k);
  }
}

// Node ordering -> unknown ordering: node j's b unknowns take new indices b j .. b j + b - 1.
__global__ void k_expand_perm(const int32_t* nperm, const int32_t* niperm, int npts, int b, int32_t* perm,
                              int32_t* iperm) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= npts * b) return;
  const int k = u / b, c = u - k * b;
  perm[u] = b * nperm[k] + c;
  iperm[u] = b * niperm[k] + c;
}

// Every lattice point of a block's bounding box must hold exactly one of its unknowns.
__global__ void k_lattice_mark(const int32_t* coords, int n, int dim, const int32_t* bp, int nblocks,
                               const NdBlock* blks, unsigned* bitmap, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const NdBlock bk = blks[block_of(bp, nblocks, i)];
  const int x = coords[(size_t)i * dim] - bk.lo0[0];
  const int y = dim > 1 ? coords[(size_t)i * dim + 1] - bk.lo0[1] : 0;
  const int z = dim > 2 ? coords[(size_t)i * dim + 2] - bk.lo0[2] : 0;
  const int64_t lin = bk.unk_off + (int64_t)x + (int64_t)bk.ext[0] * ((int64_t)y + (int64_t)bk.ext[1] * z);
  const unsigned bit = 1u << (lin & 31);
  if (atomicOr(&bitmap[lin >> 5], bit) & bit) raise_error(err, HM_ERR_INVALID_ARG, 3, i);
}

// ------------------------------------------------------------------------------------
// Nested-dissection box tree, built by one CTA level by level (breadth first).
// Rule: leaf if the box holds <= leaf points or its longest extent is < 3; otherwise
// split the longest axis (lowest axis on ties) at mid = (lo + hi) / 2; the lower half,
// the upper half and then the separator plane are numbered; points within a box or a
// separator lexicographically (x fastest); tree nodes in postorder.
// ------------------------------------------------------------------------------------
struct NdTree {
  int* lo;      // 3 per node
  int* hi;      // 3 per node
  int* axis;    // -1 for a leaf
  int* mid;
  int* left;
  int* right;
  int* par;
  int* depth;
  int* sub;     // nodes in subtree
  int* post;    // postorder id
  int* own;     // first new index of the node's own unknowns
  int* pts;     // first new index of the subtree's unknowns
  int* lvl_ptr; // BFS level boundaries (<= 64 levels)
  int* count;   // [0] nodes, [1] levels
};

// Block b's part of the tree scratch (nodes are numbered within the block).
constexpr int kNdLvlPtr = 70;  // per-block BFS level slots
__host__ __device__ inline NdTree nd_shift(NdTree t, int off, int b) {
  t.lo += 3 * (size_t)off; t.hi += 3 * (size_t)off;
  t.axis += off; t.mid += off; t.left += off; t.right += off; t.par += off; t.depth += off;
  t.sub += off; t.post += off; t.own += off; t.pts += off;
  t.lvl_ptr += kNdLvlPtr * (size_t)b;
  t.count += 2 * (size_t)b;
  return t;
}

__device__ __forceinline__ int64_t box_count(const int* lo, const int* hi, int dim) {
  int64_t c = 1;
  for (int d = 0; d < dim; ++d) c *= (int64_t)(hi[d] - lo[d] + 1);
  return c;
}

__device__ int block_excl_scan(int v, int* total, int* sh) {
  // sh: >= 33 ints; blockDim.x multiple of 32, <= 1024
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sh[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  const int before = wid > 0 ? sh[wid - 1] : 0;
  *total = sh[nw - 1];
  __syncthreads();
  return before + x - v;
}

// One CTA per block; outputs (block-local postorder) at the block's node offset.
__global__ void __launch_bounds__(1024) k_nd_tree(NdTree t0, const NdBlock* blks, int dim, int leaf,
                                                  int* first, int* parent, int* level, int* err) {
  const NdBlock bk = blks[blockIdx.x];
  const NdTree t = nd_shift(t0, bk.node_off, blockIdx.x);
  const int3 ext = make_int3(bk.ext[0], bk.ext[1], bk.ext[2]);
  const int cap = bk.cap;
  first += bk.node_off;
  parent += bk.node_off;
  level += bk.node_off;
  __shared__ int sh[40];
  __shared__ int s_nodes, s_lb, s_le, s_nlev;
  if (threadIdx.x == 0) {
    const int e[3] = {ext.x, ext.y, ext.z};
    for (int d = 0; d < 3; ++d) { t.lo[d] = 0; t.hi[d] = d < dim ? e[d] - 1 : 0; }
    t.par[0] = -1;
    t.depth[0] = 0;
    s_nodes = 1; s_lb = 0; s_le = 1; s_nlev = 0;
    t.lvl_ptr[0] = 0;
  }
  __syncthreads();
  // breadth-first expansion
  while (true) {
    const int lb = s_lb, le = s_le;
    if (lb >= le) break;
    for (int base = lb; base < le; base += blockDim.x) {
      const int v = base + threadIdx.x;
      int split = 0, ax = -1;
      if (v < le) {
        const int* lo = t.lo + 3 * v;
        const int* hi = t.hi + 3 * v;
        int longest = 0;
        for (int d = 0; d < dim; ++d) {
          const int e = hi[d] - lo[d] + 1;
          if (e > longest) { longest = e; ax = d; }
        }
        const int64_t cnt = box_count(lo, hi, dim);
        split = (cnt > leaf && longest >= 3) ? 1 : 0;
        if (!split) ax = -1;
      }
      int total;
      const int pre = block_excl_scan(split, &total, sh);
      const int nodes0 = s_nodes;
      if (v < le) {
        t.axis[v] = ax;
        if (split) {
          const int l = nodes0 + 2 * pre, r = l + 1;
          if (r >= cap) { raise_error(err, HM_ERR_CAPACITY, 10, v); }
          else {
            const int* lo = t.lo + 3 * v;
            const int* hi = t.hi + 3 * v;
            const int m = (lo[ax] + hi[ax]) / 2;
            t.mid[v] = m;
            for (int d = 0; d < 3; ++d) {
              t.lo[3 * l + d] = lo[d]; t.hi[3 * l + d] = hi[d];
              t.lo[3 * r + d] = lo[d]; t.hi[3 * r + d] = hi[d];
            }
            t.hi[3 * l + ax] = m - 1;
            t.lo[3 * r + ax] = m + 1;
            t.par[l] = v; t.par[r] = v;
            t.depth[l] = t.depth[v] + 1; t.depth[r] = t.depth[v] + 1;
            t.left[v] = l; t.right[v] = r;
          }
        } else {
          t.left[v] = -1; t.right[v] = -1; t.mid[v] = 0;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_nodes = nodes0 + 2 * total;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      s_nlev += 1;
      t.lvl_ptr[s_nlev] = le;
      s_lb = le;
      s_le = s_nodes;
      if (s_nlev >= 63 && s_le > s_lb) { raise_error(err, HM_ERR_CAPACITY, 11, 0); s_le = s_lb; }
    }
    __syncthreads();
  }
  const int nnodes = s_nodes, nlev = s_nlev;
  // bottom-up subtree sizes
  for (int L = nlev - 1; L >= 0; --L) {
    for (int v = t.lvl_ptr[L] + threadIdx.x; v < t.lvl_ptr[L + 1]; v += blockDim.x)
      t.sub[v] = t.axis[v] < 0 ? 1 : 1 + t.sub[t.left[v]] + t.sub[t.right[v]];
    __syncthreads();
  }
  // top-down postorder ids and unknown offsets: post[] temporarily holds post_start
  if (threadIdx.x == 0) { t.post[0] = 0; t.pts[0] = 0; }
  __syncthreads();
  for (int L = 0; L < nlev; ++L) {
    for (int v = t.lvl_ptr[L] + threadIdx.x; v < t.lvl_ptr[L + 1]; v += blockDim.x) {
      const int ps = t.post[v], pt = t.pts[v];
      if (t.axis[v] >= 0) {
        const int l = t.left[v], r = t.right[v];
        t.post[l] = ps;
        t.post[r] = ps + t.sub[l];
        t.pts[l] = pt;
        const int64_t cl = box_count(t.lo + 3 * l, t.hi + 3 * l, dim);
        const int64_t cr = box_count(t.lo + 3 * r, t.hi + 3 * r, dim);
        t.pts[r] = pt + (int)cl;
        t.own[v] = pt + (int)(cl + cr);
      } else {
        t.own[v] = pt;
      }
    }
    __syncthreads();
  }
  for (int v = threadIdx.x; v < nnodes; v += blockDim.x) t.post[v] = t.post[v] + t.sub[v] - 1;
  __syncthreads();
  for (int v = threadIdx.x; v < nnodes; v += blockDim.x) {
    const int q = t.post[v];
    first[q] = t.own[v];
    parent[q] = t.par[v] >= 0 ? t.post[t.par[v]] : -1;
    level[q] = t.depth[v];
  }
  if (threadIdx.x == 0) {
    t.count[0] = nnodes;
    t.count[1] = nlev;
  }
}

// New index of every unknown: descend the box tree to the node that owns it.
__global__ void k_nd_perm(const int32_t* coords, int n, int dim, NdTree t0, const int32_t* bp,
                          int nblocks, const NdBlock* blks, int32_t* perm, int32_t* iperm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int blk = block_of(bp, nblocks, i);
  const NdBlock bk = blks[blk];
  const NdTree t = nd_shift(t0, bk.node_off, blk);
  int c[3] = {0, 0, 0};
  c[0] = coords[(size_t)i * dim] - bk.lo0[0];
  if (dim > 1) c[1] = coords[(size_t)i * dim + 1] - bk.lo0[1];
  if (dim > 2) c[2] = coords[(size_t)i * dim + 2] - bk.lo0[2];
  int v = 0;
  for (int guard = 0; guard < 64; ++guard) {
    const int ax = t.axis[v];
    int blo[3], bhi[3];
    for (int d = 0; d < 3; ++d) { blo[d] = t.lo[3 * v + d]; bhi[d] = t.hi[3 * v + d]; }
    bool here = ax < 0;
    if (!here) {
      const int m = t.mid[v];
      if (c[ax] < m) { v = t.left[v]; continue; }
      if (c[ax] > m) { v = t.right[v]; continue; }
      blo[ax] = m; bhi[ax] = m;
      here = true;
    }
    const int e0 = bhi[0] - blo[0] + 1, e1 = bhi[1] - blo[1] + 1;
    const int rank = (c[0] - blo[0]) + e0 * ((c[1] - blo[1]) + e1 * (c[2] - blo[2]));
    const int nw = bk.unk_off + t.own[v] + rank;
    perm[nw] = i;
    iperm[i] = nw;
    return;
  }
}

// The blocks' trees side by side: a forest in postorder (each tree's root last in its
// range, parent -1), first indices shifted by the block's unknown offset.
__global__ void k_nd_forest(const NdBlock* blks, const int* first_t, const int* parent_t, const int* level_t,
                            int32_t* first, int32_t* parent, int32_t* level) {
  const NdBlock bk = blks[blockIdx.x];
  for (int q = blockIdx.y * blockDim.x + threadIdx.x; q < bk.nodes; q += gridDim.y * blockDim.x) {
    const int src = bk.node_off + q, dst = bk.forest_off + q;
    first[dst] = bk.unk_off + first_t[src];
    parent[dst] = parent_t[src] >= 0 ? bk.forest_off + parent_t[src] : -1;
    level[dst] = level_t[src];
  }
}

__global__ void k_iperm(const int32_t* perm, int n, int32_t* iperm, unsigned* bitmap, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int o = perm[i];
  if (o < 0 || o >= n) { raise_error(err, HM_ERR_INVALID_ARG, 4, i); return; }
  const unsigned bit = 1u << (o & 31);
  if (atomicOr(&bitmap[o >> 5], bit) & bit) { raise_error(err, HM_ERR_INVALID_ARG, 5, i); return; }
  iperm[o] = i;
}

__global__ void k_node_of(const int32_t* first, int nf, int n, int32_t* node_of) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = nf;  // largest q with first[q] <= i
  while (hi - lo > 1) {
    const int m = (lo + hi) >> 1;
    if (first[m] <= i) lo = m; else hi = m;
  }
  node_of[i] = lo;
}

// ------------------------------------------------------------------------------------
// Permuted CSR (new numbering), rows sorted; psrc keeps the original entry index.
// ------------------------------------------------------------------------------------
__global__ void k_prow_len(const int64_t* rowptr, const int32_t* perm, int n, int64_t* len) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int o = perm[i];
  len[i] = rowptr[o + 1] - rowptr[o];
}

__global__ void k_scan_local(const int64_t* in, int64_t* out, int64_t* bsum, int n) {
  // 256 threads x 4 items, exclusive scan within the block
  __shared__ int64_t sh[256];
  const int base = blockIdx.x * 1024;
  int64_t v[4], s = 0;
  for (int q = 0; q < 4; ++q) {
    const int i = base + threadIdx.x * 4 + q;
    v[q] = i < n ? in[i] : 0;
    s += v[q];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int64_t y = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += y;
    __syncthreads();
  }
  int64_t run = sh[threadIdx.x] - s;
  for (int q = 0; q < 4; ++q) {
    const int i = base + threadIdx.x * 4 + q;
    if (i < n) out[i] = run;
    run += v[q];
  }
  if (threadIdx.x == 255) bsum[blockIdx.x] = sh[255];
}

__global__ void k_scan_sums(int64_t* bsum, int nb, int64_t* total) {
  if (threadIdx.x != 0) return;
  int64_t run = 0;
  for (int b = 0; b < nb; ++b) {
    const int64_t v = bsum[b];
    bsum[b] = run;
    run += v;
  }
  *total = run;
}

__global__ void k_scan_add(int64_t* out, const int64_t* bsum, int n) {
  const int i = blockIdx.x * 1024 + threadIdx.x;
  for (int q = 0; q < 4; ++q) {
    const int j = i + q * 256;
    if (j < n) out[j] += bsum[blockIdx.x];
  }
}

// out[0..n] exclusive scan of in[0..n-1]; out[n] = total.  tmp holds ceil(n/1024) entries.
static void exclusive_scan(const int64_t* in, int64_t* out, int64_t* tmp, int n, cudaStream_t s) {
  const int nb = (n + 1023) / 1024;
  k_scan_local<<<nb, 256, 0, s>>>(in, out, tmp, n);
  k_scan_sums<<<1, 32, 0, s>>>(tmp, nb, out + n);
  k_scan_add<<<nb, 256, 0, s>>>(out, tmp, n);
}

__global__ void k_prow_fill(const int64_t* rowptr, const int32_t* colidx, const int32_t* perm,
                            const int32_t* iperm, const int64_t* prowptr, int n, int32_t* pcol,
                            int64_t* psrc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int o = perm[i];
  const int64_t b = rowptr[o], e = rowptr[o + 1], pb = prowptr[i];
  for (int64_t k = b; k < e; ++k) {
    const int j = iperm[colidx[k]];
    int64_t pos = pb + (k - b);
    // insertion into the sorted prefix
    while (pos > pb && pcol[pos - 1] > j) {
      pcol[pos] = pcol[pos - 1];
      psrc[pos] = psrc[pos - 1];
      --pos;
    }
    pcol[pos] = j;
    psrc[pos] = k;
  }
}

// ------------------------------------------------------------------------------------
// Frontal index sets of the fronts of one tree level (one CTA per front):
// I_p^f = sorted unique( S_p  U  (U_c I_c^f) ) restricted to indices after I_p, where
// S_p are the graph neighbours of I_p numbered after I_p (Eq. couplingSet).
// Candidates are gathered in shared memory, bitonic-sorted and de-duplicated; the list
// is appended to the I^f arena at an atomically claimed offset.
// ------------------------------------------------------------------------------------
constexpr int kSymCap = 32768;  // largest candidate list (one CTA's shared memory)
constexpr int kSymFast = 2048;  // candidate capacity of the first pass

// I_p^f of front q with a candidate buffer of `cap` entries in shared memory.  Returns
// false (nothing written) if the candidate list does not fit.  Every thread calls it.
__device__ bool symbolic_front(int q, int* buf, int cap, const int32_t* first, const int32_t* child_ptr,
                               const int32_t* child_list, const int64_t* prowptr, const int32_t* pcol,
                               int32_t* nupd, int64_t* ifoff, int32_t* iflist, unsigned long long* cursor,
                               int64_t capacity, int* err) {
  __shared__ int cnt;
  __shared__ int sh[40];
  __shared__ long long s_off;
  const int b = first[q], e = first[q + 1];
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  // S_p candidates
  for (int r = b + (threadIdx.x >> 5); r < e; r += (blockDim.x >> 5)) {
    const int64_t rb = prowptr[r], re = prowptr[r + 1];
    for (int64_t k = rb + (threadIdx.x & 31); k < re; k += 32) {
      const int j = pcol[k];
      if (j >= e) {
        const int pos = atomicAdd(&cnt, 1);
        if (pos < cap) buf[pos] = j;
      }
    }
  }
  // children's update index sets
  for (int c = child_ptr[q]; c < child_ptr[q + 1]; ++c) {
    const int ch = child_list[c];
    const int64_t o = ifoff[ch];
    const int nc = nupd[ch];
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      const int j = iflist[o + t];
      if (j >= e) {
        const int pos = atomicAdd(&cnt, 1);
        if (pos < cap) buf[pos] = j;
      }
    }
  }
  __syncthreads();
  const int total = cnt;
  __syncthreads();  // cnt is reused by the next front of a persistent CTA
  if (total > cap) return false;
  int n2 = 1;
  while (n2 < total) n2 <<= 1;
  for (int t = total + threadIdx.x; t < n2; t += blockDim.x) buf[t] = INT_MAX;
  __syncthreads();
  // bitonic sort ascending
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < n2 / 2; t += blockDim.x) {
        const int lo = 2 * stride * (t / stride) + (t % stride);
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const int a = buf[lo], c = buf[hi];
        if ((a > c) == up) { buf[lo] = c; buf[hi] = a; }
      }
      __syncthreads();
    }
  }
  // unique: each thread handles a contiguous chunk
  const int per = (n2 + blockDim.x - 1) / blockDim.x;
  const int t0 = threadIdx.x * per;
  int mine = 0;
  for (int t = t0; t < min(t0 + per, n2); ++t) {
    const int v = buf[t];
    if (v != INT_MAX && (t == 0 || buf[t - 1] != v)) ++mine;
  }
  int uniq;
  const int pre = block_excl_scan(mine, &uniq, sh);
  if (threadIdx.x == 0) {
    const unsigned long long off = atomicAdd(cursor, (unsigned long long)uniq);
    if ((int64_t)(off + uniq) > capacity) {
      raise_error(err, HM_ERR_CAPACITY, -1, q);
      s_off = -1;
    } else {
      s_off = (long long)off;
    }
    nupd[q] = uniq;
    ifoff[q] = (int64_t)off;
  }
  __syncthreads();
  if (s_off >= 0) {
    int w = pre;
    for (int t = t0; t < min(t0 + per, n2); ++t) {
      const int v = buf[t];
      if (v != INT_MAX && (t == 0 || buf[t - 1] != v)) iflist[s_off + w++] = v;
    }
  }
  __syncthreads();
  return true;
}

// First pass of a level: one CTA per front with a small candidate buffer (many CTAs per
// SM); fronts whose candidates do not fit are queued for the second pass.
__global__ void __launch_bounds__(512) k_symbolic_fast(
    const int* fronts, const int32_t* first, const int32_t* child_ptr, const int32_t* child_list,
    const int64_t* prowptr, const int32_t* pcol, int32_t* nupd, int64_t* ifoff, int32_t* iflist,
    unsigned long long* cursor, int64_t capacity, int* deferred, int* ndeferred, int* err) {
  __shared__ int buf[kSymFast];
  const int q = fronts[blockIdx.x];
  if (!symbolic_front(q, buf, kSymFast, first, child_ptr, child_list, prowptr, pcol, nupd, ifoff, iflist,
                      cursor, capacity, err) &&
      threadIdx.x == 0)
    deferred[atomicAdd(ndeferred, 1)] = q;
}

// Second pass: persistent CTAs with the full buffer take the queued fronts.
__global__ void __launch_bounds__(1024) k_symbolic_slow(
    const int32_t* first, const int32_t* child_ptr, const int32_t* child_list, const int64_t* prowptr,
    const int32_t* pcol, int32_t* nupd, int64_t* ifoff, int32_t* iflist, unsigned long long* cursor,
    int64_t capacity, const int* deferred, const int* ndeferred, int* next, int* err) {
  extern __shared__ int bufl[];
  __shared__ int idx;
  for (;;) {
    if (threadIdx.x == 0) idx = atomicAdd(next, 1);
    __syncthreads();
    const int i = idx;
    __syncthreads();
    if (i >= *ndeferred) return;
    const int q = deferred[i];
    if (!symbolic_front(q, bufl, kSymCap, first, child_ptr, child_list, prowptr, pcol, nupd, ifoff, iflist,
                        cursor, capacity, err) &&
        threadIdx.x == 0)
      raise_error(err, HM_ERR_CAPACITY, q, kSymCap);
  }
}

// Position of each entry of I_c^f inside the parent's front [I_p ; I_p^f].
__global__ void k_relmap(const int32_t* parent, const int32_t* first, const int32_t* nupd,
                         const int64_t* ifoff, const int32_t* iflist, int nf, int32_t* relmap,
                         int* err) {
  const int c = blockIdx.x;
  if (c >= nf) return;
  const int p = parent[c];
  const int64_t oc = ifoff[c];
  const int nc = nupd[c];
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    const int v = iflist[oc + t];
    if (p < 0) { relmap[oc + t] = -1; continue; }
    const int b = first[p], e = first[p + 1];
    int pos;
    if (v < e) {
      pos = v - b;
      if (v < b) raise_error(err, HM_ERR_INVALID_ARG, 20, c);
    } else {
      const int32_t* L = iflist + ifoff[p];
      int lo = 0, hi = nupd[p];
      while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (L[m] < v) lo = m + 1; else hi = m;
      }
      if (lo >= nupd[p] || L[lo] != v) raise_error(err, HM_ERR_INVALID_ARG, 21, c);
      pos = (e - b) + lo;
    }
    relmap[oc + t] = pos;
  }
}

// Destination (element offset in the front arena) of every lower-triangle entry of the
// permuted matrix: entry (i, j), i >= j, belongs to the front owning column j (Eq. fbar);
// -1 for upper-triangle entries.
__global__ void k_amap(const int64_t* prowptr, const int32_t* pcol, const int32_t* node_of,
                       const int32_t* first, const int32_t* nupd, const int64_t* ifoff,
                       const int32_t* iflist, const int64_t* front_off, const int* nhat, int n,
                       int64_t* amap, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t k = prowptr[i]; k < prowptr[i + 1]; ++k) {
    const int j = pcol[k];
    if (j > i) { amap[k] = -1; continue; }
    const int q = node_of[j];
    const int b = first[q], e = first[q + 1];
    const int lc = j - b;
    int lr;
    if (i < e) {
      lr = i - b;
    } else {
      const int32_t* L = iflist + ifoff[q];
      int lo = 0, hi = nupd[q];
      while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (L[m] < i) lo = m + 1; else hi = m;
      }
      if (lo >= nupd[q] || L[lo] != i) { raise_error(err, HM_ERR_INVALID_ARG, 30, i); amap[k] = -1; continue; }
      lr = (e - b) + lo;
    }
    amap[k] = front_off[q] + (int64_t)lr + (int64_t)lc * nhat[q];
  }
}

void launch_amap(hm_sys_s* sys) {
  const int n = sys->n;
  k_amap<<<(n + 255) / 256, 256, 0, sys->ctx->stream>>>(
      sys->d_prowptr, sys->d_pcol, sys->d_node_of, sys->d_first, sys->d_nupd, sys->d_ifoff,
      sys->d_iflist, sys->plan.d_front_off, sys->plan.d_nhat, n, sys->d_amap, sys->d_err);
}

// ------------------------------------------------------------------------------------
// A's lower-triangle entries grouped by the tree depth of their front (a counting sort:
// per block of entries a depth histogram, exclusive offsets depth-major, then placement),
// so that the factorization scatters one level at a time into reused front storage.
// The order within a depth is not fixed, but every entry has its own destination.
// ------------------------------------------------------------------------------------
__global__ void k_lev_count(const int64_t* __restrict__ amap, const int32_t* __restrict__ pcol,
                            const int32_t* __restrict__ node_of, const int* __restrict__ flevel, int64_t nnz,
                            int64_t chunk, int nlev, int64_t* __restrict__ counts) {
  extern __shared__ int hist[];
  for (int i = threadIdx.x; i < nlev; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int64_t b0 = blockIdx.x * chunk, b1 = min(nnz, b0 + chunk);
  for (int64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x)
    if (amap[k] >= 0) atomicAdd(&hist[flevel[node_of[pcol[k]]]], 1);
  __syncthreads();
  for (int i = threadIdx.x; i < nlev; i += blockDim.x) counts[(int64_t)blockIdx.x * nlev + i] = hist[i];
}

// Block l: counts[b][l] becomes the number of depth-l entries of blocks before b (an
// exclusive scan over b, 256 threads, each over a run of consecutive b); range[2 l + 1]
// receives the depth's total.
__global__ void __launch_bounds__(256) k_lev_scan(int64_t* __restrict__ counts, int nb, int nlev,
                                                   int64_t* __restrict__ range) {
  __shared__ int64_t part[256];
  const int l = blockIdx.x, t = threadIdx.x;
  const int run = (nb + 255) / 256, b0 = min(nb, t * run), b1 = min(nb, b0 + run);
  int64_t s = 0;
  for (int b = b0; b < b1; ++b) s += counts[(int64_t)b * nlev + l];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < 256; d <<= 1) {  // inclusive scan of the runs' sums
    const int64_t v = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run0 = t ? part[t - 1] : 0;
  for (int b = b0; b < b1; ++b) {
    const int64_t c = counts[(int64_t)b * nlev + l];
    counts[(int64_t)b * nlev + l] = run0;
    run0 += c;
  }
  if (t == 255) range[2 * l + 1] = part[255];
}

// range[2 l], range[2 l + 1]: the positions of depth l (depths in order).
__global__ void k_lev_ranges(int nlev, int64_t* __restrict__ range) {
  if (threadIdx.x != 0) return;
  int64_t s = 0;
  for (int l = 0; l < nlev; ++l) {
    const int64_t t = range[2 * l + 1];
    range[2 * l] = s;
    s += t;
    range[2 * l + 1] = s;
  }
}

__global__ void k_lev_place(const int64_t* __restrict__ amap, const int64_t* __restrict__ psrc,
                            const int32_t* __restrict__ pcol, const int32_t* __restrict__ node_of,
                            const int* __restrict__ flevel, int64_t nnz, int64_t chunk, int nlev,
                            const int64_t* __restrict__ offs, const int64_t* __restrict__ range,
                            int64_t* __restrict__ src, int64_t* __restrict__ dst) {
  extern __shared__ int cur[];
  for (int i = threadIdx.x; i < nlev; i += blockDim.x) cur[i] = 0;
  __syncthreads();
  const int64_t b0 = blockIdx.x * chunk, b1 = min(nnz, b0 + chunk);
  for (int64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
    const int64_t d = amap[k];
    if (d < 0) continue;
    const int l = flevel[node_of[pcol[k]]];
    const int64_t pos = range[2 * l] + offs[(int64_t)blockIdx.x * nlev + l] + atomicAdd(&cur[l], 1);
    src[pos] = psrc[k];
    dst[pos] = d;
  }
}

static int build_level_scatter(hm_sys_s* sys, const int64_t* d_amap, std::vector<void*>* tmp) {
  cudaStream_t s = sys->ctx->stream;
  const int nlev = sys->plan.nlevels;
  const int64_t nnz = sys->nnz;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((nnz + 2047) / 2048, (int64_t)sys->ctx->num_sms * 8));
  const int64_t chunk = (nnz + nb - 1) / nb;
  int64_t* counts = nullptr;
  HM_TRY(dev_alloc_ctx(sys->ctx, tmp, (void**)&counts, sizeof(int64_t) * (size_t)nb * nlev));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_lev_range, sizeof(int64_t) * 2 * nlev));
  const size_t hs = sizeof(int) * (size_t)nlev;
  if (hs > 48 * 1024) { set_last_error("elimination tree deeper than 12288 levels"); return HM_ERR_CAPACITY; }
  k_lev_count<<<nb, 256, hs, s>>>(d_amap, sys->d_pcol, sys->d_node_of, sys->plan.d_flevel, nnz, chunk, nlev,
                                  counts);
  k_lev_scan<<<nlev, 256, 0, s>>>(counts, nb, nlev, sys->d_lev_range);
  k_lev_ranges<<<1, 32, 0, s>>>(nlev, sys->d_lev_range);
  // (nnz bounds the lower entries; the ranges stay on the device, so no host round trip)
  HM_TRY(dev_alloc(sys, (void**)&sys->d_scat_src, sizeof(int64_t) * std::max<int64_t>(nnz, 1)));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_scat_dst, sizeof(int64_t) * std::max<int64_t>(nnz, 1)));
  k_lev_place<<<nb, 256, hs, s>>>(d_amap, sys->d_psrc, sys->d_pcol, sys->d_node_of, sys->plan.d_flevel, nnz, chunk,
                                  nlev, counts, sys->d_lev_range, sys->d_scat_src, sys->d_scat_dst);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

// ------------------------------------------------------------------------------------
// Host driver of the symbolic analysis.
// ------------------------------------------------------------------------------------
static int tmp_alloc(hm_sys_s* sys, std::vector<void*>* tmp, void** p, size_t bytes) {
  return dev_alloc_ctx(sys->ctx, tmp, p, bytes);
}

int analyze_impl(hm_sys_s* sys, const int64_t* rowptr, const int32_t* colidx, int dim,
                 const int32_t* coords, const int32_t* perm_in, int nfronts_in,
                 const int32_t* first_in, const int32_t* parent_in, int nblocks,
                 const int32_t* block_ptr) {
  cudaStream_t s = sys->ctx->stream;
  const int n = sys->n;
  std::vector<void*> tmp;
  struct Guard {
    hm_ctx_s* ctx;
    std::vector<void*>* t;
    ~Guard() { dev_free_all(ctx, t); }
  } guard{sys->ctx, &tmp};

  host_mark("analyze: enter");
  HM_TRY(dev_alloc(sys, (void**)&sys->d_err, 4 * sizeof(int)));
  HM_CUDA(cudaMemsetAsync(sys->d_err, 0, 4 * sizeof(int), s));
  // pattern
  int64_t ends[2];
  HM_TRY(copy_in(sys, ends, rowptr, sizeof(int64_t)));
  HM_TRY(copy_in(sys, ends + 1, rowptr + n, sizeof(int64_t)));
  if (ends[0] != 0 || ends[1] < n) { set_last_error("rowptr[0] must be 0 and nnz >= n"); return HM_ERR_INVALID_ARG; }
  sys->nnz = ends[1];
  HM_TRY(dev_alloc(sys, (void**)&sys->d_rowptr, sizeof(int64_t) * (n + 1)));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_colidx, sizeof(int32_t) * sys->nnz));
  HM_CUDA(cudaMemcpyAsync(sys->d_rowptr, rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault, s));
  HM_CUDA(cudaMemcpyAsync(sys->d_colidx, colidx, sizeof(int32_t) * sys->nnz, cudaMemcpyDefault, s));
  // independent blocks (one when no batch is given); GMRES runs per block and RHS
  if (nblocks < 1 || (nblocks > 1 && block_ptr == nullptr)) {
    set_last_error("nblocks >= 1 and block_ptr[nblocks + 1] required");
    return HM_ERR_INVALID_ARG;
  }
  sys->h_seg_ptr.assign(nblocks + 1, 0);
  if (block_ptr) HM_TRY(copy_in(sys, sys->h_seg_ptr.data(), block_ptr, sizeof(int32_t) * (nblocks + 1)));
  else sys->h_seg_ptr[1] = n;
  if (sys->h_seg_ptr[0] != 0 || sys->h_seg_ptr[nblocks] != n) {
    set_last_error("block_ptr[0] must be 0 and block_ptr[nblocks] = n");
    return HM_ERR_INVALID_ARG;
  }
  for (int b = 0; b < nblocks; ++b)
    if (sys->h_seg_ptr[b + 1] <= sys->h_seg_ptr[b]) {
      set_last_error("every block needs at least one unknown");
      return HM_ERR_INVALID_ARG;
    }
  sys->nseg = nblocks;
  HM_TRY(dev_alloc(sys, (void**)&sys->d_seg_ptr, sizeof(int32_t) * (nblocks + 1)));
  HM_CUDA(cudaMemcpyAsync(sys->d_seg_ptr, sys->h_seg_ptr.data(), sizeof(int32_t) * (nblocks + 1),
                          cudaMemcpyHostToDevice, s));
  k_csr_check<<<(n + 255) / 256, 256, 0, s>>>(sys->d_rowptr, sys->d_colidx, n, sys->d_seg_ptr, nblocks,
                                              sys->d_err);
  HM_TRY(check_device_error(sys, "analyze: CSR check"));
  host_mark("analyze: CSR check");

  HM_TRY(dev_alloc(sys, (void**)&sys->d_perm, sizeof(int32_t) * n));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_iperm, sizeof(int32_t) * n));
  unsigned* bitmap = nullptr;
  HM_TRY(tmp_alloc(sys, &tmp, (void**)&bitmap, sizeof(unsigned) * ((size_t)n / 32 + 1)));
  HM_CUDA(cudaMemsetAsync(bitmap, 0, sizeof(unsigned) * ((size_t)n / 32 + 1), s));
  int nf = 0;
  if (perm_in == nullptr) {
    if (coords == nullptr || dim < 2 || dim > 3) {
      set_last_error("grid_coords (dim 2 or 3) or a user ordering is required");
      return HM_ERR_INVALID_ARG;
    }
    sys->dim = dim;
    // vector problems: the dissection runs on the nodes (points), b unknowns each
    const int bdof = sys->ctx->opts.dofs_per_node;
    if (n % bdof) { set_last_error("n must be a multiple of dofs_per_node"); return HM_ERR_INVALID_ARG; }
    const int npts = n / bdof;
    std::vector<int> bp(sys->h_seg_ptr.begin(), sys->h_seg_ptr.end());
    for (auto& v : bp) {
      if (v % bdof) { set_last_error("block boundaries must be multiples of dofs_per_node"); return HM_ERR_INVALID_ARG; }
      v /= bdof;
    }
    int32_t* d_segp = sys->d_seg_ptr;
    int32_t* d_coords = nullptr;
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_coords, sizeof(int32_t) * (size_t)n * dim));
    HM_CUDA(cudaMemcpyAsync(d_coords, coords, sizeof(int32_t) * (size_t)n * dim, cudaMemcpyDefault, s));
    int32_t* d_pc = d_coords;  // point coordinates
    int32_t *d_pperm = sys->d_perm, *d_piperm = sys->d_iperm;
    if (bdof > 1) {
      HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_segp, sizeof(int32_t) * bp.size()));
      HM_CUDA(cudaMemcpyAsync(d_segp, bp.data(), sizeof(int32_t) * bp.size(), cudaMemcpyHostToDevice, s));
      HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_pc, sizeof(int32_t) * (size_t)npts * dim));
      HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_pperm, sizeof(int32_t) * (size_t)npts));
      HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_piperm, sizeof(int32_t) * (size_t)npts));
      k_node_coords<<<(npts + 255) / 256, 256, 0, s>>>(d_coords, npts, bdof, dim, d_pc, sys->d_err);
      HM_TRY(check_device_error(sys, "analyze: node coordinates"));
    }
    // bounding box of every block
    int* d_bb = nullptr;
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_bb, 6 * sizeof(int) * (size_t)nblocks));
    std::vector<int> hbb(6 * (size_t)nblocks);
    for (int b = 0; b < nblocks; ++b)
      for (int d = 0; d < 3; ++d) { hbb[6 * b + d] = INT_MAX; hbb[6 * b + 3 + d] = INT_MIN; }
    HM_CUDA(cudaMemcpyAsync(d_bb, hbb.data(), hbb.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    int maxblk = 0;
    for (int b = 0; b < nblocks; ++b) maxblk = std::max(maxblk, bp[b + 1] - bp[b]);
    const int chunk = 256 * 16;
    k_bbox<<<dim3(nblocks, (maxblk + chunk - 1) / chunk), 256, 0, s>>>(d_pc, dim, d_segp, chunk, d_bb);
    HM_CUDA(cudaMemcpyAsync(hbb.data(), d_bb, hbb.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    std::vector<NdBlock> blks(nblocks);
    int node_total = 0;
    for (int b = 0; b < nblocks; ++b) {
      NdBlock& bk = blks[b];
      int64_t cnt = 1;
      for (int d = 0; d < 3; ++d) {
        bk.lo0[d] = d < dim ? hbb[6 * b + d] : 0;
        bk.ext[d] = d < dim ? hbb[6 * b + 3 + d] - hbb[6 * b + d] + 1 : 1;
        cnt *= bk.ext[d];
      }
      bk.unk_off = bp[b];
      bk.n = bp[b + 1] - bp[b];
      if (cnt != bk.n) {
        set_last_error("grid_coords of every block must fill their bounding box exactly");
        return HM_ERR_INVALID_ARG;
      }
      bk.node_off = node_total;
      bk.cap = bk.n + 1;
      node_total += bk.cap;
      bk.forest_off = 0;
      bk.nodes = 0;
    }
    NdBlock* d_blks = nullptr;
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_blks, sizeof(NdBlock) * (size_t)nblocks));
    HM_CUDA(cudaMemcpyAsync(d_blks, blks.data(), sizeof(NdBlock) * (size_t)nblocks, cudaMemcpyHostToDevice, s));
    k_lattice_mark<<<(npts + 255) / 256, 256, 0, s>>>(d_pc, npts, dim, d_segp, nblocks, d_blks, bitmap,
                                                      sys->d_err);
    HM_TRY(check_device_error(sys, "analyze: lattice check"));
    host_mark("analyze: bbox + lattice");
    // trees, one CTA per block
    NdTree t;
    int* tree = nullptr;
    const size_t cap = (size_t)node_total;
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&tree,
                     sizeof(int) * (cap * 16 + (size_t)(kNdLvlPtr + 2) * nblocks + 8)));
    t.lo = tree;
    t.hi = tree + 3 * cap;
    t.axis = tree + 6 * cap;
    t.mid = tree + 7 * cap;
    t.left = tree + 8 * cap;
    t.right = tree + 9 * cap;
    t.par = tree + 10 * cap;
    t.depth = tree + 11 * cap;
    t.sub = tree + 12 * cap;
    t.post = tree + 13 * cap;
    t.own = tree + 14 * cap;
    t.pts = tree + 15 * cap;
    t.lvl_ptr = tree + 16 * cap;
    t.count = tree + 16 * cap + (size_t)kNdLvlPtr * nblocks;
    int *d_first_t = nullptr, *d_parent_t = nullptr, *d_level_t = nullptr;
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_first_t, sizeof(int) * (cap + 1)));
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_parent_t, sizeof(int) * cap));
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_level_t, sizeof(int) * cap));
    {
      ProfScope ps(sys->ctx, PC_ND, Work{0.0, 64.0 * cap});
      k_nd_tree<<<nblocks, 1024, 0, s>>>(t, d_blks, dim, std::max(1, sys->ctx->opts.nd_leaf / bdof), d_first_t,
                                         d_parent_t,
                                         d_level_t, sys->d_err);
    }
    std::vector<int> cnts(2 * (size_t)nblocks);
    HM_CUDA(cudaMemcpyAsync(cnts.data(), t.count, sizeof(int) * cnts.size(), cudaMemcpyDeviceToHost, s));
    HM_TRY(check_device_error(sys, "analyze: nested dissection"));
    host_mark("analyze: nd tree");
    for (int b = 0; b < nblocks; ++b) {
      blks[b].forest_off = nf;
      blks[b].nodes = cnts[2 * b];
      nf += cnts[2 * b];
    }
    HM_CUDA(cudaMemcpyAsync(d_blks, blks.data(), sizeof(NdBlock) * (size_t)nblocks, cudaMemcpyHostToDevice, s));
    int32_t *d_first_f = nullptr, *d_parent_f = nullptr, *d_level_f = nullptr;
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_first_f, sizeof(int32_t) * (nf + 1)));
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_parent_f, sizeof(int32_t) * nf));
    HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_level_f, sizeof(int32_t) * nf));
    {
      ProfScope ps(sys->ctx, PC_ND, Work{0.0, (4.0 * dim + 8.0) * n + 24.0 * nf}, 2);
      int maxnodes = 1;
      for (const auto& bk : blks) maxnodes = std::max(maxnodes, bk.nodes);
      k_nd_forest<<<dim3(nblocks, (maxnodes + 255) / 256), 256, 0, s>>>(d_blks, d_first_t, d_parent_t, d_level_t,
                                                                       d_first_f, d_parent_f, d_level_f);
      k_nd_perm<<<(npts + 255) / 256, 256, 0, s>>>(d_pc, npts, dim, t, d_segp, nblocks, d_blks, d_pperm,
                                                   d_piperm);
      if (bdof > 1)
        k_expand_perm<<<(n + 255) / 256, 256, 0, s>>>(d_pperm, d_piperm, npts, bdof, sys->d_perm, sys->d_iperm);
    }
    sys->h_first.resize(nf + 1);
    sys->h_parent.resize(nf);
    sys->h_level.resize(nf);
    HM_CUDA(cudaMemcpyAsync(sys->h_first.data(), d_first_f, sizeof(int) * nf, cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(sys->h_parent.data(), d_parent_f, sizeof(int) * nf, cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(sys->h_level.data(), d_level_f, sizeof(int) * nf, cudaMemcpyDeviceToHost, s));
    HM_TRY(check_device_error(sys, "analyze: permutation"));
    host_mark("analyze: permutation");
    for (int q = 0; q < nf; ++q) sys->h_first[q] *= bdof;  // points -> unknowns
    sys->h_first[nf] = n;
  } else {
    nf = nfronts_in;
    if (nf <= 0 || first_in == nullptr || parent_in == nullptr) {
      set_last_error("user ordering needs nfronts, first and parent");
      return HM_ERR_INVALID_ARG;
    }
    HM_CUDA(cudaMemcpyAsync(sys->d_perm, perm_in, sizeof(int32_t) * n, cudaMemcpyDefault, s));
    k_iperm<<<(n + 255) / 256, 256, 0, s>>>(sys->d_perm, n, sys->d_iperm, bitmap, sys->d_err);
    sys->h_first.resize(nf + 1);
    sys->h_parent.resize(nf);
    HM_TRY(copy_in(sys, sys->h_first.data(), first_in, sizeof(int32_t) * (nf + 1)));
    HM_TRY(copy_in(sys, sys->h_parent.data(), parent_in, sizeof(int32_t) * nf));
    HM_TRY(check_device_error(sys, "analyze: user permutation"));
    if (sys->h_first[0] != 0 || sys->h_first[nf] != n) { set_last_error("first[0] = 0, first[nf] = n required"); return HM_ERR_INVALID_ARG; }
    for (int q = 0; q < nf; ++q) {
      if (sys->h_first[q + 1] <= sys->h_first[q]) { set_last_error("every tree node needs >= 1 unknown"); return HM_ERR_INVALID_ARG; }
      const int p = sys->h_parent[q];
      if ((q == nf - 1 && p >= 0) || (p >= 0 && (p <= q || p >= nf))) {
        set_last_error("parent[] must list children before parents (postorder; roots have -1)");
        return HM_ERR_INVALID_ARG;
      }
    }
    sys->h_level.assign(nf, 0);
    for (int q = nf - 1; q >= 0; --q)
      sys->h_level[q] = sys->h_parent[q] < 0 ? 0 : sys->h_level[sys->h_parent[q]] + 1;
  }
  sys->nf = nf;
  HM_TRY(dev_alloc(sys, (void**)&sys->d_first, sizeof(int32_t) * (nf + 1)));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_parent, sizeof(int32_t) * nf));
  HM_CUDA(cudaMemcpyAsync(sys->d_first, sys->h_first.data(), sizeof(int32_t) * (nf + 1), cudaMemcpyHostToDevice, s));
  HM_CUDA(cudaMemcpyAsync(sys->d_parent, sys->h_parent.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
  // children (ascending) on host and device
  auto& cptr = sys->h_child_ptr;
  auto& clist = sys->h_child_list;
  cptr.assign(nf + 1, 0);
  for (int q = 0; q < nf; ++q)
    if (sys->h_parent[q] >= 0) cptr[sys->h_parent[q] + 1]++;
  for (int q = 0; q < nf; ++q) cptr[q + 1] += cptr[q];
  clist.assign(std::max(cptr[nf], 1), 0);
  {
    std::vector<int32_t> cur(cptr.begin(), cptr.end() - 1);
    for (int q = 0; q < nf; ++q)  // ascending q: children listed in ascending order
      if (sys->h_parent[q] >= 0) clist[cur[sys->h_parent[q]]++] = q;
  }
  HM_TRY(dev_alloc(sys, (void**)&sys->d_child_ptr, sizeof(int32_t) * (nf + 1)));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_child_list, sizeof(int32_t) * clist.size()));
  HM_CUDA(cudaMemcpyAsync(sys->d_child_ptr, cptr.data(), sizeof(int32_t) * (nf + 1), cudaMemcpyHostToDevice, s));
  HM_CUDA(cudaMemcpyAsync(sys->d_child_list, clist.data(), sizeof(int32_t) * clist.size(), cudaMemcpyHostToDevice, s));
  host_mark("analyze: children");
  HM_TRY(dev_alloc(sys, (void**)&sys->d_node_of, sizeof(int32_t) * n));
  k_node_of<<<(n + 255) / 256, 256, 0, s>>>(sys->d_first, nf, n, sys->d_node_of);
  // permuted CSR
  int64_t* len = nullptr;
  int64_t* bs = nullptr;
  HM_TRY(tmp_alloc(sys, &tmp, (void**)&len, sizeof(int64_t) * n));
  HM_TRY(tmp_alloc(sys, &tmp, (void**)&bs, sizeof(int64_t) * ((size_t)n / 1024 + 2)));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_prowptr, sizeof(int64_t) * (n + 1)));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_pcol, sizeof(int32_t) * sys->nnz));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_psrc, sizeof(int64_t) * sys->nnz));
  {
    ProfScope ps(sys->ctx, PC_PERMUTE_CSR, Work{0.0, 32.0 * n + 16.0 * sys->nnz + 12.0 * sys->nnz}, 5);
    k_prow_len<<<(n + 255) / 256, 256, 0, s>>>(sys->d_rowptr, sys->d_perm, n, len);
    exclusive_scan(len, sys->d_prowptr, bs, n, s);
    k_prow_fill<<<(n + 255) / 256, 256, 0, s>>>(sys->d_rowptr, sys->d_colidx, sys->d_perm, sys->d_iperm,
                                                sys->d_prowptr, n, sys->d_pcol, sys->d_psrc);
  }
  // symbolic, level by level (deepest first)
  int maxlev = 0;
  for (int q = 0; q < nf; ++q) maxlev = std::max(maxlev, sys->h_level[q]);
  std::vector<int> order;
  std::vector<int> lvl_begin(maxlev + 2, 0);
  {
    std::vector<std::vector<int>> by(maxlev + 1);
    for (int q = 0; q < nf; ++q) by[sys->h_level[q]].push_back(q);
    for (int l = maxlev; l >= 0; --l) {
      lvl_begin[maxlev - l] = (int)order.size();
      for (int q : by[l]) order.push_back(q);
    }
    lvl_begin[maxlev + 1] = (int)order.size();
  }
  int* d_order = nullptr;
  HM_TRY(tmp_alloc(sys, &tmp, (void**)&d_order, sizeof(int) * order.size()));
  HM_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, s));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_nupd, sizeof(int32_t) * nf));
  HM_TRY(dev_alloc(sys, (void**)&sys->d_ifoff, sizeof(int64_t) * (nf + 1)));
  unsigned long long* cursor = nullptr;
  HM_TRY(tmp_alloc(sys, &tmp, (void**)&cursor, sizeof(unsigned long long)));
  HM_CUDA(cudaFuncSetAttribute(k_symbolic_slow, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSymCap * (int)sizeof(int)));  // 128 KB + < 1 KB static
  // per level: deferred-front count and queue cursor, then the queue itself
  int* dq = nullptr;
  HM_TRY(tmp_alloc(sys, &tmp, (void**)&dq, sizeof(int) * (2 * (size_t)(maxlev + 1) + nf)));
  int64_t capacity = (int64_t)32 * n + 65536;
  for (int attempt = 0; attempt < 4; ++attempt) {
    HM_TRY(dev_alloc(sys, (void**)&sys->d_iflist, sizeof(int32_t) * capacity));
    HM_CUDA(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s));
    HM_CUDA(cudaMemsetAsync(sys->d_err, 0, 4 * sizeof(int), s));
    HM_CUDA(cudaMemsetAsync(dq, 0, sizeof(int) * 2 * (size_t)(maxlev + 1), s));
    int* queue = dq + 2 * (maxlev + 1);
    for (int L = 0; L <= maxlev; ++L) {
      const int cntL = lvl_begin[L + 1] - lvl_begin[L];
      if (cntL == 0) continue;
      ProfScope ps(sys->ctx, PC_SYMBOLIC, Work{}, 2);
      k_symbolic_fast<<<cntL, 512, 0, s>>>(d_order + lvl_begin[L], sys->d_first, sys->d_child_ptr,
                                            sys->d_child_list, sys->d_prowptr, sys->d_pcol, sys->d_nupd,
                                            sys->d_ifoff, sys->d_iflist, cursor, capacity, queue,
                                            dq + 2 * L, sys->d_err);
      k_symbolic_slow<<<std::min(cntL, sys->ctx->num_sms), 1024, kSymCap * sizeof(int), s>>>(
          sys->d_first, sys->d_child_ptr, sys->d_child_list, sys->d_prowptr, sys->d_pcol, sys->d_nupd,
          sys->d_ifoff, sys->d_iflist, cursor, capacity, queue, dq + 2 * L, dq + 2 * L + 1, sys->d_err);
    }
    int herr[4];
    HM_CUDA(cudaMemcpyAsync(herr, sys->d_err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    HM_CUDA(cudaGetLastError());
    if (herr[0] == HM_ERR_CAPACITY && herr[1] == -1) {  // arena too small: grow and retry
      capacity *= 4;
      continue;
    }
    if (herr[0] != 0) return check_device_error(sys, "analyze: symbolic");
    break;
  }
  host_mark("analyze: symbolic");
  unsigned long long total = 0;
  HM_CUDA(cudaMemcpyAsync(&total, cursor, sizeof(total), cudaMemcpyDeviceToHost, s));
  sys->h_nupd.resize(nf);
  sys->h_ifoff.resize(nf + 1);
  HM_CUDA(cudaMemcpyAsync(sys->h_nupd.data(), sys->d_nupd, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaMemcpyAsync(sys->h_ifoff.data(), sys->d_ifoff, sizeof(int64_t) * nf, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  sys->if_total = (int64_t)total;
  sys->h_ifoff[nf] = (int64_t)total;
  HM_TRY(dev_alloc(sys, (void**)&sys->d_relmap, sizeof(int32_t) * std::max<int64_t>(total, 1)));
  {
    ProfScope ps(sys->ctx, PC_SYMBOLIC, Work{0.0, 12.0 * total});
    k_relmap<<<nf, 256, 0, s>>>(sys->d_parent, sys->d_first, sys->d_nupd, sys->d_ifoff, sys->d_iflist, nf,
                                sys->d_relmap, sys->d_err);
  }
  HM_TRY(check_device_error(sys, "analyze: relative maps"));
  host_mark("analyze: relative maps");
  {
    // shape signature of the analysis: sketch widths learned by the adaptive rank rule
    // for the same shape (and precision) are reused
    uint64_t h = 0x9E3779B97F4A7C15ull ^ (uint64_t)sys->n ^ ((uint64_t)sys->nf << 32) ^ (uint64_t)sys->precision;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 0x100000001B3ull; h ^= h >> 29; };
    for (int q = 0; q < sys->nf; ++q)
      mix(((uint64_t)(sys->h_first[q + 1] - sys->h_first[q]) << 40) ^ ((uint64_t)sys->h_nupd[q] << 8) ^
          (uint64_t)sys->h_level[q]);
    sys->shape_sig = h;
    auto it = sys->ctx->level_widths.find(h);
    sys->level_width = it != sys->ctx->level_widths.end() ? it->second : std::vector<int>();
  }
  HM_TRY(build_plan(sys));
  host_mark("analyze: build_plan");
  // the assembly map is needed only to group the entries by depth
  HM_TRY(tmp_alloc(sys, &tmp, (void**)&sys->d_amap, sizeof(int64_t) * sys->nnz));
  {
    ProfScope ps(sys->ctx, PC_SYMBOLIC, Work{0.0, 24.0 * sys->nnz});
    launch_amap(sys);
  }
  HM_TRY(check_device_error(sys, "analyze: assembly map"));
  host_mark("analyze: assembly map");
  {
    ProfScope ps(sys->ctx, PC_GROUP, Work{0.0, 48.0 * sys->nnz}, 4);
    HM_TRY(build_level_scatter(sys, sys->d_amap, &tmp));
  }
  sys->d_amap = nullptr;  // freed with the analysis temporaries
  host_mark("analyze: entries by depth");
  return check_device_error(sys, "analyze: entries by depth");
}

}  // namespace hm
