// hm_api.cu -- the extern "C" boundary (include/hodlr_mf.h) and host utilities.
#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "hm_internal.h"

namespace hm {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

void host_mark(const char* what) {
  static const bool on = getenv("HM_TRACE_HOST") && getenv("HM_TRACE_HOST")[0] == '1';
  if (!on) return;
  using clk = std::chrono::steady_clock;
  static thread_local clk::time_point last = clk::now();
  const clk::time_point now = clk::now();
  fprintf(stderr, "[hm host] %-28s %9.3f ms\n", what,
          std::chrono::duration<double, std::milli>(now - last).count());
  last = now;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

std::unique_lock<std::mutex> alloc_lock(const hm_ctx_s* ctx) {
  return ctx->shared ? std::unique_lock<std::mutex>(ctx->shared->mu) : std::unique_lock<std::mutex>();
}

int dev_alloc_ctx(hm_ctx_s* ctx, std::vector<void*>* owner, void** p, size_t bytes) {
  *p = nullptr;
  bytes = std::max<size_t>(bytes, 16);
  auto lk = alloc_lock(ctx);
  SharedBudget* sb = ctx->shared;
  if (sb && sb->limit && sb->used + bytes > sb->limit) {
    set_last_error("shared HBM budget exceeded: " + std::to_string(sb->used + bytes) + " > " +
                   std::to_string(sb->limit));
    return HM_ERR_OUT_OF_MEMORY;
  }
  if (ctx->opts.hbm_budget && ctx->allocated + bytes > ctx->opts.hbm_budget) {
    set_last_error("HBM budget exceeded: " + std::to_string(ctx->allocated + bytes) + " > " +
                   std::to_string(ctx->opts.hbm_budget));
    return HM_ERR_OUT_OF_MEMORY;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_last_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    return HM_ERR_OUT_OF_MEMORY;
  }
  ctx->allocated += bytes;
  if (sb) sb->used += bytes;
  owner->push_back(*p);
  // remember the size for the budget through a side table
  ctx->allocs.push_back((void*)(uintptr_t)bytes);
  ctx->allocs.push_back(*p);
  return HM_OK;
}

void dev_free_all(hm_ctx_s* ctx, std::vector<void*>* owner) {
  auto lk = alloc_lock(ctx);
  for (void* p : *owner) {
    for (size_t i = 0; i + 1 < ctx->allocs.size(); i += 2) {
      if (ctx->allocs[i + 1] == p) {
        const size_t b = (size_t)(uintptr_t)ctx->allocs[i];
        ctx->allocated -= b;
        if (ctx->shared) ctx->shared->used -= b;
        ctx->allocs.erase(ctx->allocs.begin() + i, ctx->allocs.begin() + i + 2);
        break;
      }
    }
    cudaFreeAsync(p, ctx->stream);
  }
  owner->clear();
}

// Moves an idle system to another context that shares its memory pool and budget: the
// records of all its allocations (factor, plan, apply plans, GMRES workspace) move to
// `to`, whose stream runs the system's later work and frees.  `ready` (may be null) is
// an event recorded on the old context's stream after the system's last work there; it
// is waited for on the host, and nothing is enqueued on the old stream (its owner may
// be capturing a graph on it).  The caller guarantees that no other thread uses the
// system.
int move_sys(hm_sys_s* sys, hm_ctx_s* to, cudaEvent_t ready) {
  hm_ctx_s* from = sys->ctx;
  if (from == to) return HM_OK;
  if (!from->shared || from->shared != to->shared || from->pool != to->pool) {
    set_last_error("move_sys: the contexts do not share a memory pool and budget");
    return HM_ERR_INVALID_ARG;
  }
  if (ready) HM_CUDA(cudaEventSynchronize(ready));
  auto lk = alloc_lock(from);
  auto move = [&](const std::vector<void*>& owner) {
    for (void* p : owner)
      for (size_t i = 0; i + 1 < from->allocs.size(); i += 2) {
        if (from->allocs[i + 1] != p) continue;
        const size_t b = (size_t)(uintptr_t)from->allocs[i];
        from->allocated -= b;
        from->allocs.erase(from->allocs.begin() + i, from->allocs.begin() + i + 2);
        to->allocated += b;
        to->allocs.push_back((void*)(uintptr_t)b);
        to->allocs.push_back(p);
        break;
      }
  };
  move(sys->allocs);
  move(sys->plan_allocs);
  move(sys->gm.allocs);
  for (const auto& kv : sys->solve_plans) move(kv.second->allocs);
  sys->ctx = to;
  return HM_OK;
}

int dev_alloc(hm_sys_s* sys, void** p, size_t bytes) { return dev_alloc_ctx(sys->ctx, &sys->allocs, p, bytes); }

// Bytes of the allocations in `owner` (sizes from the context's side table).
static double owned_bytes(const hm_ctx_s* ctx, const std::vector<void*>& owner) {
  auto lk = alloc_lock(ctx);
  std::unordered_map<const void*, size_t> size;
  for (size_t i = 0; i + 1 < ctx->allocs.size(); i += 2) size[ctx->allocs[i + 1]] = (size_t)(uintptr_t)ctx->allocs[i];
  double b = 0;
  for (const void* p : owner) {
    auto it = size.find(p);
    if (it != size.end()) b += (double)it->second;
  }
  return b;
}

size_t sys_bytes(const hm_sys_s* sys) {
  double b = owned_bytes(sys->ctx, sys->allocs) + owned_bytes(sys->ctx, sys->plan_allocs) +
             owned_bytes(sys->ctx, sys->gm.allocs);
  for (const auto& kv : sys->solve_plans) b += owned_bytes(sys->ctx, kv.second->allocs);
  return (size_t)b;
}

int copy_in(hm_sys_s* sys, void* dst, const void* src, size_t bytes) {
  HM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, sys->ctx->stream));
  HM_CUDA(cudaStreamSynchronize(sys->ctx->stream));
  return HM_OK;
}

int check_device_error(hm_sys_s* sys, const char* where) {
  int h[4] = {0, 0, 0, 0};
  HM_CUDA(cudaMemcpyAsync(h, sys->d_err, sizeof(h), cudaMemcpyDeviceToHost, sys->ctx->stream));
  HM_CUDA(cudaStreamSynchronize(sys->ctx->stream));
  HM_CUDA(cudaGetLastError());
  if (h[0] != 0) {
    set_last_error(std::string(where) + ": device status " + std::to_string(h[0]) + " (" +
                   std::to_string(h[1]) + ", " + std::to_string(h[2]) + ")");
    return h[0];
  }
  return HM_OK;
}

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

cudaEvent_t Tuner::get() {
  if (next < pool.size()) return pool[next++];
  cudaEvent_t e;
  cudaEventCreate(&e);
  pool.push_back(e);
  ++next;
  return e;
}

// Right-hand sides of a tuning pass: a fixed, nonzero pattern.
__global__ void k_tune_rhs(double* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)((uint32_t)(i * 2654435761ull) % 1024u) / 1024.0 - 0.5;
}

const char* prof_cat_name(int c) {
  static const char* names[PC_COUNT] = {
      "nd_order", "symbolic", "permute_csr", "scatter_A", "extend_add", "dense_potrf",
      "dense_trsm", "gemm_factor", "sketch", "householder_qr", "jacobi_svd", "leaf_solve",
      "core_lu_inverse", "spd_inverse", "apply_up", "apply_down", "gemm_apply", "spmv", "gmres_dots",
      "gmres_gs_update", "gmres_small", "vector_ops", "memset", "dense_sweep", "bdlr", "hodlr_apply_up",
      "hodlr_apply_down", "gemm_tensor_core", "pack_factor", "entries_by_depth"};
  return (c >= 0 && c < PC_COUNT) ? names[c] : "?";
}

static void destroy_sys(hm_sys_s* sys) {
  if (!sys) return;
  cudaStreamSynchronize(sys->ctx->stream);
  for (auto& kv : sys->solve_plans) dev_free_all(sys->ctx, &kv.second->allocs);
  sys->solve_plans.clear();
  dev_free_all(sys->ctx, &sys->gm.allocs);
  if (sys->gm.h_res) cudaFreeHost(sys->gm.h_res);
  dev_free_all(sys->ctx, &sys->plan_allocs);
  dev_free_all(sys->ctx, &sys->allocs);
  delete sys;
}

}  // namespace hm

namespace hm {

static int with_device_io(hm_sys_t sys, int nrhs, const double* in, double* out,
                          int (*fn)(hm_sys_t, int, const double*, double*, void*), void* arg) {
  const size_t bytes = sizeof(double) * (size_t)sys->n * nrhs;
  std::vector<void*> tmp;
  const double* din = in;
  double* dout = out;
  const bool out_host = !is_device_ptr(out);
  if (!is_device_ptr(in)) {
    void* p;
    HM_TRY(dev_alloc_ctx(sys->ctx, &tmp, &p, bytes));
    HM_CUDA(cudaMemcpyAsync(p, in, bytes, cudaMemcpyHostToDevice, sys->ctx->stream));
    din = (const double*)p;
  }
  if (out_host) {
    void* p;
    int s = dev_alloc_ctx(sys->ctx, &tmp, &p, bytes);
    if (s != HM_OK) { dev_free_all(sys->ctx, &tmp); return s; }
    dout = (double*)p;
  }
  int st = fn(sys, nrhs, din, dout, arg);
  if (out_host && (st == HM_OK || st == HM_ERR_NO_CONVERGENCE)) {
    cudaError_t e = cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, sys->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sys->ctx->stream);
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); st = HM_ERR_CUDA; }
  }
  cudaStreamSynchronize(sys->ctx->stream);
  dev_free_all(sys->ctx, &tmp);
  return st;
}

struct SolveArgs {
  double rtol;
  int max_iters;
  hm_solve_info* info;
};

struct DirectArgs {
  int refine;
  hm_solve_info* info;
};

static int direct_fn(hm_sys_t sys, int nrhs, const double* b, double* x, void* arg) {
  DirectArgs* a = (DirectArgs*)arg;
  return direct_impl(sys, nrhs, b, a->refine, x, a->info);
}

static int solve_fn(hm_sys_t sys, int nrhs, const double* b, double* x, void* arg) {
  SolveArgs* a = (SolveArgs*)arg;
  return gmres_impl(sys, nrhs, b, a->rtol, a->max_iters, x, a->info);
}

template <typename T>
static int apply_fn_t(hm_sys_t sys, int nrhs, const double* r, double* z) {
  cudaStream_t s = sys->ctx->stream;
  const int n = sys->n;
  const int64_t nn = (int64_t)n * nrhs;
  std::vector<void*> tmp;
  void *rp, *rT, *zT;
  HM_TRY(dev_alloc_ctx(sys->ctx, &tmp, &rp, sizeof(double) * nn));
  HM_TRY(dev_alloc_ctx(sys->ctx, &tmp, &rT, sizeof(T) * nn));
  HM_TRY(dev_alloc_ctx(sys->ctx, &tmp, &zT, sizeof(T) * nn));
  launch_permute_in(r, (double*)rp, sys->d_perm, n, nrhs, s);
  launch_cast_to<T>((const double*)rp, (T*)rT, nn, s);
  int st = apply_impl(sys, nrhs, rT, zT);
  if (st == HM_OK) {
    launch_cast_from<T>((const T*)zT, (double*)rp, nn, s);
    launch_permute_out((const double*)rp, z, sys->d_perm, n, nrhs, s);
    cudaStreamSynchronize(s);
    st = check_device_error(sys, "apply");
  }
  cudaStreamSynchronize(s);
  dev_free_all(sys->ctx, &tmp);
  return st;
}

static int apply_fn(hm_sys_t sys, int nrhs, const double* r, double* z, void*) {
  return sys->precision == HM_PREC_FP64 ? apply_fn_t<double>(sys, nrhs, r, z)
                                        : apply_fn_t<float>(sys, nrhs, r, z);
}

}  // namespace hm

using namespace hm;

extern "C" {

int hm_default_opts(hm_opts* o) {
  if (!o) return HM_ERR_INVALID_ARG;
  memset(o, 0, sizeof(*o));
  o->device = 0;
  o->precision = HM_PREC_MIXED;
  o->nd_leaf = 64;
  o->hodlr_leaf = 64;
  o->n_c = 64;
  o->samples = 48;
  o->seed = 0x5EEDull;
  o->restart = 30;
  o->hbm_budget = 0;
  o->stream = nullptr;
  o->dofs_per_node = 1;
  o->compressor = HM_COMP_RRF;
  o->bdlr_depth = 1;
  o->wait_limit = 0;
  o->adaptive_rank = 0;
  o->inject_wait_timeout = 0;
  o->compress_ff = 0;
  o->keep_fronts = 0;
  return HM_OK;
}

int hm_create(hm_ctx_t* out, const hm_opts* opts) {
  if (!out) return HM_ERR_INVALID_ARG;
  *out = nullptr;
  hm_opts o;
  if (opts) o = *opts; else hm_default_opts(&o);
  if (o.precision != HM_PREC_FP64 && o.precision != HM_PREC_MIXED && o.precision != HM_PREC_MIXED_BF16) {
    set_last_error("precision must be HM_PREC_FP64, HM_PREC_MIXED or HM_PREC_MIXED_BF16");
    return HM_ERR_INVALID_ARG;
  }
  // widest sketch: beyond these widths the factorizations of large fronts (64^3 hex in
  // FP32 at 128, 40^3 hex in FP64 at 80) were measured wrong; the cause is not traced
  const int kmax = o.precision == HM_PREC_FP64 ? 64 : 96;
  if (o.nd_leaf < 1 || o.hodlr_leaf < 2 || o.hodlr_leaf > 64 || o.n_c < 0 || o.n_c > 128 ||
      o.samples < 1 || o.samples > kmax || o.restart < 1 || o.restart > 200 || o.dofs_per_node < 1 ||
      o.dofs_per_node > 8 || (o.compressor != HM_COMP_RRF && o.compressor != HM_COMP_BDLR) ||
      o.bdlr_depth < 1 || o.bdlr_depth > 8 || o.wait_limit < 0 ||
      (o.inject_wait_timeout != 0 && o.inject_wait_timeout != 1) ||
      (o.adaptive_rank != 0 && o.adaptive_rank != 1) || (o.compress_ff != 0 && o.compress_ff != 1) ||
      (o.compress_ff == 1 && o.compressor != HM_COMP_RRF) || (o.keep_fronts != 0 && o.keep_fronts != 1)) {
    set_last_error("option out of range: nd_leaf>=1, 2<=hodlr_leaf<=64, 0<=n_c<=128, "
                   "1<=samples<=" + std::to_string(kmax) + ", 1<=restart<=200, 1<=dofs_per_node<=8, "
                   "compressor RRF or BDLR, 1<=bdlr_depth<=8, wait_limit>=0, adaptive_rank and "
                   "inject_wait_timeout 0 or 1, compress_ff 0 or 1 (range finder only), keep_fronts 0 or 1");
    return HM_ERR_INVALID_ARG;
  }
  int ndev = 0;
  HM_CUDA(cudaGetDeviceCount(&ndev));
  if (o.device < 0 || o.device >= ndev) {
    set_last_error("no such CUDA device");
    return HM_ERR_INVALID_ARG;
  }
  HM_CUDA(cudaSetDevice(o.device));
  hm_ctx_s* ctx = new hm_ctx_s();
  ctx->opts = o;
  if (o.stream) {
    ctx->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      set_last_error("cudaStreamCreate failed");
      return HM_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  {
    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof(pp));
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = o.device;
    if (cudaMemPoolCreate(&ctx->pool, &pp) != cudaSuccess) {
      if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
      delete ctx;
      set_last_error("cudaMemPoolCreate failed");
      return HM_ERR_CUDA;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaDeviceProp prop;
  HM_CUDA(cudaGetDeviceProperties(&prop, o.device));
  ctx->max_smem = (int)prop.sharedMemPerBlockOptin;
  ctx->num_sms = prop.multiProcessorCount;
  int st = dense_fact_setup(ctx->max_smem);
  if (st == HM_OK) st = dense_comp_setup(ctx->max_smem);
  if (st == HM_OK) st = dense_tc_setup(ctx->max_smem);
  if (st == HM_OK) st = gemm_async_setup(ctx->max_smem);
  if (st == HM_OK) st = solve_setup(ctx->max_smem);
  if (st == HM_OK) st = hodlr_apply_setup(ctx->max_smem);
  if (st != HM_OK) {
    cudaMemPoolDestroy(ctx->pool);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return st;
  }
  *out = ctx;
  return HM_OK;
}

int hm_ctx_destroy(hm_ctx_t ctx) {
  if (!ctx) return HM_ERR_INVALID_ARG;
  cudaSetDevice(ctx->opts.device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& r : ctx->prof.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto& e : ctx->prof.pool) cudaEventDestroy(e);
  for (auto& e : ctx->tune.pool) cudaEventDestroy(e);
  if (ctx->pool && ctx->own_pool) {
    cudaStreamSynchronize(ctx->stream);
    cudaMemPoolDestroy(ctx->pool);
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return HM_OK;
}

int hm_analyze(hm_ctx_t ctx, int32_t n, const int64_t* rowptr, const int32_t* colidx, int32_t dim,
               const int32_t* grid_coords, const int32_t* perm_in, int32_t nfronts_in,
               const int32_t* first_in, const int32_t* parent_in, hm_sys_t* out) {
  if (!ctx || !out || n <= 0 || !rowptr || !colidx) {
    set_last_error("hm_analyze: null argument or n <= 0");
    return HM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  cudaSetDevice(ctx->opts.device);
  hm_sys_s* sys = new hm_sys_s();
  sys->ctx = ctx;
  sys->n = n;
  sys->precision = ctx->opts.precision;
  int st = analyze_impl(sys, rowptr, colidx, dim, grid_coords, perm_in, nfronts_in, first_in, parent_in, 1,
                        nullptr);
  if (st != HM_OK) {
    destroy_sys(sys);
    return st;
  }
  *out = sys;
  return HM_OK;
}

int hm_analyze_batch(hm_ctx_t ctx, int32_t n, const int64_t* rowptr, const int32_t* colidx, int32_t dim,
                     const int32_t* grid_coords, int32_t nblocks, const int32_t* block_ptr, hm_sys_t* out) {
  if (!ctx || !out || n <= 0 || !rowptr || !colidx || !grid_coords || nblocks < 1 || !block_ptr) {
    set_last_error("hm_analyze_batch: null argument, n <= 0 or nblocks < 1");
    return HM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  cudaSetDevice(ctx->opts.device);
  hm_sys_s* sys = new hm_sys_s();
  sys->ctx = ctx;
  sys->n = n;
  sys->precision = ctx->opts.precision;
  int st = analyze_impl(sys, rowptr, colidx, dim, grid_coords, nullptr, 0, nullptr, nullptr, nblocks, block_ptr);
  if (st != HM_OK) {
    destroy_sys(sys);
    return st;
  }
  *out = sys;
  return HM_OK;
}

int hm_get_sizes(hm_sys_t sys, int32_t* n, int32_t* nfronts) {
  if (!sys) return HM_ERR_INVALID_ARG;
  if (n) *n = sys->n;
  if (nfronts) *nfronts = sys->nf;
  return HM_OK;
}

int hm_get_ordering(hm_sys_t sys, int32_t* perm, int32_t* first, int32_t* parent, int32_t* level) {
  if (!sys) return HM_ERR_INVALID_ARG;
  cudaSetDevice(sys->ctx->opts.device);
  if (perm) HM_TRY(copy_in(sys, perm, sys->d_perm, sizeof(int32_t) * sys->n));
  if (first) memcpy(first, sys->h_first.data(), sizeof(int32_t) * (sys->nf + 1));
  if (parent) memcpy(parent, sys->h_parent.data(), sizeof(int32_t) * sys->nf);
  if (level) memcpy(level, sys->h_level.data(), sizeof(int32_t) * sys->nf);
  return HM_OK;
}

int hm_get_symbolic(hm_sys_t sys, int32_t* nupd, int64_t* if_off, int32_t* if_list, int32_t* relmap) {
  if (!sys) return HM_ERR_INVALID_ARG;
  cudaSetDevice(sys->ctx->opts.device);
  const int nf = sys->nf;
  std::vector<int64_t> off(nf + 1, 0);
  for (int q = 0; q < nf; ++q) off[q + 1] = off[q] + sys->h_nupd[q];
  if (nupd) memcpy(nupd, sys->h_nupd.data(), sizeof(int32_t) * nf);
  if (if_off) memcpy(if_off, off.data(), sizeof(int64_t) * (nf + 1));
  if (if_list || relmap) {
    std::vector<int32_t> L(std::max<int64_t>(sys->if_total, 1)), R(std::max<int64_t>(sys->if_total, 1));
    HM_TRY(copy_in(sys, L.data(), sys->d_iflist, sizeof(int32_t) * sys->if_total));
    HM_TRY(copy_in(sys, R.data(), sys->d_relmap, sizeof(int32_t) * sys->if_total));
    for (int q = 0; q < nf; ++q) {
      const int64_t src = sys->h_ifoff[q];
      if (if_list) memcpy(if_list + off[q], L.data() + src, sizeof(int32_t) * sys->h_nupd[q]);
      if (relmap) memcpy(relmap + off[q], R.data() + src, sizeof(int32_t) * sys->h_nupd[q]);
    }
  }
  return HM_OK;
}

}  // extern "C"

namespace hm {

// Adaptive rank (the tolerance rule of Section 2.2): a block whose rank reached its
// sketch width was cut by the width, not by tol.  Double the width of every front level
// holding such a block (up to the widest sketch accepted) and factor again, until no
// block is capped or no width can grow; remember the widths for this shape.  FP32 (and
// the BF16 sampling mode) only.
static int grow_widths(hm_sys_s* sys, const double* d_vals, double tol, int* refactor) {
  // the widest sketch hm_create accepts; FP64 systems keep their width: a factorization
  // with grown (per-level, uneven) FP64 widths of the 40^3 elasticity problem read out of
  // bounds, and the cause is not yet found
  if (sys->precision == HM_PREC_FP64) return HM_OK;
  const int kmax = 96;
  for (int round = 0; round < 4; ++round) {
    const Plan& P = sys->plan;
    std::vector<int> r(std::max(P.nrank, 1));
    if (P.nrank) HM_TRY(copy_in(sys, r.data(), sys->d_ranks, sizeof(int) * P.nrank));
    std::vector<int> width = sys->level_width;
    if (width.empty()) width.assign(P.nlevels, sys->ctx->opts.samples);
    std::vector<char> capped(P.nlevels, 0);
    std::vector<int> room(P.nlevels, 0);  // largest block dimension at the level
    for (const auto& h : P.hf) {
      const int l = P.fg[h.q].level;
      if (h.kf > 0) {
        capped[l] |= r[h.rank_slot_f] >= h.kf && h.kf < std::min(h.nu, h.np);
        room[l] = std::max(room[l], std::min(h.nu, h.np));
      }
      for (const auto& nd : h.nodes) {
        const int m = std::min(nd.mid - nd.lo, nd.hi - nd.mid);
        capped[l] |= r[nd.rank_slot] >= nd.kb && nd.kb < m;
        room[l] = std::max(room[l], m);
      }
    }
    bool grow = false;
    for (int l = 0; l < P.nlevels; ++l)
      if (capped[l] && width[l] < std::min(kmax, room[l])) {
        width[l] = std::min(std::min(2 * width[l], kmax), room[l]);
        grow = true;
      }
    if (!grow) break;
    sys->level_width = width;
    HM_TRY(rebuild_plan(sys));
    ++*refactor;
    HM_TRY(factor_impl(sys, d_vals, tol));
  }
  if (!sys->level_width.empty()) sys->ctx->level_widths[sys->shape_sig] = sys->level_width;
  return HM_OK;
}

}  // namespace hm

extern "C" {

int hm_factor(hm_sys_t sys, const double* values, double tol, hm_factor_info* info) {
  if (!sys || !values) return HM_ERR_INVALID_ARG;
  cudaSetDevice(sys->ctx->opts.device);
  sys->factored = false;
  const double* d_vals = values;
  void* tmpv = nullptr;
  std::vector<void*> tmp;
  if (!is_device_ptr(values)) {
    HM_TRY(dev_alloc_ctx(sys->ctx, &tmp, &tmpv, sizeof(double) * sys->nnz));
    HM_CUDA(cudaMemcpyAsync(tmpv, values, sizeof(double) * sys->nnz, cudaMemcpyHostToDevice,
                            sys->ctx->stream));
    d_vals = (const double*)tmpv;
  }
  int st = factor_impl(sys, d_vals, tol);
  int refactor = 0;
  if (st == HM_OK && sys->ctx->opts.adaptive_rank) st = grow_widths(sys, d_vals, tol, &refactor);
  cudaStreamSynchronize(sys->ctx->stream);
  dev_free_all(sys->ctx, &tmp);
  if (st != HM_OK) return st;
  sys->factored = true;
  sys->tol = tol;
  if (info) {
    info->refactorizations = refactor;
    int mw = 0;
    for (const auto& h : sys->plan.hf) {
      mw = std::max(mw, h.kf);
      for (int k : h.kl) mw = std::max(mw, k);
    }
    info->max_width = mw;
    const Plan& P = sys->plan;
    info->nfronts = sys->nf;
    info->nlevels = P.nlevels;
    info->n_hodlr = (int)P.hf.size();
    std::vector<int> r(std::max(P.nrank, 1));
    if (P.nrank) HM_TRY(copy_in(sys, r.data(), sys->d_ranks, sizeof(int) * P.nrank));
    int mx = 0, capped = 0;
    for (const auto& h : P.hf) {
      if (h.kf > 0) {
        mx = std::max(mx, r[h.rank_slot_f]);
        capped += r[h.rank_slot_f] >= h.kf && h.kf < std::min(h.nu, h.np);
      }
      for (const auto& nd : h.nodes) {
        mx = std::max(mx, r[nd.rank_slot]);
        capped += r[nd.rank_slot] >= nd.kb && nd.kb < std::min(nd.mid - nd.lo, nd.hi - nd.mid);
      }
    }
    info->max_rank = mx;
    info->rank_capped = capped;
    info->factor_bytes = P.factor_bytes;
    const int es = sys->precision == HM_PREC_FP64 ? 8 : 4;
    info->front_bytes = (double)P.front_total * es;
    info->stored_bytes = P.stored_bytes;
    // the conventional method on the same tree: L, and in elimination order (children
    // before parents) the peak of L so far + live updates + the current front
    double L = 0, live = 0, peak = 0;
    for (int q = 0; q < sys->nf; ++q) {
      const double np = P.fg[q].np, nu = P.fg[q].nu, nh = P.fg[q].nhat;
      peak = std::max(peak, L + live + nh * (nh + 1) / 2);
      for (int c : sys->children(q)) live -= (double)P.fg[c].nu * (P.fg[c].nu + 1) / 2;
      L += np * (np + 1) / 2 + np * nu;
      live += nu * (nu + 1) / 2;
    }
    peak = std::max(peak, L);
    info->conventional_bytes = L * es;
    info->conventional_peak_bytes = peak * es;
    info->device_bytes = owned_bytes(sys->ctx, sys->allocs) + owned_bytes(sys->ctx, sys->plan_allocs);
    host_mark("factor: info");
  }
  return HM_OK;
}

int hm_autotune(hm_sys_t sys, const double* values, double tol, int32_t nrhs, int32_t reps, int32_t* nsites) {
  if (!sys || !values || nrhs < 1 || nrhs > 64 || reps < 1 || reps > 16) return HM_ERR_INVALID_ARG;
  hm_ctx_s* ctx = sys->ctx;
  if (ctx->prof.on) { set_last_error("hm_autotune while the launch profiler is on"); return HM_ERR_STATE; }
  cudaSetDevice(ctx->opts.device);
  cudaStream_t s = ctx->stream;
  std::vector<void*> tmp;
  const double* d_vals = values;
  void *pv = nullptr, *pb = nullptr, *px = nullptr;
  const int64_t nn = (int64_t)sys->n * nrhs;
  if (!is_device_ptr(values)) {
    HM_TRY(dev_alloc_ctx(ctx, &tmp, &pv, sizeof(double) * sys->nnz));
    HM_CUDA(cudaMemcpyAsync(pv, values, sizeof(double) * sys->nnz, cudaMemcpyHostToDevice, s));
    d_vals = (const double*)pv;
  }
  int st = dev_alloc_ctx(ctx, &tmp, &pb, sizeof(double) * nn);
  if (st == HM_OK) st = dev_alloc_ctx(ctx, &tmp, &px, sizeof(double) * nn);
  if (st != HM_OK) { dev_free_all(ctx, &tmp); return st; }
  k_tune_rhs<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>((double*)pb, nn);
  // every pass: the factorization and two GMRES iterations with all sites forced to one
  // variant; per site the mean time of one launch, the best over the repetitions
  // GEMM sites: five (3 = large SIMT tiles, 4 = tensor cores, where built); the dense
  // apply sites four, the HODLR apply four, panel QR two
  constexpr int kVariants = 5;
  std::unordered_map<uint64_t, std::array<double, kVariants>> best;
  for (int rep = 0; rep < reps && st == HM_OK; ++rep)
    for (int v = 0; v < kVariants && st == HM_OK; ++v) {
      ctx->tune.force = v;
      ctx->tune.rec = true;
      ctx->tune.recs.clear();
      ctx->tune.next = 0;
      st = factor_impl(sys, d_vals, tol);
      if (st == HM_OK) {
        sys->factored = true;
        const int gs = gmres_impl(sys, nrhs, (const double*)pb, 1e-300, 2, (double*)px, nullptr);
        if (gs != HM_OK && gs != HM_ERR_NO_CONVERGENCE) st = gs;
      }
      if (cudaStreamSynchronize(s) != cudaSuccess && st == HM_OK) st = HM_ERR_CUDA;
      if (st != HM_OK) break;
      std::unordered_map<uint64_t, std::pair<double, int>> sum;
      for (const auto& r : ctx->tune.recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
        auto& e = sum[r.key];
        e.first += ms;
        e.second += 1;
      }
      for (const auto& kv : sum) {
        auto it = best.find(kv.first);
        if (it == best.end()) it = best.emplace(kv.first, std::array<double, kVariants>{1e30, 1e30, 1e30, 1e30, 1e30}).first;
        it->second[v] = std::min(it->second[v], kv.second.first / kv.second.second);
      }
    }
  ctx->tune.force = -1;
  ctx->tune.rec = false;
  ctx->tune.recs.clear();
  int tuned = 0;
  if (st == HM_OK) {
    // the default stays unless another variant is clearly faster (3%: timing noise)
    for (const auto& kv : best) {
      int c = 0;
      for (int v = 1; v < kVariants; ++v)
        if (kv.second[v] < 0.97 * kv.second[0] && kv.second[v] < kv.second[c]) c = v;
      ctx->tune.choice[kv.first] = c;
      ++tuned;
    }
    // graphs captured before tuning keep the old variants
    for (auto& kv : sys->solve_plans) {
      SolvePlan* sp = kv.second.get();
      if (sp->graph_exec) cudaGraphExecDestroy(sp->graph_exec);
      sp->graph_exec = nullptr;
      sp->graph_in = nullptr;
      sp->last_in = nullptr;
    }
    st = factor_impl(sys, d_vals, tol);
  }
  cudaStreamSynchronize(s);
  dev_free_all(ctx, &tmp);
  sys->factored = st == HM_OK;
  if (st == HM_OK) sys->tol = tol;
  if (nsites) *nsites = tuned;
  return st;
}

int hm_tune_force(hm_ctx_t ctx, int32_t variant) {
  if (!ctx || variant < -1 || variant > 4) return HM_ERR_INVALID_ARG;
  ctx->tune.force = variant;
  return HM_OK;
}

int hm_solve(hm_sys_t sys, int32_t nrhs, const double* b, double rtol, int32_t max_iters, double* x,
             hm_solve_info* info) {
  if (!sys || !b || !x || nrhs < 1 || nrhs > 64 || max_iters < 0) return HM_ERR_INVALID_ARG;
  if (!sys->factored) { set_last_error("hm_solve before hm_factor"); return HM_ERR_STATE; }
  cudaSetDevice(sys->ctx->opts.device);
  SolveArgs a{rtol, max_iters, info};
  return with_device_io(sys, nrhs, b, x, solve_fn, &a);
}

int hm_direct_solve(hm_sys_t sys, int32_t nrhs, const double* b, int32_t refine, double* x,
                    hm_solve_info* info) {
  if (!sys || !b || !x || nrhs < 1 || nrhs > 64 || refine < 0 || refine > 100) return HM_ERR_INVALID_ARG;
  if (!sys->factored) { set_last_error("hm_direct_solve before hm_factor"); return HM_ERR_STATE; }
  cudaSetDevice(sys->ctx->opts.device);
  DirectArgs a{refine, info};
  return with_device_io(sys, nrhs, b, x, direct_fn, &a);
}

int hm_precond_apply(hm_sys_t sys, int32_t nrhs, const double* r, double* z) {
  if (!sys || !r || !z || nrhs < 1 || nrhs > 64) return HM_ERR_INVALID_ARG;
  if (!sys->factored) { set_last_error("hm_precond_apply before hm_factor"); return HM_ERR_STATE; }
  cudaSetDevice(sys->ctx->opts.device);
  return with_device_io(sys, nrhs, r, z, apply_fn, nullptr);
}

int hm_get_update(hm_sys_t sys, int32_t front, double* U) {
  if (!sys || !U || front < 0 || front >= sys->nf) return HM_ERR_INVALID_ARG;
  if (!sys->factored) return HM_ERR_STATE;
  cudaSetDevice(sys->ctx->opts.device);
  const FrontGeom& g = sys->plan.fg[front];
  if (sys->plan.reuse && g.level > 1) {  // levels 0 and 1 are the last ones in their banks
    set_last_error("hm_get_update: the front storage of depth " + std::to_string(g.level) +
                   " was reused; create the context with keep_fronts = 1");
    return HM_ERR_STATE;
  }
  const int es = sys->precision == HM_PREC_FP64 ? 8 : 4;
  std::vector<unsigned char> buf((size_t)g.nhat * g.nhat * es + 8);
  HM_TRY(copy_in(sys, buf.data(), (char*)sys->d_front + g.off * es, (size_t)g.nhat * g.nhat * es));
  for (int c = 0; c < g.nu; ++c)
    for (int r = 0; r < g.nu; ++r) {
      const size_t idx = (size_t)(g.np + r) + (size_t)(g.np + c) * g.nhat;
      U[r + (size_t)c * g.nu] = es == 8 ? ((double*)buf.data())[idx] : (double)((float*)buf.data())[idx];
    }
  return HM_OK;
}

int hm_get_front_ranks(hm_sys_t sys, int32_t front, int32_t* kind, int32_t* ranks, int32_t* nr) {
  if (!sys || front < 0 || front >= sys->nf) return HM_ERR_INVALID_ARG;
  cudaSetDevice(sys->ctx->opts.device);
  const FrontGeom& g = sys->plan.fg[front];
  if (kind) *kind = g.hodlr >= 0 ? 1 : 0;
  if (g.hodlr < 0) { if (nr) *nr = 0; return HM_OK; }
  const HFront& h = sys->plan.hf[g.hodlr];
  std::vector<int> r(std::max(sys->plan.nrank, 1));
  HM_TRY(copy_in(sys, r.data(), sys->d_ranks, sizeof(int) * sys->plan.nrank));
  int k = 0;
  if (ranks) ranks[k] = h.kf > 0 ? r[h.rank_slot_f] : 0;
  ++k;
  for (const auto& nd : h.nodes) {
    if (ranks) ranks[k] = r[nd.rank_slot];
    ++k;
  }
  if (nr) *nr = k;
  return HM_OK;
}

int hm_get_hodlr_block(hm_sys_t sys, int32_t front, int32_t level, int32_t node, int32_t* m,
                       int32_t* n, int32_t* k, int32_t* rank, double* U, double* V) {
  if (!sys || front < 0 || front >= sys->nf) return HM_ERR_INVALID_ARG;
  if (!sys->factored) return HM_ERR_STATE;
  cudaSetDevice(sys->ctx->opts.device);
  const FrontGeom& g = sys->plan.fg[front];
  if (g.hodlr < 0) { set_last_error("not a HODLR front"); return HM_ERR_INVALID_ARG; }
  const HFront& h = sys->plan.hf[g.hodlr];
  const int es = sys->precision == HM_PREC_FP64 ? 8 : 4;
  int rows_u, rows_v, cols, slot;
  int64_t u_off, v_off, ldu, ldv;
  const void* ubase;
  if (level < 0) {
    rows_u = h.nu; rows_v = h.np; cols = h.kf; slot = h.rank_slot_f;
    ubase = sys->d_w; u_off = h.w_off; ldu = h.nu;
    v_off = h.bo_off; ldv = h.np;
  } else {
    const HNodeGeom* nd = nullptr;
    for (const auto& x : h.nodes)
      if (x.level == level && x.index == node) nd = &x;
    if (!nd) { set_last_error("no such HODLR node"); return HM_ERR_INVALID_ARG; }
    rows_u = nd->mid - nd->lo; rows_v = nd->hi - nd->mid; cols = h.kl[level]; slot = nd->rank_slot;
    ubase = sys->d_bo; u_off = h.bo_off + (int64_t)h.col[level] * h.np + nd->lo; ldu = h.np;
    v_off = h.bo_off + (int64_t)h.col[level] * h.np + nd->mid; ldv = h.np;
  }
  if (m) *m = rows_u;
  if (n) *n = rows_v;
  if (k) *k = cols;
  if (rank) {
    int r = 0;
    if (cols > 0) HM_TRY(copy_in(sys, &r, sys->d_ranks + slot, sizeof(int)));
    *rank = r;
  }
  auto fetch = [&](const void* base, int64_t off, int64_t ld, int rows, double* out) -> int {
    // the block spans (cols - 1) * ld + rows elements from its first entry
    const size_t span = cols > 0 ? (size_t)(cols - 1) * ld + rows : 0;
    std::vector<unsigned char> buf(span * es + 8);
    if (span > 0) HM_TRY(copy_in(sys, buf.data(), (const char*)base + off * es, span * es));
    for (int c = 0; c < cols; ++c)
      for (int r = 0; r < rows; ++r) {
        const size_t i = (size_t)r + (size_t)c * ld;
        out[r + (size_t)c * rows] = es == 8 ? ((double*)buf.data())[i] : (double)((float*)buf.data())[i];
      }
    return HM_OK;
  };
  if (U) HM_TRY(fetch(ubase, u_off, ldu, rows_u, U));
  if (V) HM_TRY(fetch(sys->d_bo, v_off, ldv, rows_v, V));
  return HM_OK;
}

int hm_profile_enable(hm_ctx_t ctx, int enable) {
  if (!ctx) return HM_ERR_INVALID_ARG;
  cudaSetDevice(ctx->opts.device);
  HM_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& r : ctx->prof.recs) {
    ctx->prof.pool.push_back(r.a);
    ctx->prof.pool.push_back(r.b);
  }
  ctx->prof.recs.clear();
  ctx->prof.on = enable != 0;
  return HM_OK;
}

int hm_profile_read(hm_ctx_t ctx, int32_t max_entries, hm_prof_entry* out, int32_t* n) {
  if (!ctx || !n) return HM_ERR_INVALID_ARG;
  cudaSetDevice(ctx->opts.device);
  HM_CUDA(cudaStreamSynchronize(ctx->stream));
  std::vector<hm_prof_entry> agg(PC_COUNT);
  for (int c = 0; c < PC_COUNT; ++c) {
    memset(&agg[c], 0, sizeof(hm_prof_entry));
    strncpy(agg[c].name, prof_cat_name(c), sizeof(agg[c].name) - 1);
  }
  for (const auto& r : ctx->prof.recs) {
    float ms = 0.f;
    HM_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    hm_prof_entry& e = agg[r.cat];
    e.launches += 1;
    e.kernels += r.kernels;
    e.ms += ms;
    e.flops += r.w.flops;
    e.bytes += r.w.bytes;
  }
  int k = 0;
  for (int c = 0; c < PC_COUNT; ++c) {
    if (agg[c].launches == 0) continue;
    if (out && k < max_entries) out[k] = agg[c];
    ++k;
  }
  *n = k;
  return HM_OK;
}

int hm_destroy(hm_sys_t sys) {
  if (!sys) return HM_ERR_INVALID_ARG;
  cudaSetDevice(sys->ctx->opts.device);
  destroy_sys(sys);
  return HM_OK;
}

const char* hm_status_str(int s) {
  switch (s) {
    case HM_OK: return "ok";
    case HM_ERR_INVALID_ARG: return "invalid argument";
    case HM_ERR_NOT_SPD: return "matrix (pivot block) not positive definite";
    case HM_ERR_NO_CONVERGENCE: return "GMRES did not converge";
    case HM_ERR_OUT_OF_MEMORY: return "out of device memory or HBM budget";
    case HM_ERR_CUDA: return "CUDA error";
    case HM_ERR_CAPACITY: return "capacity exceeded";
    case HM_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case HM_ERR_STATE: return "call out of order";
    case HM_ERR_BREAKDOWN: return "breakdown (singular core)";
    default: return "unknown status";
  }
}

const char* hm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
