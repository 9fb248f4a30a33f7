// hm_server.cu -- serving runtime: a request loop over many matrices that keeps their
// factorizations resident on the device, batches the right-hand sides that wait for the
// same matrix into one multi-RHS solve (continuous batching), admits work by an HBM
// budget, and overlaps the work of different matrices on the device.
//
// Design.  The server owns W worker threads, each with its own context (CUDA stream and
// stream-ordered memory pool, budget = total budget / W).  A matrix is bound to one
// worker when it is registered (round robin), so its system (analysis, factors, apply
// plans, GMRES workspace) lives in that worker's context and every call on it comes
// from that thread.  Workers run concurrently, so solves of matrices on different
// workers overlap on the GPU.  A worker takes the oldest waiting request, joins every
// other waiting request for the same matrix (in arrival order, up to max_batch_rhs
// right-hand sides in all) and solves them in one hm_solve: each right-hand side is its
// own GMRES instance, so a request's answer does not depend on its companions beyond
// rounding.  The first request for a matrix analyses and factors it (a miss); the
// system then stays resident until evicted.  Admission: when an allocation of the
// worker's context would exceed its budget, the least recently used resident system of
// that worker is destroyed and the step retried; a matrix that does not fit alone fails
// its requests with HM_ERR_OUT_OF_MEMORY.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "hm_internal.h"

namespace hm {

using Clock = std::chrono::steady_clock;

struct SrvMatrix {
  int n = 0, dim = 0, worker = 0;
  double tol = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colidx, coords;
  std::vector<double> values;
  hm_sys_t sys = nullptr;       // resident system (worker-owned), or null
  size_t bytes = 0;             // device bytes while resident
  int64_t last_use = 0;         // worker-local use counter (LRU)
};

struct SrvRequest {
  int64_t id = 0;
  int matrix = 0, nrhs = 0;
  const double* b = nullptr;
  double* x = nullptr;
  double rtol = 1e-10;
  Clock::time_point t_submit, t_done;
  bool done = false;
  int status = HM_OK;
  hm_solve_info info{};
  int batch_rhs = 0;  // right-hand sides in the solve that served it
};

struct SrvWorker {
  hm_ctx_t ctx = nullptr;
  std::thread th;
  std::deque<SrvRequest*> q;
  int64_t clock = 0;
  SrvMatrix* last = nullptr;  // matrix of the previous batch
};

}  // namespace hm

struct hm_server_s {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int max_batch_rhs = 64;
  std::vector<hm::SrvWorker> workers;
  std::vector<std::unique_ptr<hm::SrvMatrix>> matrices;  // stable addresses
  std::vector<std::unique_ptr<hm::SrvRequest>> requests;  // index = id
  std::vector<double> latency_ms;
  int64_t completed = 0, failed = 0, batches = 0, batched_rhs = 0, factorizations = 0, evictions = 0;
};

namespace hm {

static size_t ctx_bytes(hm_ctx_t ctx) { return ctx->allocated; }

// Destroys the least recently used resident system of worker w (not `keep`); false if
// there is none.  Only worker w creates or destroys its systems.
static bool evict_one(hm_server_s* S, int w, int keep) {
  SrvMatrix* victim = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (int m = 0; m < (int)S->matrices.size(); ++m) {
      SrvMatrix* M = S->matrices[m].get();
      if (M->worker != w || !M->sys || m == keep) continue;
      if (!victim || M->last_use < victim->last_use) victim = M;
    }
    if (!victim) return false;
    S->evictions++;
  }
  hm_destroy(victim->sys);
  victim->sys = nullptr;
  victim->bytes = 0;
  if (S->workers[w].last == victim) S->workers[w].last = nullptr;
  return true;
}

// Makes matrix m resident on worker w (analyze + factor), evicting on budget misses.
static int make_resident(hm_server_s* S, int w, int m, SrvMatrix& M) {
  if (M.sys) return HM_OK;
  hm_ctx_t ctx = S->workers[w].ctx;
  for (;;) {
    const size_t before = ctx_bytes(ctx);
    hm_sys_t sys = nullptr;
    int st = hm_analyze(ctx, M.n, M.rowptr.data(), M.colidx.data(), M.dim, M.coords.data(), nullptr, 0,
                        nullptr, nullptr, &sys);
    if (st == HM_OK) {
      hm_factor_info fi;
      st = hm_factor(sys, M.values.data(), M.tol, &fi);
      if (st != HM_OK) hm_destroy(sys);
    }
    if (st == HM_OK) {
      M.sys = sys;
      M.bytes = ctx_bytes(ctx) - before;
      std::lock_guard<std::mutex> lk(S->mu);
      S->factorizations++;
      return HM_OK;
    }
    if (st != HM_ERR_OUT_OF_MEMORY || !evict_one(S, w, m)) return st;
  }
}

static void worker_loop(hm_server_s* S, int w) {
  SrvWorker& W = S->workers[w];
  cudaSetDevice(W.ctx->opts.device);
  std::vector<double> B, X;
  for (;;) {
    std::vector<SrvRequest*> batch;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !W.q.empty(); });
      if (W.q.empty()) return;  // stopping and drained
      // continuous batching: the oldest request and every later one for its matrix
      const int m = W.q.front()->matrix;
      int rhs = 0;
      for (auto it = W.q.begin(); it != W.q.end();) {
        SrvRequest* r = *it;
        if (r->matrix == m && (batch.empty() || rhs + r->nrhs <= S->max_batch_rhs)) {
          batch.push_back(r);
          rhs += r->nrhs;
          it = W.q.erase(it);
        } else {
          ++it;
        }
      }
    }
    const int m = batch.front()->matrix;
    SrvMatrix* Mp;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      Mp = S->matrices[m].get();
    }
    SrvMatrix& M = *Mp;
    // one system's transient solve state (apply plans, GMRES workspace) per worker
    if (W.last && W.last != Mp && W.last->sys) release_solve_state(W.last->sys);
    W.last = Mp;
    int st = make_resident(S, w, m, M);
    int nrhs = 0;
    double rtol = 1.0;
    for (SrvRequest* r : batch) { nrhs += r->nrhs; rtol = std::min(rtol, r->rtol); }
    hm_solve_info info{};
    if (st == HM_OK) {
      M.last_use = ++W.clock;
      const size_t n = (size_t)M.n;
      B.assign(n * nrhs, 0.0);
      X.assign(n * nrhs, 0.0);
      int c = 0;
      for (SrvRequest* r : batch) {
        std::copy(r->b, r->b + n * r->nrhs, B.begin() + n * c);
        c += r->nrhs;
      }
      // The GMRES workspace grows with n x right-hand sides ((2 restart + 6) FP64 vectors
      // per column); columns are solved in chunks that keep it within a quarter of the
      // worker's budget, so large systems do not evict their neighbours for workspace.
      const hm_opts& o = W.ctx->opts;
      int chunk = nrhs;
      if (o.hbm_budget) {
        const double per_col = (2.0 * o.restart + 6.0) * 8.0 * (double)n;
        chunk = std::max(1, std::min(nrhs, (int)(0.25 * (double)o.hbm_budget / per_col)));
      }
      info.converged = 1;
      for (int c0 = 0; c0 < nrhs && (st == HM_OK || st == HM_ERR_NO_CONVERGENCE); c0 += chunk) {
        const int nc = std::min(chunk, nrhs - c0);
        hm_solve_info ci{};
        int cs = hm_solve(M.sys, nc, B.data() + n * c0, rtol, 4000, X.data() + n * c0, &ci);
        while (cs == HM_ERR_OUT_OF_MEMORY && evict_one(S, w, m))  // workspace: make room
          cs = hm_solve(M.sys, nc, B.data() + n * c0, rtol, 4000, X.data() + n * c0, &ci);
        if (st == HM_OK) st = cs;
        info.iters = std::max(info.iters, ci.iters);
        info.restarts = std::max(info.restarts, ci.restarts);
        info.relres = std::max(info.relres, ci.relres);
        info.converged = info.converged && ci.converged;
      }
      if (st == HM_OK || st == HM_ERR_NO_CONVERGENCE) {
        c = 0;
        for (SrvRequest* r : batch) {
          std::copy(X.begin() + n * c, X.begin() + n * (c + r->nrhs), r->x);
          c += r->nrhs;
        }
      }
    }
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    S->batches++;
    S->batched_rhs += nrhs;
    for (SrvRequest* r : batch) {
      r->status = st;
      r->info = info;
      r->batch_rhs = nrhs;
      r->t_done = now;
      r->done = true;
      if (st == HM_OK) {
        S->completed++;
        S->latency_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
      } else {
        S->failed++;
      }
    }
    S->cv_done.notify_all();
  }
}

static double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t i = (size_t)std::min<double>((double)v.size() - 1, std::max(0.0, p * (double)(v.size() - 1) + 0.5));
  return v[i];
}

}  // namespace hm

using namespace hm;

extern "C" {

int hm_server_create(const hm_opts* opts, int32_t nworkers, int32_t max_batch_rhs, hm_server_t* out) {
  if (!out || nworkers < 1 || nworkers > 16 || max_batch_rhs < 1 || max_batch_rhs > 64) {
    set_last_error("hm_server_create: need 1 <= nworkers <= 16 and 1 <= max_batch_rhs <= 64");
    return HM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  hm_opts o;
  if (opts) o = *opts; else hm_default_opts(&o);
  o.stream = nullptr;  // every worker owns its stream
  if (o.hbm_budget) o.hbm_budget /= (size_t)nworkers;
  hm_server_s* S = new hm_server_s();
  S->max_batch_rhs = max_batch_rhs;
  S->workers.resize(nworkers);
  for (int w = 0; w < nworkers; ++w) {
    const int st = hm_create(&S->workers[w].ctx, &o);
    if (st != HM_OK) {
      for (int v = 0; v < w; ++v) hm_ctx_destroy(S->workers[v].ctx);
      delete S;
      return st;
    }
  }
  for (int w = 0; w < nworkers; ++w) S->workers[w].th = std::thread(worker_loop, S, w);
  *out = S;
  return HM_OK;
}

int hm_server_add_matrix(hm_server_t S, int32_t n, const int64_t* rowptr, const int32_t* colidx,
                         const double* values, int32_t dim, const int32_t* grid_coords, double tol,
                         int32_t* matrix_id) {
  if (!S || n <= 0 || !rowptr || !colidx || !values || !grid_coords || dim < 2 || dim > 3 || !matrix_id) {
    set_last_error("hm_server_add_matrix: null argument, n <= 0 or dim not 2/3");
    return HM_ERR_INVALID_ARG;
  }
  SrvMatrix M;
  M.n = n;
  M.dim = dim;
  M.tol = tol;
  M.rowptr.assign(rowptr, rowptr + n + 1);
  const int64_t nnz = M.rowptr[n];
  if (M.rowptr[0] != 0 || nnz < n) {
    set_last_error("hm_server_add_matrix: rowptr[0] must be 0 and nnz >= n");
    return HM_ERR_INVALID_ARG;
  }
  M.colidx.assign(colidx, colidx + nnz);
  M.values.assign(values, values + nnz);
  M.coords.assign(grid_coords, grid_coords + (size_t)n * dim);
  std::lock_guard<std::mutex> lk(S->mu);
  M.worker = (int)(S->matrices.size() % S->workers.size());
  S->matrices.push_back(std::make_unique<SrvMatrix>(std::move(M)));
  *matrix_id = (int32_t)S->matrices.size() - 1;
  return HM_OK;
}

int hm_server_submit(hm_server_t S, int32_t matrix_id, int32_t nrhs, const double* b, double* x, double rtol,
                     int64_t* request_id) {
  if (!S || !b || !x || !request_id || nrhs < 1) {
    set_last_error("hm_server_submit: null argument or nrhs < 1");
    return HM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (matrix_id < 0 || matrix_id >= (int)S->matrices.size() || nrhs > S->max_batch_rhs) {
    set_last_error("hm_server_submit: unknown matrix or nrhs above max_batch_rhs");
    return HM_ERR_INVALID_ARG;
  }
  auto r = std::make_unique<SrvRequest>();
  r->id = (int64_t)S->requests.size();
  r->matrix = matrix_id;
  r->nrhs = nrhs;
  r->b = b;
  r->x = x;
  r->rtol = rtol;
  r->t_submit = Clock::now();
  S->workers[S->matrices[matrix_id]->worker].q.push_back(r.get());
  *request_id = r->id;
  S->requests.push_back(std::move(r));
  S->cv_work.notify_all();
  return HM_OK;
}

int hm_server_wait(hm_server_t S, int64_t request_id, hm_solve_info* info, double* latency_ms,
                   int32_t* batch_rhs) {
  if (!S) return HM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (request_id < 0 || request_id >= (int64_t)S->requests.size()) {
    set_last_error("hm_server_wait: unknown request");
    return HM_ERR_INVALID_ARG;
  }
  SrvRequest* r = S->requests[request_id].get();
  S->cv_done.wait(lk, [&] { return r->done; });
  if (info) *info = r->info;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  if (batch_rhs) *batch_rhs = r->batch_rhs;
  return r->status;
}

int hm_server_get_stats(hm_server_t S, hm_server_stats* st) {
  if (!S || !st) return HM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  st->completed = S->completed;
  st->failed = S->failed;
  st->batches = S->batches;
  st->batched_rhs = S->batched_rhs;
  st->factorizations = S->factorizations;
  st->evictions = S->evictions;
  st->p50_ms = percentile(S->latency_ms, 0.50);
  st->p99_ms = percentile(S->latency_ms, 0.99);
  size_t resident = 0;
  for (auto& W : S->workers) resident += W.ctx->allocated;
  st->device_bytes = (double)resident;
  return HM_OK;
}

int hm_server_destroy(hm_server_t S) {
  if (!S) return HM_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  for (auto& W : S->workers)
    if (W.th.joinable()) W.th.join();
  // the worker threads are gone: free every resident system and context from here
  for (auto& M : S->matrices)
    if (M->sys) {
      cudaSetDevice(S->workers[M->worker].ctx->opts.device);
      hm_destroy(M->sys);
    }
  for (auto& W : S->workers) hm_ctx_destroy(W.ctx);
  delete S;
  return HM_OK;
}

}  // extern "C"
