// hm_server.cu -- serving runtime: a request loop over many matrices that keeps their
// factorizations resident on the device, solves the right-hand sides of one matrix
// together and lets new ones join a running solve (continuous batching), admits work by
// an HBM budget, and overlaps the work of different matrices on the device.
//
// Design.  The server owns W worker threads, each with its own context (CUDA stream);
// the contexts share one stream-ordered memory pool and one HBM budget, so memory one
// worker frees is the next one's to use, and a matrix may take the whole budget.
// Requests wait in one queue.  A free worker takes the oldest waiting request whose
// matrix no worker holds (a matrix resident on another worker that is idle is left to
// that worker, which keeps the matrix's solve state).  A matrix that is not resident is
// analysed and factored by the worker that takes it (a miss); one that is resident on
// another worker moves to the taker's context (its solve state is dropped, its
// factorization stays where it is in the pool).  The worker then runs a GMRES session
// over a fixed number of slots (right-hand-side columns, each its own GMRES instance):
// every waiting request for the matrix that fits the free slots is put in, and after
// each restart cycle the converged requests leave (their answers are returned at once)
// and newly arrived requests for the matrix take the free slots.  A request therefore
// never waits for a running solve of its matrix to finish, and its answer is the one it
// gets alone (each column has its own Krylov space and its own restart boundaries).
// Workers run concurrently, so solves of different matrices overlap on the GPU.
// Admission by estimate: before a matrix is analysed and factored (and before a
// session's GMRES workspace is allocated), the worker destroys the least recently used
// resident systems that no worker holds (of any worker) until the bytes held plus the
// estimate fit the budget.  The estimate of a matrix is the footprint it had when last
// resident (plus an eighth), else the bytes per nonzero of the largest matrix of its
// dimension seen so far (a fixed per-nonzero figure before any); a session's is its
// slots times the GMRES and apply vectors per column (plus a quarter and 4 MiB).  Should
// the estimate fall short, the allocation that exceeds the budget fails and the step is
// retried after one more eviction (counted as oom_retries).  With nothing left to evict
// while other workers run sessions, the worker waits for one of them to end (meanwhile
// running sessions take no new requests, so they end); a matrix that does not fit with
// every other session gone fails with HM_ERR_OUT_OF_MEMORY.
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
  int n = 0, dim = 0;
  int worker = -1;              // worker whose context holds the resident system (-1: none)
  int serving = -1;             // worker holding it now: session, move, eviction or release
  double tol = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colidx, coords;
  std::vector<double> values;
  hm_sys_t sys = nullptr;       // resident system (worker-owned), or null
  size_t bytes = 0;             // device bytes while resident
  size_t bytes_seen = 0;        // footprint when last resident (0: never)
  int64_t nnz = 0;
  int64_t last_use = 0;         // server-wide use counter (LRU)
  cudaEvent_t ready = nullptr;  // recorded on the holder's stream when it lets go of the system
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
  bool busy = false;          // between taking a request and the end of its session
  SrvMatrix* last = nullptr;  // matrix whose solve state this worker keeps (its last session)
};

}  // namespace hm

struct hm_server_s {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int max_batch_rhs = 64;
  std::deque<hm::SrvRequest*> q;   // waiting requests, in arrival order
  std::vector<hm::SrvWorker> workers;
  std::vector<std::unique_ptr<hm::SrvMatrix>> matrices;  // stable addresses
  std::vector<std::unique_ptr<hm::SrvRequest>> requests;  // index = id
  std::vector<double> latency_ms;
  int64_t completed = 0, failed = 0, batches = 0, batched_rhs = 0, factorizations = 0, evictions = 0;
  int64_t joined = 0;  // requests that entered a running session
  int64_t oom_retries = 0;  // budget misses the estimate did not foresee
  int64_t moved = 0;        // resident systems moved to another worker's context
  int64_t memory_waits = 0; // waits for another worker's session to end, for memory
  int64_t clock = 0;        // use counter (LRU)
  int in_session = 0;       // workers inside a GMRES session
  int mem_waiters = 0;      // workers waiting for memory (sessions take no joiners then)
  int64_t sessions_ended = 0;
  hm::SharedBudget budget;  // shared by the workers' contexts (one memory pool)
};

namespace hm {

// Device bytes the workers hold together.
static size_t held_bytes(hm_server_s* S) {
  std::lock_guard<std::mutex> lk(S->budget.mu);
  return S->budget.used;
}

// Destroys the least recently used resident system that no worker holds (any worker's;
// not matrix `keep`); false if there is none.  The caller (worker w) holds no lock.
static bool evict_one(hm_server_s* S, int w, int keep) {
  SrvMatrix* victim = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (int m = 0; m < (int)S->matrices.size(); ++m) {
      SrvMatrix* M = S->matrices[m].get();
      if (M->serving >= 0 || !M->sys || m == keep) continue;
      if (!victim || M->last_use < victim->last_use) victim = M;
    }
    if (!victim) return false;
    victim->serving = w;  // held while it is destroyed
    if (S->workers[victim->worker].last == victim) S->workers[victim->worker].last = nullptr;
    S->evictions++;
  }
  // the system moves to this worker first: its frees then run on this worker's own
  // stream (another worker's stream may be capturing a graph); a system that cannot move
  // stays resident where it is
  if (move_sys(victim->sys, S->workers[w].ctx, victim->ready) != HM_OK) {
    std::lock_guard<std::mutex> lk(S->mu);
    victim->serving = -1;
    S->evictions--;
    S->cv_work.notify_all();
    return false;
  }
  hm_destroy(victim->sys);
  std::lock_guard<std::mutex> lk(S->mu);
  victim->sys = nullptr;
  victim->bytes = 0;
  victim->worker = -1;
  victim->serving = -1;
  S->cv_work.notify_all();  // requests for it may be taken again
  return true;
}

// After an allocation failed with nothing left to evict: waits until a session of
// another worker ends and returns true, or returns false at once when no other worker
// is in a session (then the work does not fit the budget).  While a worker waits,
// running sessions take no new requests, so they end.
static bool wait_for_memory(hm_server_s* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->in_session == 0) return false;
  const int64_t ended = S->sessions_ended;
  S->mem_waiters++;
  S->memory_waits++;
  S->cv_done.wait(lk, [&] { return S->sessions_ended != ended; });
  S->mem_waiters--;
  return true;
}

// Estimated device bytes of matrix M when resident (see the header comment).
static size_t estimate_bytes(hm_server_s* S, const SrvMatrix& M) {
  if (M.bytes_seen) return M.bytes_seen + M.bytes_seen / 8;  // an eighth to spare
  std::lock_guard<std::mutex> lk(S->mu);
  // the bytes per nonzero of the largest matrix of the same dimension seen so far (small
  // systems carry fixed costs that would overstate a large one)
  double per_nnz = M.dim == 3 ? 1024.0 : 512.0;
  int64_t best = 0;
  for (const auto& o : S->matrices)
    if (o->bytes_seen && o->dim == M.dim && o->nnz > best) {
      per_nnz = (double)o->bytes_seen / (double)o->nnz;
      best = o->nnz;
    }
  return (size_t)(per_nnz * (double)M.nnz);
}

// Evicts least recently used idle systems (not m) until `need` more bytes fit the
// budget (or nothing is left to evict).
static void admit(hm_server_s* S, int w, int m, size_t need) {
  const size_t budget = S->budget.limit;
  if (!budget) return;
  while (held_bytes(S) + need > budget && evict_one(S, w, m)) {
  }
}

// Retries `step` (an allocating step of worker w for matrix m) after one more eviction,
// or after another worker's session ended, while it fails for lack of memory.
template <class F>
static int with_memory(hm_server_s* S, int w, int m, F step) {
  for (;;) {
    const int st = step();
    if (st != HM_ERR_OUT_OF_MEMORY) return st;
    if (!evict_one(S, w, m) && !wait_for_memory(S)) return st;
    std::lock_guard<std::mutex> lk(S->mu);
    S->oom_retries++;
  }
}

// Makes matrix m resident on worker w (analyze + factor), admitted by its estimate.
static int make_resident(hm_server_s* S, int w, int m, SrvMatrix& M) {
  if (M.sys) return HM_OK;
  hm_ctx_t ctx = S->workers[w].ctx;
  admit(S, w, m, estimate_bytes(S, M));
  return with_memory(S, w, m, [&]() -> int {
    hm_sys_t sys = nullptr;
    hm_factor_info fi;
    int st = hm_analyze(ctx, M.n, M.rowptr.data(), M.colidx.data(), M.dim, M.coords.data(), nullptr, 0,
                        nullptr, nullptr, &sys);
    if (st == HM_OK) {
      st = hm_factor(sys, M.values.data(), M.tol, &fi);
      if (st != HM_OK) hm_destroy(sys);
    }
    if (st != HM_OK) return st;
    const size_t bytes = sys_bytes(sys);
    std::lock_guard<std::mutex> lk(S->mu);
    M.sys = sys;
    M.bytes = bytes;
    M.bytes_seen = M.bytes;
    S->factorizations++;
    return HM_OK;
  });
}

// Completes request r (status st; x already written) under the server lock.
static void finish(hm_server_s* S, SrvRequest* r, int st, const hm_solve_info& info, int batch_rhs) {
  r->status = st;
  r->info = info;
  r->batch_rhs = batch_rhs;
  r->t_done = Clock::now();
  r->done = true;
  if (st == HM_OK) {
    S->completed++;
    S->latency_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
  } else {
    S->failed++;
  }
}

// Moves the waiting requests for matrix m (arrival order) that fit `free_slots` from the
// queue into `out`; the caller holds the lock.
static void take_requests(hm_server_s* S, int m, int free_slots, std::vector<SrvRequest*>* out) {
  for (auto it = S->q.begin(); it != S->q.end() && free_slots > 0;) {
    SrvRequest* r = *it;
    if (r->matrix == m && r->nrhs <= free_slots) {
      out->push_back(r);
      free_slots -= r->nrhs;
      it = S->q.erase(it);
    } else {
      ++it;
    }
  }
}

// A GMRES session on matrix M: requests join at restart boundaries, leave when done.
// Every request the session takes is appended to `owned`: the caller fails those still
// open if the session returns an error.  `entered` is set once the session counts in
// in_session; the caller ends it there after releasing the matrix.
static int run_session(hm_server_s* S, int w, int m, SrvMatrix& M, std::vector<SrvRequest*>& owned,
                       bool* entered) {
  const std::vector<SrvRequest*> first = owned;
  int rhs0 = 0;
  for (SrvRequest* r : first) rhs0 += r->nrhs;
  // slots: room for about as many joiners as the session starts with, within the GMRES
  // workspace a quarter of a worker's share of the budget allows ((2 restart + 6) FP64
  // vectors each)
  int slots = 1;
  while (slots < std::min(2 * rhs0, S->max_batch_rhs)) slots *= 2;
  slots = std::min(slots, S->max_batch_rhs);
  const hm_opts& o = S->workers[w].ctx->opts;
  if (S->budget.limit) {
    const double per_col = (2.0 * o.restart + 6.0) * 8.0 * (double)M.n;
    slots = std::max(rhs0 > 0 ? std::min(rhs0, S->max_batch_rhs) : 1,
                     std::min(slots, (int)(0.25 * (double)S->budget.limit / S->workers.size() / per_col)));
  }
  // the session's GMRES workspace (V, Z and the work vectors of every slot) and its apply
  // buffers, admitted by estimate (with a quarter and 4 MiB to spare) before allocation
  admit(S, w, m, (size_t)(1.25 * ((2.0 * o.restart + 10.0) * 8.0 * (double)M.n * slots) + (4u << 20)));
  HM_TRY(with_memory(S, w, m, [&] { return gm_session_begin(M.sys, slots); }));
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_session++;  // until the worker releases the matrix (workers short of memory wait)
    *entered = true;
  }
  struct Live { SrvRequest* r; int slot0; };
  std::vector<Live> live;
  std::vector<char> used(slots, 0);
  const size_t n = (size_t)M.n;
  auto put = [&](SrvRequest* r) -> int {
    int s0 = -1;  // first run of r->nrhs free slots
    for (int k = 0; k + r->nrhs <= slots && s0 < 0; ++k) {
      bool ok = true;
      for (int c = 0; c < r->nrhs; ++c) ok = ok && !used[k + c];
      if (ok) s0 = k;
    }
    if (s0 < 0) return HM_ERR_CAPACITY;
    for (int c = 0; c < r->nrhs; ++c) {
      HM_TRY(gm_session_put(M.sys, s0 + c, r->b + n * c, r->rtol, 4000));
      used[s0 + c] = 1;
    }
    live.push_back(Live{r, s0});
    return HM_OK;
  };
  int total_rhs = 0;
  for (SrvRequest* r : first) {
    HM_TRY(put(r));
    total_rhs += r->nrhs;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->batches++;
    S->batched_rhs += total_rhs;
  }
  while (!live.empty()) {
    int its = 0;
    HM_TRY(gm_session_cycle(M.sys, &its));
    // requests whose every column converged (or hit its cap) leave
    std::vector<std::pair<SrvRequest*, std::pair<int, hm_solve_info>>> done;
    for (size_t i = 0; i < live.size();) {
      SrvRequest* r = live[i].r;
      bool all = true, conv = true;
      hm_solve_info info{};
      info.converged = 1;
      for (int c = 0; c < r->nrhs; ++c) {
        double rr = 0;
        int it = 0;
        const int state = gm_session_state(M.sys, live[i].slot0 + c, &rr, &it);
        all = all && state != 0;
        conv = conv && state == 1;
        info.iters = std::max(info.iters, it);
        info.relres = std::max(info.relres, rr);
      }
      if (!all) { ++i; continue; }
      info.converged = conv ? 1 : 0;
      for (int c = 0; c < r->nrhs; ++c) {
        HM_TRY(gm_session_take(M.sys, live[i].slot0 + c, r->x + n * c));
        used[live[i].slot0 + c] = 0;
      }
      done.push_back({r, {conv ? HM_OK : HM_ERR_NO_CONVERGENCE, info}});
      live.erase(live.begin() + (long)i);
    }
    std::vector<SrvRequest*> joiners;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto& d : done) finish(S, d.first, d.second.first, d.second.second, slots);
      if (!done.empty()) S->cv_done.notify_all();
      int free_slots = 0;
      for (int k = 0; k < slots; ++k) free_slots += used[k] ? 0 : 1;
      if (S->mem_waiters == 0) take_requests(S, m, free_slots, &joiners);  // else: end soon
      owned.insert(owned.end(), joiners.begin(), joiners.end());
      S->joined += (int64_t)joiners.size();
      int add = 0;
      for (SrvRequest* r : joiners) add += r->nrhs;
      S->batched_rhs += add;
    }
    for (SrvRequest* r : joiners) {
      const int ps = put(r);
      if (ps == HM_ERR_CAPACITY) {  // no contiguous run of free slots: back to the queue's head
        std::lock_guard<std::mutex> lk(S->mu);
        S->batched_rhs -= r->nrhs;
        S->joined -= 1;
        owned.erase(std::find(owned.begin(), owned.end(), r));
        S->q.push_front(r);
        S->cv_work.notify_all();
      } else if (ps != HM_OK) {
        return ps;
      }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    M.last_use = ++S->clock;
  }
  return HM_OK;
}

static void worker_loop(hm_server_s* S, int w) {
  SrvWorker& W = S->workers[w];
  cudaSetDevice(W.ctx->opts.device);
  for (;;) {
    std::vector<SrvRequest*> batch;
    int m = -1, from = -1;
    SrvMatrix* Mp = nullptr;
    SrvMatrix* rel = nullptr;  // previous matrix whose solve state is released here
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // the oldest request whose matrix no worker holds, unless it is resident on another
      // worker that is idle (that worker takes it and keeps its solve state)
      int first_nrhs = 0;
      auto pick = [&]() -> bool {
        for (SrvRequest* r : S->q) {
          SrvMatrix* M = S->matrices[r->matrix].get();
          if (M->serving >= 0) continue;
          if (M->worker >= 0 && M->worker != w && !S->workers[M->worker].busy) continue;
          m = r->matrix;
          Mp = M;
          first_nrhs = r->nrhs;
          return true;
        }
        return false;
      };
      S->cv_work.wait(lk, [&] { return S->stop || pick(); });
      if (!Mp) return;  // stopping, and nothing this worker can take
      Mp->serving = w;
      W.busy = true;
      S->cv_work.notify_all();  // requests left to this worker while it was idle are free now
      from = Mp->sys ? Mp->worker : -1;
      if (from >= 0 && from != w && S->workers[from].last == Mp) S->workers[from].last = nullptr;
      if (W.last && W.last != Mp) {
        // one system's transient solve state (apply plans, GMRES workspace) per worker;
        // a previous matrix held by another worker is that worker's to release
        if (W.last->sys && W.last->serving < 0 && W.last->worker == w) {
          rel = W.last;
          rel->serving = w;
        }
        W.last = nullptr;
      }
      // the session's starting columns: within a quarter of a worker's share of the
      // budget for the GMRES workspace (the oldest request always fits)
      int cap = S->max_batch_rhs;
      const hm_opts& o = W.ctx->opts;
      if (S->budget.limit) {
        const double per_col = (2.0 * o.restart + 6.0) * 8.0 * (double)Mp->n;
        cap = std::max(first_nrhs,
                       std::min(cap, (int)(0.25 * (double)S->budget.limit / S->workers.size() / per_col)));
      }
      take_requests(S, m, cap, &batch);
    }
    if (rel) {
      release_solve_state(rel->sys);
      std::lock_guard<std::mutex> lk(S->mu);
      rel->serving = -1;
      S->cv_work.notify_all();
    }
    SrvMatrix& M = *Mp;
    int st = HM_OK;
    bool entered = false;
    if (from >= 0 && from != w) {  // resident on another worker: move it here
      st = move_sys(M.sys, W.ctx, M.ready);
      std::lock_guard<std::mutex> lk(S->mu);
      if (st == HM_OK) {
        M.worker = w;
        S->moved++;
      }
    }
    if (st == HM_OK) {
      {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!M.sys) M.worker = w;
      }
      st = make_resident(S, w, m, M);
    }
    if (st == HM_OK) {
      {
        std::lock_guard<std::mutex> lk(S->mu);
        M.last_use = ++S->clock;
      }
      st = run_session(S, w, m, M, batch, &entered);
    }
    if (M.sys) {  // marks the end of the system's work on this stream for a later mover
      if (!M.ready) cudaEventCreateWithFlags(&M.ready, cudaEventDisableTiming);
      if (M.ready) cudaEventRecord(M.ready, W.ctx->stream);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (!M.sys) M.worker = -1;
    if (M.sys && M.worker == w) W.last = Mp;
    M.serving = -1;
    W.busy = false;
    if (entered) {  // the matrix is evictable now: workers waiting for memory retry
      S->in_session--;
      S->sessions_ended++;
    }
    for (SrvRequest* r : batch)  // requests still open after a failure fail with it
      if (!r->done) finish(S, r, st == HM_OK ? HM_ERR_CUDA : st, hm_solve_info{}, 0);
    S->cv_done.notify_all();
    S->cv_work.notify_all();  // the matrix is free for other workers again
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
  hm_server_s* S = new hm_server_s();
  S->budget.limit = o.hbm_budget;  // one budget for all workers
  o.hbm_budget = 0;
  S->max_batch_rhs = max_batch_rhs;
  S->workers.resize(nworkers);
  for (int w = 0; w < nworkers; ++w) {
    const int st = hm_create(&S->workers[w].ctx, &o);
    if (st != HM_OK) {
      for (int v = w - 1; v >= 0; --v) hm_ctx_destroy(S->workers[v].ctx);
      delete S;
      return st;
    }
    hm_ctx_s* ctx = S->workers[w].ctx;
    ctx->shared = &S->budget;
    if (w > 0) {  // the memory pool of worker 0 serves every worker
      cudaMemPoolDestroy(ctx->pool);
      ctx->pool = S->workers[0].ctx->pool;
      ctx->own_pool = false;
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
  M.nnz = nnz;
  M.coords.assign(grid_coords, grid_coords + (size_t)n * dim);
  std::lock_guard<std::mutex> lk(S->mu);
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
  S->q.push_back(r.get());
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
  st->device_bytes = (double)held_bytes(S);
  st->joined = S->joined;
  st->oom_retries = S->oom_retries;
  st->moved = S->moved;
  st->memory_waits = S->memory_waits;
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
  for (auto& M : S->matrices) {
    if (M->sys && M->worker >= 0) {
      cudaSetDevice(S->workers[M->worker].ctx->opts.device);
      hm_destroy(M->sys);
    }
    if (M->ready) cudaEventDestroy(M->ready);
  }
  for (int w = (int)S->workers.size() - 1; w >= 0; --w) hm_ctx_destroy(S->workers[w].ctx);  // pool owner last
  delete S;
  return HM_OK;
}

}  // extern "C"
