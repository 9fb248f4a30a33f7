// hm_noalloc.cu -- a preconditioner apply that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: applications whose device memory
// is owned entirely by another allocator (a framework's caching pool, or a fixed memory
// budget that must not be exceeded behind its back), allocator or memory-pressure
// callbacks that must not re-enter the CUDA allocator, and latency-critical loops that
// cannot wait on the driver's allocator.  hm_precond_apply allocates three temporary
// n x nrhs blocks per call, and replays its launches from a CUDA graph it captures and
// instantiates (the driver allocates for both); this variant keeps the temporaries in
// one file-scope device array of fixed size instead and launches the same kernels one by
// one, never through a graph.  It synchronizes the context's stream before returning.
#include <mutex>

#include "hm_internal.h"

namespace hm {

// n * nrhs limit of the allocation-free apply.
constexpr int64_t kNoAllocMaxElems = 262144;

// Per-call temporaries: the permuted FP64 copy of r, then the factor-precision input
// and output blocks, kNoAllocMaxElems doubles each (6 MiB in all).  Every GPU that loads
// the library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[3 * kNoAllocMaxElems];

// Device address of g_noalloc_scratch.  In host code the symbol is only a host-side
// stand-in, not a device address, so the address is looked up with cudaGetSymbolAddress,
// with the context's device current, at the first allocation-free call on each context
// (the lookup allocates nothing).  Keeping it per context rather than per process means
// a context created after a device reset never reuses an address from before the reset.
static std::mutex g_noalloc_mu;

static int noalloc_scratch(hm_ctx_s* ctx, double** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!ctx->noalloc_scratch) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      set_last_error(std::string("hm_precond_apply_noalloc: cudaGetSymbolAddress: ") +
                     cudaGetErrorString(e));
      return HM_ERR_CUDA;
    }
    ctx->noalloc_scratch = p;
  }
  *out = (double*)ctx->noalloc_scratch;
  return HM_OK;
}

template <typename T>
static int apply_noalloc_t(hm_sys_s* sys, int nrhs, const double* r, double* z, double* scratch) {
  cudaStream_t s = sys->ctx->stream;
  const int n = sys->n;
  const int64_t nn = (int64_t)n * nrhs;
  double* rp = scratch;
  T* rT = (T*)(scratch + kNoAllocMaxElems);
  T* zT = (T*)(scratch + 2 * kNoAllocMaxElems);
  launch_permute_in(r, rp, sys->d_perm, n, nrhs, s);
  launch_cast_to<T>(rp, rT, nn, s);
  HM_TRY(apply_impl_eager(sys, nrhs, rT, zT));  // kernel launches only: no graph, no allocation
  launch_cast_from<T>(zT, rp, nn, s);
  launch_permute_out(rp, z, sys->d_perm, n, nrhs, s);
  HM_CUDA(cudaStreamSynchronize(s));
  HM_CUDA(cudaGetLastError());
  return check_device_error(sys, "hm_precond_apply_noalloc");
}

}  // namespace hm

using namespace hm;

extern "C" int hm_precond_apply_noalloc(hm_sys_t sys, int32_t nrhs, const double* r, double* z) {
  if (!sys || !r || !z || nrhs < 1 || nrhs > 64) {
    set_last_error("hm_precond_apply_noalloc: null argument or nrhs outside 1..64");
    return HM_ERR_INVALID_ARG;
  }
  if ((int64_t)sys->n * nrhs > kNoAllocMaxElems) {
    set_last_error("hm_precond_apply_noalloc: n * nrhs = " + std::to_string((int64_t)sys->n * nrhs) +
                   " exceeds the fixed maximum of " + std::to_string(kNoAllocMaxElems));
    return HM_ERR_CAPACITY;
  }
  if (!sys->factored) {
    set_last_error("hm_precond_apply_noalloc before hm_factor");
    return HM_ERR_STATE;
  }
  if (sys->solve_plans.find(nrhs) == sys->solve_plans.end()) {
    set_last_error("hm_precond_apply_noalloc: no workspace for this nrhs yet; call hm_precond_apply "
                   "or hm_solve once with the same nrhs first");
    return HM_ERR_STATE;
  }
  const int dev = sys->ctx->opts.device;
  if (cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("hm_precond_apply_noalloc: cudaSetDevice failed");
    return HM_ERR_CUDA;
  }
  if (!is_device_ptr(r) || !is_device_ptr(z)) {
    set_last_error("hm_precond_apply_noalloc: r and z must be device pointers");
    return HM_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  HM_TRY(noalloc_scratch(sys->ctx, &scratch));
  return sys->precision == HM_PREC_FP64 ? apply_noalloc_t<double>(sys, nrhs, r, z, scratch)
                                        : apply_noalloc_t<float>(sys, nrhs, r, z, scratch);
}
