// nk_sr_step_noalloc: the SR step of nk_sr_step for callers that cannot
// allocate device memory.
//
// Some callers have no way to obtain scratch memory: code that runs inside a
// host framework which owns the device allocator and forbids raw cudaMalloc,
// plugins that are handed only a stream and a few tensors, and latency-bound
// loops that must never block on an allocation.  For them this entry point
// takes its scratch from one fixed device array that lives in the library
// image (NK_SR_NOALLOC_MAX_BYTES bytes, held by every GPU that loads the
// library until the process exits).  The caller still passes every input and
// output; nothing is allocated or freed here.
//
// In host code the name of a __device__ array is only a host-side stand-in, not
// a device address, so the device address is looked up with
// cudaGetSymbolAddress, once per device, by the first call made on that device
// (with that device current), and cached.  Make that first call before any
// stream capture.  Every call shares the one array: calls that overlap on the
// GPU (different streams, or different host threads) race on it and must be
// serialised by the caller.  The array keeps the contents of the last call;
// the SR step initialises every scratch word it reads (the CG vectors, the
// reduction partials and the scalar block, whose convergence flag is cleared
// with cudaMemsetAsync), so no stale value is ever used.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace nk {

static __device__ __align__(256) unsigned char g_sr_scratch[NK_SR_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 128;
static void* g_sr_scratch_addr[kMaxDevices];
static std::mutex g_sr_scratch_mu;

// Device address of g_sr_scratch on the current device (looked up once).
static nk_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(NK_ERR_CUDA, "nk_sr_step_noalloc: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(NK_ERR_UNSUPPORTED, "nk_sr_step_noalloc: device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_sr_scratch_mu);
  if (!g_sr_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sr_scratch);
    if (e != cudaSuccess || !p)
      return fail(NK_ERR_CUDA, "nk_sr_step_noalloc: cudaGetSymbolAddress failed: %s",
                  cudaGetErrorString(e));
    g_sr_scratch_addr[dev] = p;
  }
  *out = g_sr_scratch_addr[dev];
  return NK_OK;
}

}  // namespace nk

using namespace nk;

extern "C" nk_status nk_sr_step_noalloc(nk_rbm* rbm, const int8_t* sigma, const void* t,
                                        const double* eloc, const double* weights, int64_t ns,
                                        int32_t n_chains, double diag_shift, double lr,
                                        int32_t n_cg, double cg_rtol, int32_t prec,
                                        double* info_out, void* stream) {
  if (!rbm) return fail(NK_ERR_INVALID_ARG, "nk_sr_step_noalloc: rbm is NULL");
  if (ns < 1) return fail(NK_ERR_INVALID_ARG, "nk_sr_step_noalloc: ns < 1");
  if (rbm->n < 1 || rbm->m < 1)
    return fail(NK_ERR_SHAPE, "nk_sr_step_noalloc: n = %d, m = %d", rbm->n, rbm->m);
  const size_t need = sr_scratch_bytes(rbm->n, rbm->m, rbm->is_complex ? 1 : 0, ns);
  if (need > (size_t)NK_SR_NOALLOC_MAX_BYTES)
    return fail(NK_ERR_SHAPE,
                "nk_sr_step_noalloc: this problem (n = %d, m = %d, ns = %lld) needs %zu B of "
                "scratch, more than the built-in %zu B; use nk_sr_step with caller scratch",
                rbm->n, rbm->m, (long long)ns, need, (size_t)NK_SR_NOALLOC_MAX_BYTES);
  void* scratch = nullptr;
  if (nk_status e = noalloc_scratch(&scratch)) return e;
  return nk_sr_step(rbm, sigma, t, eloc, weights, ns, n_chains, diag_shift, lr, n_cg, cg_rtol,
                    prec, scratch, (size_t)NK_SR_NOALLOC_MAX_BYTES, info_out, stream);
}
