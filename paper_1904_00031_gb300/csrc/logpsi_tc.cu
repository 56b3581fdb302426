// K1 (tensor-core path): placeholder until the tcgen05 kernel lands.
#include "common.cuh"
#include "internal.h"

namespace nk {

nk_status launch_logpsi_bf16(const nk_rbm* r, const int8_t* sigma, int64_t ns, double* logpsi,
                             void* theta_out, cudaStream_t st) {
  (void)r; (void)sigma; (void)ns; (void)logpsi; (void)theta_out; (void)st;
  return fail(NK_ERR_UNSUPPORTED, "nk_rbm_logpsi: NK_PREC_BF16X2 not built yet");
}

}  // namespace nk
