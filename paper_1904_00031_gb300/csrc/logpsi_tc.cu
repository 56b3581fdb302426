// K1 (tensor-core path): theta = [W | b] [sigma; 1] on the tensor cores (W | b
// split into BF16 hi + lo planes by nk_rbm_prepare, sigma exact in BF16, FP32
// accumulation in TMEM), ln cosh fused into the epilogue and summed per
// configuration in FP64, a . sigma added in FP64 (Sec. 2.2.2, RbmSpin).  With
// logpsi NULL the epilogue only stores theta and / or tanh(theta).
#include <vector>

#include "tc.cuh"

namespace nk {

nk_status launch_logpsi_bf16(const nk_rbm* r, const int8_t* sigma, int64_t ns, double* logpsi,
                             void* theta_out, cudaStream_t st, void* t_out) {
  WsLayout L(r->n, r->m, r->is_complex);
  FwdTcArgs A{};
  A.sigma = sigma;
  A.ns = ns;
  A.n = r->n;
  A.m = r->m;
  A.cplx = r->is_complex;
  A.mode = 1;
  A.mt = L.mt;
  A.na64 = L.na64;
  A.rows = r->m;
  A.a = r->a;
  A.logpsi = logpsi;
  A.theta_out = theta_out;
  A.t_out = t_out;
  A.nseg_req = r->theta_segs;
  return launch_fwd_tc(A, (const char*)r->ws + L.wbf, st);
}

nk_status launch_logpsi_bf16_fused(const nk_logpsi_item* items, const int* idx, int n,
                                   cudaStream_t st) {
  std::vector<FwdTcArgs> args((size_t)n);
  std::vector<const void*> planes((size_t)n);
  for (int u = 0; u < n; ++u) {
    const nk_logpsi_item& it = items[idx[u]];
    const nk_rbm* r = it.rbm;
    WsLayout L(r->n, r->m, r->is_complex);
    FwdTcArgs& A = args[u];
    A = FwdTcArgs{};
    A.sigma = it.sigma;
    A.ns = it.ns;
    A.n = r->n;
    A.m = r->m;
    A.cplx = r->is_complex;
    A.mode = 1;
    A.mt = L.mt;
    A.na64 = L.na64;
    A.rows = r->m;
    A.a = r->a;
    A.logpsi = it.logpsi_out;
    A.theta_out = it.theta_out;
    A.nseg_req = r->theta_segs;
    planes[u] = (const char*)r->ws + L.wbf;
  }
  return launch_fwd_tc_fused(args.data(), planes.data(), n, st);
}

}  // namespace nk
