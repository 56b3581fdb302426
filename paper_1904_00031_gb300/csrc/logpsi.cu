// K1 (FP32 path): ln psi(sigma) = a . sigma + sum_j ln cosh(theta_j),
// theta = W sigma + b (Sec. 2.2.2: RbmSpin; an RBM is a one-layer FFNN with
// ln cosh activation).  theta is computed as the augmented contraction
// [W | b] [sigma; 1] on the CUDA cores (16-site chunks summed in FP32 and
// carried with TwoSum: theta to about one FP32 rounding), ln cosh is fused into
// the epilogue and summed per sample in FP64; a . sigma is added in FP64 from
// the master a.
// Without a ln psi output the epilogue only stores theta and / or tanh(theta)
// (the local energies need theta; the backward recomputes tanh(theta) per
// chunk of samples).
#include "common.cuh"
#include "internal.h"
#include "sgemm.cuh"

namespace nk {

template <bool CPLX>
struct LogpsiEpi {
  using F = typename SgTypes<CPLX>::F;
  int m, n;
  int64_t ns;
  F* theta_out;            // [ns][m] or null
  F* t_out;                // [ns][m] tanh(theta) or null
  const double* a;         // master a (F64)
  const int8_t* sigma;
  double* logpsi;          // c128 [ns], or null: theta / tanh(theta) only, no ln cosh

  __device__ __forceinline__ void tile(float (&ar)[4][4], float (&ai)[4][4], int64_t sb, int jb,
                                       double2 (&part)[4]) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      int64_t s = sb + p;
      if (s >= ns) continue;
      float lr = 0.f, li = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int j = jb + 16 * q;
        if (j >= m) continue;
        if constexpr (CPLX) {
          if (logpsi) {
            cf l = lncosh_c(cf{ar[p][q], ai[p][q]});
            lr += l.x;
            li += l.y;
          }
          if (theta_out) theta_out[s * m + j] = make_float2(ar[p][q], ai[p][q]);
          if (t_out) {
            cf t = tanh_c(cf{ar[p][q], ai[p][q]});
            t_out[s * m + j] = make_float2(t.x, t.y);
          }
        } else {
          if (logpsi) lr += lncosh_f(ar[p][q]);
          if (theta_out) theta_out[s * m + j] = ar[p][q];
          if (t_out) t_out[s * m + j] = tanh_f(ar[p][q]);
        }
      }
      part[p].x += (double)lr;
      part[p].y += (double)li;
    }
  }

  __device__ __forceinline__ void finish(int64_t s, double2 v) {
    if (!logpsi) return;
    double vr = 0.0, vi = 0.0;
    const int8_t* sg = sigma + s * n;
    for (int i = 0; i < n; ++i) {
      double si = (double)sg[i];
      if (CPLX) {
        vr += a[2 * i] * si;
        vi += a[2 * i + 1] * si;
      } else {
        vr += a[i] * si;
      }
    }
    logpsi[2 * s] = v.x + vr;
    logpsi[2 * s + 1] = v.y + vi;
  }
};

template <bool CPLX>
__global__ void __launch_bounds__(kSgThreads) logpsi_fp32_kernel(const int8_t* __restrict__ sigma,
                                                                 int64_t ns, int n, int m,
                                                                 const void* __restrict__ xw,
                                                                 int rows, const double* a,
                                                                 double* logpsi, void* theta_out,
                                                                 void* t_out) {
  LogpsiEpi<CPLX> epi;
  epi.m = m;
  epi.n = n;
  epi.ns = ns;
  epi.theta_out = reinterpret_cast<typename SgTypes<CPLX>::F*>(theta_out);
  epi.t_out = reinterpret_cast<typename SgTypes<CPLX>::F*>(t_out);
  epi.a = a;
  epi.sigma = sigma;
  epi.logpsi = logpsi;
  sgemm_rowreduce<CPLX, LogpsiEpi<CPLX>, true>(sigma, ns, n, xw, rows, n + 1, epi);
}

// Up to kLogpsiBatch problems of one field in one launch: CTA b runs sample
// tile b - start[k] of problem k, as that problem's own launch would.
constexpr int kLogpsiBatch = 64;
struct LogpsiFp32Job {
  const int8_t* sigma;
  int64_t ns;
  int n, m;
  const void* xw;
  const double* a;
  double* logpsi;
  void* theta_out;
};
struct LogpsiFp32Batch {
  int n;
  int start[kLogpsiBatch + 1];
  LogpsiFp32Job j[kLogpsiBatch];
};

template <bool CPLX>
__global__ void __launch_bounds__(kSgThreads) logpsi_fp32_batch(const __grid_constant__ LogpsiFp32Batch B) {
  int k = 0;
  while (k + 1 < B.n && (int)blockIdx.x >= B.start[k + 1]) ++k;
  const LogpsiFp32Job& J = B.j[k];
  LogpsiEpi<CPLX> epi;
  epi.m = J.m;
  epi.n = J.n;
  epi.ns = J.ns;
  epi.theta_out = reinterpret_cast<typename SgTypes<CPLX>::F*>(J.theta_out);
  epi.t_out = nullptr;
  epi.a = J.a;
  epi.sigma = J.sigma;
  epi.logpsi = J.logpsi;
  sgemm_rowreduce<CPLX, LogpsiEpi<CPLX>, true>(J.sigma, J.ns, J.n, J.xw, J.m, J.n + 1, epi,
                                               (int)blockIdx.x - B.start[k]);
}

nk_status launch_logpsi_fp32_fused(const nk_logpsi_item* items, const int* idx, int n,
                                   cudaStream_t st) {
  for (int field = 0; field < 2; ++field) {
    for (int u0 = 0; u0 < n;) {
      LogpsiFp32Batch B;
      B.n = 0;
      B.start[0] = 0;
      int u = u0;
      for (; u < n && B.n < kLogpsiBatch; ++u) {
        const nk_logpsi_item& it = items[idx[u]];
        const nk_rbm* r = it.rbm;
        if ((r->is_complex ? 1 : 0) != field) continue;
        WsLayout L(r->n, r->m, r->is_complex);
        B.j[B.n] = LogpsiFp32Job{it.sigma, it.ns, r->n, r->m, (const char*)r->ws + L.xw, r->a,
                                 it.logpsi_out, it.theta_out};
        B.start[B.n + 1] = B.start[B.n] + (int)((it.ns + kSgBS - 1) / kSgBS);
        ++B.n;
      }
      u0 = u;
      if (B.n == 0) continue;
      if (field) logpsi_fp32_batch<true><<<B.start[B.n], kSgThreads, 0, st>>>(B);
      else logpsi_fp32_batch<false><<<B.start[B.n], kSgThreads, 0, st>>>(B);
      if (nk_status e = check_launch("nk_batch_logpsi")) return e;
    }
  }
  return NK_OK;
}

nk_status launch_logpsi_fp32(const nk_rbm* r, const int8_t* sigma, int64_t ns, double* logpsi,
                             void* theta_out, cudaStream_t st, void* t_out) {
  WsLayout L(r->n, r->m, r->is_complex);
  const char* ws = (const char*)r->ws;
  int64_t blocks = (ns + kSgBS - 1) / kSgBS;
  if (r->is_complex)
    logpsi_fp32_kernel<true><<<(unsigned)blocks, kSgThreads, 0, st>>>(
        sigma, ns, r->n, r->m, ws + L.xw, r->m, r->a, logpsi, theta_out, t_out);
  else
    logpsi_fp32_kernel<false><<<(unsigned)blocks, kSgThreads, 0, st>>>(
        sigma, ns, r->n, r->m, ws + L.xw, r->m, r->a, logpsi, theta_out, t_out);
  return check_launch("nk_rbm_logpsi");
}

}  // namespace nk
