// Supervised learning of a target wavefunction (Sec. 2.2.3): the negative log
// overlap loss of Eq. 1 estimated from samples of the target, its gradient as
// one adjoint contraction of the analytic RBM log-derivatives (Sec. 2.2.5), and
// an AdaMax update (the optimiser list of Sec. 2.2.3; Kingma and Ba,
// Algorithm 2).
//
// With samples sigma_s of |tar|^2 and weights w_s (1/ns, or the caller's, normalised),
// ratios R_s = psi(sigma_s) / tar(sigma_s) give
//   L = -log(|<R>|^2 / <|R|^2>),
//   dL/dconj(alpha) x 2 = sum_s conj(O_s) g_s,  g_s = 2 w_s (|R_s|^2 / <|R|^2> - conj(R_s) / conj(<R>)),
// so the gradient is nk_rbm_logpsi_backward with upstream vector g.  Both L and
// g are invariant under R -> c R, so R is formed as exp(ln psi - ln tar - c)
// with c = max_s Re(ln psi - ln tar), which keeps every exponent <= 0.
//
// Passes (fixed-order reductions, no atomics, so a step is reproducible):
//   ln psi (the theta contraction with the ln cosh epilogue, at `prec`),
//   sup_max: per-block max of Re(ln psi - ln tar),
//   sup_sums: per-block sums of w R, w |R|^2 and w,
//   sup_finish (one block): <R>, <|R|^2>, L, the overlap |<R>|^2 / <|R|^2>,
//   sup_g: the upstream vector g,
//   the chunked backward (theta recomputed per chunk) -> gradient,
//   adamax: the moments and the FP64 master parameters, then the derived planes.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace nk {

namespace {

constexpr int kSupThreads = 256;
constexpr int kSupBlocks = 1024;  // partial-sum slots per quantity

// scratch layout (bytes, 256-B aligned pieces)
struct SupLayout {
  size_t lp, g, red, scal, grad, back, total;
  SupLayout(int n, int m, int cplx, int64_t ns) {
    const int64_t P = (int64_t)n + m + (int64_t)m * n;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t o = 0;
    lp = o;
    o += up((size_t)std::max<int64_t>(ns, 1) * 16);
    g = o;
    o += up((size_t)std::max<int64_t>(ns, 1) * 16);
    red = o;
    o += up((size_t)5 * kSupBlocks * 8);
    scal = o;
    o += 256;
    grad = o;
    o += up((size_t)P * (cplx ? 16 : 8));
    back = o;
    o += backward_scratch_bytes(n, m, cplx, ns);
    total = o;
  }
};

int sup_blocks(int64_t ns) {
  return (int)std::min<int64_t>(kSupBlocks, std::max<int64_t>(1, (ns + kSupThreads - 1) / kSupThreads));
}

// fixed-order block reductions (every thread gets the result)
__device__ __forceinline__ double blk_sum(double v, double* sh) {
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += sh[u];
  return t;
}

__device__ __forceinline__ double blk_max(double v, double* sh) {
  for (int off = 16; off >= 1; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = -INFINITY;
  for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t = fmax(t, sh[u]);
  return t;
}

// Re(ln psi_s - ln tar_s)
__device__ __forceinline__ double log_ratio_re(const double* lp, const double* lt, int64_t s) {
  return lp[2 * s] - lt[2 * s];
}

__global__ void __launch_bounds__(kSupThreads) sup_max_kernel(const double* __restrict__ lp,
                                                             const double* __restrict__ lt,
                                                             int64_t ns, double* red) {
  __shared__ double sh[32];
  double v = -INFINITY;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gridDim.x * blockDim.x)
    v = fmax(v, log_ratio_re(lp, lt, s));
  v = blk_max(v, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = v;
}

// R_s = exp(ln psi_s - ln tar_s - c)
__device__ __forceinline__ double2 ratio(const double* lp, const double* lt, int64_t s, double c) {
  const double e = exp(lp[2 * s] - lt[2 * s] - c);
  double sn, cs;
  sincos(lp[2 * s + 1] - lt[2 * s + 1], &sn, &cs);
  return make_double2(e * cs, e * sn);
}

// shift c = max of the block maxima (every block reads all of them)
__device__ __forceinline__ double shift_of(const double* red, int nb) {
  double c = -INFINITY;
  for (int u = 0; u < nb; ++u) c = fmax(c, red[u]);
  return c;
}

__global__ void __launch_bounds__(kSupThreads) sup_sums_kernel(const double* __restrict__ lp,
                                                              const double* __restrict__ lt,
                                                              const double* __restrict__ w,
                                                              int64_t ns, double* red, int nb) {
  __shared__ double sh[32];
  const double c = shift_of(red, nb);
  double rr = 0.0, ri = 0.0, r2 = 0.0, ws = 0.0;
  const double w0 = 1.0 / (double)ns;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double2 R = ratio(lp, lt, s, c);
    const double ww = w ? w[s] : w0;
    rr += ww * R.x;
    ri += ww * R.y;
    r2 += ww * (R.x * R.x + R.y * R.y);
    ws += ww;
  }
  rr = blk_sum(rr, sh);
  ri = blk_sum(ri, sh);
  r2 = blk_sum(r2, sh);
  ws = blk_sum(ws, sh);
  if (threadIdx.x == 0) {
    red[1 * kSupBlocks + blockIdx.x] = rr;
    red[2 * kSupBlocks + blockIdx.x] = ri;
    red[3 * kSupBlocks + blockIdx.x] = r2;
    red[4 * kSupBlocks + blockIdx.x] = ws;
  }
}

// scal: [0] c, [1] Re <R>, [2] Im <R>, [3] <|R|^2>, [4] sum w
// info: [0] L, [1] overlap |<R>|^2 / <|R|^2>, [2] c, [3] flags
__global__ void sup_finish_kernel(const double* red, int nb, double* scal, double* info) {
  if (threadIdx.x != 0) return;
  double s[5];
  s[0] = shift_of(red, nb);
  for (int q = 1; q < 5; ++q) {
    double t = 0.0;
    for (int u = 0; u < nb; ++u) t += red[q * kSupBlocks + u];
    s[q] = t;
  }
  const double ws = s[4];
  const double mr = s[1] / ws, mi = s[2] / ws, m2 = s[3] / ws;
  scal[0] = s[0];
  scal[1] = mr;
  scal[2] = mi;
  scal[3] = m2;
  scal[4] = ws;
  const double ov = (mr * mr + mi * mi) / m2;
  const double loss = -log(ov);
  double flags = 0.0;
  if (!isfinite(loss) || !isfinite(s[0])) flags = (double)(1 << NK_ERR_NONFINITE);
  if (info) {
    info[0] = loss;
    info[1] = ov;
    info[2] = s[0];
    info[3] = flags;
  }
}

// g_s = 2 (w_s / sum w) (|R_s|^2 / <|R|^2> - conj(R_s) / conj(<R>)), c128
__global__ void __launch_bounds__(kSupThreads) sup_g_kernel(const double* __restrict__ lp,
                                                           const double* __restrict__ lt,
                                                           const double* __restrict__ w,
                                                           int64_t ns, const double* scal,
                                                           double* g) {
  const double c = scal[0], mr = scal[1], mi = scal[2], m2 = scal[3], ws = scal[4];
  // 1 / conj(<R>) = <R> / |<R>|^2
  const double den = mr * mr + mi * mi;
  const double ir = mr / den, ii = mi / den;
  const double w0 = 1.0 / (double)ns;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double2 R = ratio(lp, lt, s, c);
    const double ww = 2.0 * (w ? w[s] : w0) / ws;
    // conj(R) / conj(<R>) = conj(R) * <R> / |<R>|^2
    const double qr = R.x * ir + R.y * ii;
    const double qi = R.x * ii - R.y * ir;
    g[2 * s] = ww * ((R.x * R.x + R.y * R.y) / m2 - qr);
    g[2 * s + 1] = ww * (-qi);
  }
}

// AdaMax over the real components e of the parameters (a complex parameter's
// real and imaginary parts are two components), master layout a | b | W:
//   m_e <- b1 m_e + (1 - b1) g_e,  u_e <- max(b2 u_e, |g_e|),
//   x_e <- x_e - (lr / (1 - b1^t)) m_e / u_e   (not moved while u_e = 0).
__global__ void __launch_bounds__(kSupThreads) adamax_kernel(double* a, double* b, double* wm,
                                                            int64_t na, int64_t nb,
                                                            int64_t pr, const double* __restrict__ g,
                                                            double* mom, double lr, double b1,
                                                            double b2, double bias) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < pr;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double ge = g[e];
    const double me = b1 * mom[e] + (1.0 - b1) * ge;
    const double ue = fmax(b2 * mom[pr + e], fabs(ge));
    mom[e] = me;
    mom[pr + e] = ue;
    if (ue > 0.0) {
      const double d = lr / bias * me / ue;
      if (e < na) a[e] -= d;
      else if (e < na + nb) b[e - na] -= d;
      else wm[e - na - nb] -= d;
    }
  }
}

}  // namespace

size_t supervised_scratch_bytes(int n, int m, int cplx, int64_t ns) {
  return SupLayout(n, m, cplx, ns).total;
}

nk_status run_supervised_step(nk_rbm* r, const int8_t* sigma, const double* log_target,
                              const double* weights, int64_t ns, int prec, double lr,
                              double beta1, double beta2, int step, double* moments,
                              double* grad_out, void* scratch, size_t scratch_bytes,
                              double* info, cudaStream_t st) {
  const int cplx = r->is_complex ? 1 : 0;
  SupLayout L(r->n, r->m, cplx, ns);
  if (scratch_bytes < L.total)
    return fail(NK_ERR_SHAPE, "nk_supervised_step: scratch of %zu B, need %zu B", scratch_bytes,
                L.total);
  char* sc = (char*)scratch;
  double* lp = (double*)(sc + L.lp);
  double* g = (double*)(sc + L.g);
  double* red = (double*)(sc + L.red);
  double* scal = (double*)(sc + L.scal);
  double* grad = grad_out ? grad_out : (double*)(sc + L.grad);
  nk_status e = prec == NK_PREC_BF16X2 ? launch_logpsi_bf16(r, sigma, ns, lp, nullptr, st)
                                       : launch_logpsi_fp32(r, sigma, ns, lp, nullptr, st);
  if (e) return e;
  const int nb = sup_blocks(ns);
  sup_max_kernel<<<nb, kSupThreads, 0, st>>>(lp, log_target, ns, red);
  sup_sums_kernel<<<nb, kSupThreads, 0, st>>>(lp, log_target, weights, ns, red, nb);
  sup_finish_kernel<<<1, 32, 0, st>>>(red, nb, scal, info);
  sup_g_kernel<<<nb, kSupThreads, 0, st>>>(lp, log_target, weights, ns, scal, g);
  if ((e = check_launch("nk_supervised_step"))) return e;
  if ((e = run_backward(r, sigma, ns, g, grad, prec, sc + L.back, scratch_bytes - L.back, st)))
    return e;
  if (!moments) return NK_OK;
  const int64_t c = cplx ? 2 : 1;
  const int64_t na = c * r->n, nbias = c * r->m, pr = c * ((int64_t)r->n + r->m + (int64_t)r->m * r->n);
  const double bias = 1.0 - pow(beta1, (double)step);
  const int blocks = (int)std::min<int64_t>(1024, (pr + kSupThreads - 1) / kSupThreads);
  adamax_kernel<<<blocks, kSupThreads, 0, st>>>(r->a, r->b, r->w, na, nbias, pr, grad, moments,
                                                lr, beta1, beta2, bias);
  if ((e = check_launch("nk_supervised_step"))) return e;
  return launch_prepare(r, st);
}

}  // namespace nk
