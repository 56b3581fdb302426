// K9: derived planes of an RBM from its FP64 master parameters.
//
// The ratio of amplitudes for flipping spin i (Sec. 2.2.5; RBM of Sec. 2.2.2) is
//   psi(sigma')/psi(sigma) = exp(-2 a_i s) prod_j cosh(theta_j - 2 s W_ji)/cosh(theta_j)
// with s = sigma_i, and cosh(theta - c)/cosh(theta) = cosh c - tanh(theta) sinh c.
// The tables cosh(2 W_ji), sinh(2 W_ji) let the sampling and local-energy
// kernels evaluate every factor with complex multiply-adds only.  They are
// computed in FP64 and rounded once.
#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace nk {

template <bool CPLX>
__device__ __forceinline__ void prepare_body(int bx, int gx, int n, int m, int mp,
                                             const double* __restrict__ a,
                                             const double* __restrict__ b,
                                             const double* __restrict__ w, char* __restrict__ ws,
                                             size_t o_a32, size_t o_b32, size_t o_wt,
                                             size_t o_tab, size_t o_xw) {
  const int64_t total = (int64_t)n * mp;
  for (int64_t e = bx * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gx * blockDim.x) {
    int i = (int)(e / mp), j = (int)(e % mp);
    double wr = 0.0, wi = 0.0;
    if (j < m) {
      if (CPLX) {
        wr = w[2 * ((int64_t)j * n + i)];
        wi = w[2 * ((int64_t)j * n + i) + 1];
      } else {
        wr = w[(int64_t)j * n + i];
      }
    }
    double c2 = cosh(2.0 * wr), s2 = sinh(2.0 * wr);
    if (CPLX) {
      double cy = cos(2.0 * wi), sy = sin(2.0 * wi);
      reinterpret_cast<float2*>(ws + o_wt)[e] = make_float2((float)wr, (float)wi);
      // cosh(2w) = cosh 2x cos 2y + i sinh 2x sin 2y; sinh(2w) = sinh 2x cos 2y + i cosh 2x sin 2y
      reinterpret_cast<float4*>(ws + o_tab)[e] =
          make_float4((float)(c2 * cy), (float)(s2 * sy), (float)(s2 * cy), (float)(c2 * sy));
    } else {
      reinterpret_cast<float*>(ws + o_wt)[e] = (float)wr;
      reinterpret_cast<float2*>(ws + o_tab)[e] = make_float2((float)c2, (float)s2);
    }
  }
  // augmented row-major W | b, rows j < mp, columns i <= n (column n = b)
  const int64_t total2 = (int64_t)mp * (n + 1);
  for (int64_t e = bx * (int64_t)blockDim.x + threadIdx.x; e < total2;
       e += (int64_t)gx * blockDim.x) {
    int j = (int)(e / (n + 1)), i = (int)(e % (n + 1));
    double vr = 0.0, vi = 0.0;
    if (j < m) {
      if (i < n) {
        if (CPLX) {
          vr = w[2 * ((int64_t)j * n + i)];
          vi = w[2 * ((int64_t)j * n + i) + 1];
        } else {
          vr = w[(int64_t)j * n + i];
        }
      } else {
        vr = CPLX ? b[2 * j] : b[j];
        vi = CPLX ? b[2 * j + 1] : 0.0;
      }
    }
    if (CPLX)
      reinterpret_cast<float2*>(ws + o_xw)[e] = make_float2((float)vr, (float)vi);
    else
      reinterpret_cast<float*>(ws + o_xw)[e] = (float)vr;
  }
  const int64_t t3 = bx * (int64_t)blockDim.x + threadIdx.x;
  if (t3 < n) {
    if (CPLX)
      reinterpret_cast<float2*>(ws + o_a32)[t3] = make_float2((float)a[2 * t3], (float)a[2 * t3 + 1]);
    else
      reinterpret_cast<float*>(ws + o_a32)[t3] = (float)a[t3];
  }
  if (t3 < mp) {
    double br = 0.0, bi = 0.0;
    if (t3 < m) {
      br = CPLX ? b[2 * t3] : b[t3];
      bi = CPLX ? b[2 * t3 + 1] : 0.0;
    }
    if (CPLX)
      reinterpret_cast<float2*>(ws + o_b32)[t3] = make_float2((float)br, (float)bi);
    else
      reinterpret_cast<float*>(ws + o_b32)[t3] = (float)br;
  }
}

template <bool CPLX>
__global__ void prepare_kernel(int n, int m, int mp, const double* __restrict__ a,
                               const double* __restrict__ b, const double* __restrict__ w,
                               char* __restrict__ ws, WsLayout L) {
  prepare_body<CPLX>(blockIdx.x, gridDim.x, n, m, mp, a, b, w, ws, L.a32, L.b32, L.wt, L.tab,
                     L.xw);
}

// the same for every problem of an SR batch (blockIdx.y)
__global__ void prepare_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  if (d.cplx)
    prepare_body<true>(blockIdx.x, gridDim.x, d.n, d.m, d.mp, d.a, d.b, d.w, d.ws, d.ws_a32,
                       d.ws_b32, d.ws_wt, d.ws_tab, d.ws_xw);
  else
    prepare_body<false>(blockIdx.x, gridDim.x, d.n, d.m, d.mp, d.a, d.b, d.w, d.ws, d.ws_a32,
                        d.ws_b32, d.ws_wt, d.ws_tab, d.ws_xw);
}

nk_status launch_prepare_batch(const SrDesc* D, int G, int64_t max_work, int64_t max_minb,
                               cudaStream_t st) {
  int64_t blocks = (max_work + 255) / 256;
  blocks = std::max<int64_t>(std::min<int64_t>(blocks, 152 * 8), max_minb);
  prepare_batch<<<dim3((unsigned)blocks, (unsigned)G), 256, 0, st>>>(D);
  return check_launch("prepare_batch");
}

nk_status launch_prepare(const nk_rbm* r, cudaStream_t st) {
  WsLayout L(r->n, r->m, r->is_complex);
  int64_t work = (int64_t)L.mp * (r->n + 1);
  int threads = 256;
  int64_t blocks = (work + threads - 1) / threads;
  int64_t minb = (std::max(L.mp, r->n) + threads - 1) / threads;
  blocks = std::max<int64_t>(std::min<int64_t>(blocks, 152 * 8), minb);
  if (r->is_complex)
    prepare_kernel<true><<<(unsigned)blocks, threads, 0, st>>>(r->n, r->m, L.mp, r->a, r->b, r->w,
                                                              (char*)r->ws, L);
  else
    prepare_kernel<false><<<(unsigned)blocks, threads, 0, st>>>(r->n, r->m, L.mp, r->a, r->b, r->w,
                                                               (char*)r->ws, L);
  if (nk_status e = check_launch("nk_rbm_prepare")) return e;
  return launch_bplanes_from_rbm(r, st);
}

}  // namespace nk
