// K5-K7: energy statistics and stochastic reconfiguration (Sec. 2.2.5; update
// rule Eq. 2), and K8: the backward of ln psi.
//
// The SR system (S + eps I) delta = F is solved by conjugate gradient with S
// never formed.  All algebra runs on "augmented" operands: T' = [T | 1],
// sigma' = [sigma | 1], and a parameter vector as an (m+1) x (n+1) array X'
// (X'[j][i] = x_W[j][i], X'[j][n] = x_b[j], X'[m][i] = x_a[i], X'[m][n] = 0):
//   (O x)_s         = sum_j T'_sj (X' sigma'_s)_j           (forward contraction)
//   sum_s conj(O_s) v_s = T'^H diag(v) sigma'               (adjoint contraction)
//   S x             = adjoint(w o (O x - <O x>)),  <y> = sum_s w_s y_s.
// The two contractions run at the requested precision: FP32 CUDA-core kernels
// here, or the tensor-core kernels of tc.cu (BF16 hi + lo split); CG vectors,
// inner products and every reduction are FP64, and every reduction has a fixed
// order (no atomics), so a step is bitwise reproducible.
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "internal.h"
#include "sgemm.cuh"
#include "bf16split.cuh"
#include "tc.cuh"

namespace nk {

constexpr int kVecBlocks = 1024;  // largest grid of the CG vector kernels

// Blocks of a CG vector kernel over `elems` elements: about 1024 elements per
// 256-thread block, at most kVecBlocks (the partial-sum slots of `red`), so that
// large problems keep enough loads in flight and small ones do not pay for idle
// blocks.  The single-problem and the batched launches use the same count per
// problem, so their reductions run in the same order.
static int sr_vec_blocks(int64_t elems) {
  return (int)std::min<int64_t>(kVecBlocks, std::max<int64_t>(1, (elems + 1023) / 1024));
}
constexpr int kVecThreads = 256;

// Centring partials written by the SR forward (one per CTA: sample tiles x
// hidden-tile halves), or 0 when they would not fit the partials buffer.
static int fwd_centring_parts(int64_t ns, int mt) {
  const int64_t parts = ((ns + 127) / 128) * fwd_tc_nseg(ns, mt, 0, true);
  return parts <= kVecBlocks ? (int)parts : 0;
}

// Whether the SR adjoint centres the forward's output itself (v = w (y - mean)
// formed while loading): every parameter tile's CTAs repeat that FP64 work, so
// only for at most four tiles, where the launch it saves costs more.
static bool adj_centres(int m, int cplx) {
  return (m + 1 + tc_hidden_per_tile(cplx) - 1) / tc_hidden_per_tile(cplx) <= 4;
}
// Elements per thread whose loads are issued together in the vector kernels
// (a thread's elements are still visited, and summed, in grid-stride order).
constexpr int kVecUnroll = 2;
constexpr int kAdjBK = 16;

// scalars in the scratch `scal` block
enum {
  SC_RS0 = 0, SC_RS1 = 1,   // r^H r, double-buffered by iteration parity
  SC_DONE = 2,              // converged flag
  SC_ITERS = 3,             // completed iterations
  SC_FNORM = 4,             // ||F||
  SC_EBAR_RE = 5, SC_EBAR_IM = 6,
  SC_NONFINITE = 7,
  SC_ERR = 8,               // int: a tensor-core kernel gave up a bounded wait
  SC_LEN = 16
};

SrLayout::SrLayout(int n_, int m_, int cplx_, int64_t ns_) : n(n_), m(m_), cplx(cplx_), ns(ns_) {
  ma = m + 1;
  na = n + 1;
  pa = (int64_t)ma * na;
  int tiles = ceil_div(na, 64) * ceil_div(ma, 64);
  int64_t sp = (2 * 152 + tiles - 1) / tiles;
  sp = std::min<int64_t>(sp, std::max<int64_t>(1, ns / 256));
  splits_fp32 = (int)std::max<int64_t>(1, std::min<int64_t>(sp, 64));
  splits_tc = adj_tc_splits(n, m, cplx, ns);
  const int tiles_tc = (m + 1 + tc_hidden_per_tile(cplx) - 1) / tc_hidden_per_tile(cplx);
  splits = std::min(64, std::max(2 * std::max(splits_fp32, splits_tc), (4 * 152) / tiles_tc));
  na64 = (int)round_up(n + 1, 64);
  mt1 = (m + 1 + tc_hidden_per_tile(cplx) - 1) / tc_hidden_per_tile(cplx);
  ns8 = round_up(std::max<int64_t>(ns, 1), 8);
  size_t d = cplx ? 16 : 8;  // F64 element
  size_t f = cplx ? 8 : 4;   // F32 element
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (size_t)round_up((int64_t)bytes, 256);
    return o;
  };
  x = take(pa * d);
  r = take(pa * d);
  p = take(pa * d);
  ap = take(pa * d);
  xf = take(pa * f);
  part = take((size_t)splits * pa * f);
  y = take((size_t)std::max<int64_t>(ns, 1) * 16);
  v = take((size_t)std::max<int64_t>(ns, 1) * 16);
  red = take(4 * kVecBlocks * sizeof(double));
  scal = take(SC_LEN * sizeof(double));
  sigt = take((size_t)na64 * ns8 * 2);
  sigr = take((size_t)std::max<int64_t>(ns, 1) * na64 * 2);
  xbf = take((size_t)2 * mt1 * 128 * na64 * 2);
  total = off;
}

size_t sr_scratch_bytes(int n, int m, int cplx, int64_t ns) {
  return SrLayout(n, m, cplx, ns).total;
}

int sr_choose_splits(const SrLayout& L, int prec, int requested) {
  const int h = prec == NK_PREC_BF16X2 ? L.splits_tc : L.splits_fp32;
  int s = requested > 0 ? requested : h;
  const int64_t max_useful = std::max<int64_t>(1, (L.ns + 63) / 64);
  s = (int)std::min<int64_t>(s, max_useful);
  return std::max(1, std::min(s, L.splits));
}

// ------------------------------------------------------------------ helpers

template <bool CPLX>
struct D;  // F64 element
template <>
struct D<true> {
  using T = double2;
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
};
template <>
struct D<false> {
  using T = double;
  static __device__ __forceinline__ double zero() { return 0.0; }
};

__device__ __forceinline__ double re(double x) { return x; }
__device__ __forceinline__ double re(double2 x) { return x.x; }
__device__ __forceinline__ double im(double) { return 0.0; }
__device__ __forceinline__ double im(double2 x) { return x.y; }

// Where cg_step_p also writes the BF16 hi/lo planes of p (tensor-core path):
// planes [2][mt*128][na64], p in the augmented [m+1][na] layout.  planes = NULL:
// not written (the FP32 path, or the first iteration's planes come from bplanes).
struct PlaneOut {
  uint16_t* planes = nullptr;
  int na = 1, mt = 0, na64 = 64;
};
__device__ __forceinline__ double norm2(double x) { return x * x; }
__device__ __forceinline__ double norm2(double2 x) { return x.x * x.x + x.y * x.y; }
__device__ __forceinline__ double cdot_re(double a, double b) { return a * b; }
__device__ __forceinline__ double cdot_re(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ double axpy(double a, double x, double y) { return fma(a, x, y); }
__device__ __forceinline__ double2 axpy(double a, double2 x, double2 y) {
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}

// Deterministic block reduction of one double (all threads get the result).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int u = 0; u < nw; ++u) t += sh[u];
  return t;
}

// Sum of nb block partials in a fixed order (every block gets the same value).
__device__ __forceinline__ double sum_partials(const double* red, int nb) {
  __shared__ double tot;
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int u = threadIdx.x; u < nb; u += 32) v += red[u];
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) tot = v;
  }
  __syncthreads();
  return tot;
}

// ------------------------------------------------------------------ K7 statistics

// Three passes over the samples in nb blocks (sums of per-block partials in a
// fixed order, so the result does not depend on scheduling):
//   mean:   per-block partials of sum w E_s                 -> red[2K + b], red[3K + b]
//   dev:    E = sum of those; v_s = w_s (E_s - E); per-block partials of
//           sum w |E_s - E|^2 -> red[b] and, over whole chains, of
//           sum_c (mean_c Re E - Re E)^2 -> red[K + b]      (K = kVecBlocks)
//   finish: info {E, var, error from chain means} and the scalars the CG reads.
// v_s is the vector whose adjoint contraction is F.
template <bool CPLX>
__device__ __forceinline__ void stats_mean_body(int bx, int gx, const double* __restrict__ eloc,
                                                const double* __restrict__ weights, int64_t ns,
                                                double* red) {
  const double invn = 1.0 / (double)ns;
  double sr = 0.0, si = 0.0;
  for (int64_t s = bx * (int64_t)blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gx * blockDim.x) {
    const double w = weights ? weights[s] : invn;
    sr += w * eloc[2 * s];
    si += w * eloc[2 * s + 1];
  }
  const double br = block_sum(sr);
  const double bi = block_sum(si);
  if (threadIdx.x == 0) {
    red[2 * kVecBlocks + bx] = br;
    red[3 * kVecBlocks + bx] = bi;
  }
}

template <bool CPLX>
__device__ __forceinline__ void stats_dev_body(int bx, int gx, const double* __restrict__ eloc,
                                               const double* __restrict__ weights, int64_t ns,
                                               int n_chains, double* red, void* vout, int nb) {
  const double er = sum_partials(red + 2 * kVecBlocks, nb);
  const double ei = sum_partials(red + 3 * kVecBlocks, nb);
  const double invn = 1.0 / (double)ns;
  double vv = 0.0;
  for (int64_t s = bx * (int64_t)blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gx * blockDim.x) {
    const double w = weights ? weights[s] : invn;
    const double dr = eloc[2 * s] - er, di = eloc[2 * s + 1] - ei;
    vv += w * (dr * dr + di * di);
    if (CPLX)
      reinterpret_cast<double2*>(vout)[s] = make_double2(w * dr, w * di);
    else
      reinterpret_cast<double*>(vout)[s] = w * dr;
  }
  double ce = 0.0;
  const int64_t spc = n_chains > 0 ? ns / n_chains : 0;
  if (!weights && n_chains > 1 && spc > 0) {
    for (int64_t c = bx * (int64_t)blockDim.x + threadIdx.x; c < n_chains;
         c += (int64_t)gx * blockDim.x) {
      double mc = 0.0;
      for (int64_t u = 0; u < spc; ++u) mc += eloc[2 * (c * spc + u)];
      mc /= (double)spc;
      ce += (mc - er) * (mc - er);
    }
  }
  const double bv = block_sum(vv);
  const double bc = block_sum(ce);
  if (threadIdx.x == 0) {
    red[bx] = bv;
    red[kVecBlocks + bx] = bc;
  }
}

__device__ __forceinline__ void stats_finish_body(const double* __restrict__ weights, int64_t ns,
                                                  int n_chains, const double* red, int nb,
                                                  double* info, double* scal) {
  const double er = sum_partials(red + 2 * kVecBlocks, nb);
  const double ei = sum_partials(red + 3 * kVecBlocks, nb);
  const double var = sum_partials(red, nb);
  const double ce = sum_partials(red + kVecBlocks, nb);
  const int64_t spc = n_chains > 0 ? ns / n_chains : 0;
  if (threadIdx.x == 0) {
    info[NK_INFO_E_RE] = er;
    info[NK_INFO_E_IM] = ei;
    info[NK_INFO_VAR] = var;
    info[NK_INFO_ERR] =
        (!weights && n_chains > 1 && spc > 0) ? sqrt(ce / ((double)n_chains * (n_chains - 1))) : 0.0;
    scal[SC_EBAR_RE] = er;
    scal[SC_EBAR_IM] = ei;
    scal[SC_NONFINITE] = (isfinite(er) && isfinite(ei) && isfinite(var)) ? 0.0 : 1.0;
  }
}

template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) stats_mean_kernel(const double* __restrict__ eloc,
                                                                 const double* __restrict__ weights,
                                                                 int64_t ns, double* red) {
  stats_mean_body<CPLX>(blockIdx.x, gridDim.x, eloc, weights, ns, red);
}

template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) stats_dev_kernel(const double* __restrict__ eloc,
                                                                const double* __restrict__ weights,
                                                                int64_t ns, int n_chains,
                                                                double* red, void* vout, int nb) {
  stats_dev_body<CPLX>(blockIdx.x, gridDim.x, eloc, weights, ns, n_chains, red, vout, nb);
}

__global__ void stats_finish_kernel(const double* __restrict__ weights, int64_t ns, int n_chains,
                                    const double* red, int nb, double* info, double* scal) {
  stats_finish_body(weights, ns, n_chains, red, nb, info, scal);
}

// ------------------------------------------------------------------ adjoint contraction
// part[z][j][i] = sum_{s in split z} conj(T'_sj) v_s sigma'_si   (FP32 CUDA cores)

template <bool CPLX>
__global__ void __launch_bounds__(256) adjoint_fp32_kernel(const int8_t* __restrict__ sigma,
                                                           const void* __restrict__ Tv,
                                                           const void* __restrict__ vv,
                                                           int64_t ns, int n, int m, int64_t chunk,
                                                           void* partv, const double* scal) {
  if (scal && scal[SC_DONE] != 0.0) return;
  using F = typename SgTypes<CPLX>::F;
  const F* T = reinterpret_cast<const F*>(Tv);
  const int ma = m + 1, na = n + 1;
  __shared__ __align__(16) F Zs[kAdjBK][64];
  __shared__ __align__(16) float Ss[kAdjBK][64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
  const int64_t sb = (int64_t)blockIdx.z * chunk;
  const int64_t se = std::min<int64_t>(ns, sb + chunk);
  float ar[4][4], ai[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) ar[p][q] = ai[p][q] = 0.f;
  for (int64_t k0 = sb; k0 < se; k0 += kAdjBK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int e = tid + u * 256;
      int kk = e >> 6, jj = e & 63;
      int64_t s = k0 + kk;
      int j = j0 + jj;
      F z;
      if constexpr (CPLX) {
        z = make_float2(0.f, 0.f);
        if (s < se && j <= m) {
          float2 t = j < m ? T[s * m + j] : make_float2(1.f, 0.f);
          double2 vs = reinterpret_cast<const double2*>(vv)[s];
          float vr = (float)vs.x, vi = (float)vs.y;
          // conj(t) * v
          z = make_float2(t.x * vr + t.y * vi, t.x * vi - t.y * vr);
        }
      } else {
        z = 0.f;
        if (s < se && j <= m) {
          float t = j < m ? T[s * m + j] : 1.f;
          z = t * (float)reinterpret_cast<const double*>(vv)[s];
        }
      }
      Zs[kk][jj] = z;
      int ii = jj, i = i0 + ii;
      float sv = 0.f;
      if (s < se) sv = i < n ? (float)sigma[s * n + i] : (i == n ? 1.f : 0.f);
      Ss[kk][ii] = sv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kAdjBK; ++kk) {
      F z[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) z[p] = Zs[kk][ty * 4 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float sv = Ss[kk][tx + 16 * q];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if constexpr (CPLX) {
            ar[p][q] = fmaf(z[p].x, sv, ar[p][q]);
            ai[p][q] = fmaf(z[p].y, sv, ai[p][q]);
          } else {
            ar[p][q] = fmaf(z[p], sv, ar[p][q]);
          }
        }
      }
    }
    __syncthreads();
  }
  F* part = reinterpret_cast<F*>(partv) + (int64_t)blockIdx.z * ma * na;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int j = j0 + ty * 4 + p;
    if (j >= ma) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int i = i0 + tx + 16 * q;
      if (i >= na) continue;
      if constexpr (CPLX) part[(int64_t)j * na + i] = make_float2(ar[p][q], ai[p][q]);
      else part[(int64_t)j * na + i] = ar[p][q];
    }
  }
}

template <bool CPLX>
static void launch_adjoint_fp32(const int8_t* sigma, const void* T, const void* v, int64_t ns,
                                int n, int m, int splits, void* part, const double* scal,
                                cudaStream_t st) {
  int64_t chunk = (ns + splits - 1) / splits;
  chunk = round_up(chunk, kAdjBK);
  dim3 grid(ceil_div(n + 1, 64), ceil_div(m + 1, 64), splits);
  adjoint_fp32_kernel<CPLX><<<grid, 256, 0, st>>>(sigma, T, v, ns, n, m, chunk, part, scal);
}

// ------------------------------------------------------------------ forward contraction
// y_s = sum_j T'_sj (X' sigma'_s)_j   (FP32 CUDA cores, FP64 row sums)

template <bool CPLX>
struct FwdEpi {
  using F = typename SgTypes<CPLX>::F;
  int m;
  int64_t ns;
  const F* T;
  void* y;
  __device__ __forceinline__ void tile(float (&ar)[4][4], float (&ai)[4][4], int64_t sb, int jb,
                                       double2 (&part)[4]) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      int64_t s = sb + p;
      if (s >= ns) continue;
      float pr = 0.f, pi = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int j = jb + 16 * q;
        if (j > m) continue;
        if constexpr (CPLX) {
          float2 t = j < m ? T[s * m + j] : make_float2(1.f, 0.f);
          pr += t.x * ar[p][q] - t.y * ai[p][q];
          pi += t.x * ai[p][q] + t.y * ar[p][q];
        } else {
          float t = j < m ? T[s * m + j] : 1.f;
          pr += t * ar[p][q];
        }
      }
      part[p].x += (double)pr;
      part[p].y += (double)pi;
    }
  }
  __device__ __forceinline__ void finish(int64_t s, double2 v) {
    if (CPLX) reinterpret_cast<double2*>(y)[s] = v;
    else reinterpret_cast<double*>(y)[s] = v.x;
  }
};

template <bool CPLX>
__global__ void __launch_bounds__(kSgThreads) forward_fp32_kernel(const int8_t* __restrict__ sigma,
                                                                  int64_t ns, int n, int m,
                                                                  const void* __restrict__ xf,
                                                                  const void* __restrict__ T,
                                                                  void* y, const double* scal) {
  if (scal && scal[SC_DONE] != 0.0) return;
  FwdEpi<CPLX> epi;
  epi.m = m;
  epi.ns = ns;
  epi.T = reinterpret_cast<const typename SgTypes<CPLX>::F*>(T);
  epi.y = y;
  sgemm_rowreduce<CPLX>(sigma, ns, n, xf, m + 1, n + 1, epi);
}

// ------------------------------------------------------------------ CG vector kernels

// X' (FP64) -> FP32 copy for the forward contraction
template <bool CPLX>
__global__ void to_f32_kernel(const void* __restrict__ src, void* dst, int64_t pa,
                              const double* scal) {
  if (scal[SC_DONE] != 0.0) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < pa;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (CPLX) {
      double2 v = reinterpret_cast<const double2*>(src)[e];
      reinterpret_cast<float2*>(dst)[e] = make_float2((float)v.x, (float)v.y);
    } else {
      reinterpret_cast<float*>(dst)[e] = (float)reinterpret_cast<const double*>(src)[e];
    }
  }
}

// y~ = w o (y - <y>): pass 1 writes per-block partial sums of w y (fixed grid),
// pass 2 adds them in a fixed order (every block gets the same mean) and
// writes y~.
template <bool CPLX>
__device__ __forceinline__ void center_partial_body(int bx, int gx, 
    const void* __restrict__ yv, const double* __restrict__ weights, int64_t ns, double* red,
    const double* scal) {
  if (scal[SC_DONE] != 0.0) return;
  const double invn = 1.0 / (double)ns;
  double sr = 0.0, si = 0.0;
  const int64_t stride = (int64_t)gx * blockDim.x;
  for (int64_t s0 = bx * (int64_t)blockDim.x + threadIdx.x; s0 < ns;
       s0 += kVecUnroll * stride) {
    double w[kVecUnroll];
    double2 y[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      const int64_t s = s0 + u * stride;
      if (s < ns) {
        w[u] = weights ? weights[s] : invn;
        y[u] = CPLX ? reinterpret_cast<const double2*>(yv)[s]
                    : make_double2(reinterpret_cast<const double*>(yv)[s], 0.0);
      }
    }
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      if (s0 + u * stride < ns) {
        sr += w[u] * y[u].x;
        if (CPLX) si += w[u] * y[u].y;
      }
    }
  }
  const double br = block_sum(sr);
  const double bi = block_sum(si);
  if (threadIdx.x == 0) {
    red[2 * kVecBlocks + bx] = br;
    red[3 * kVecBlocks + bx] = bi;
  }
}

template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) center_partial_kernel(
    const void* __restrict__ yv, const double* __restrict__ weights, int64_t ns, double* red,
    const double* scal) {
  center_partial_body<CPLX>(blockIdx.x, gridDim.x, yv, weights, ns, red, scal);
}

template <bool CPLX>
__device__ __forceinline__ void center_apply_body(int bx, int gx, 
    const void* __restrict__ yv, void* vout, const double* __restrict__ weights, int64_t ns,
    const double* red, const double* scal, int nb) {
  if (scal[SC_DONE] != 0.0) return;
  const double mr = sum_partials(red + 2 * kVecBlocks, nb);
  const double mi = sum_partials(red + 3 * kVecBlocks, nb);
  const double invn = 1.0 / (double)ns;
  const int64_t stride = (int64_t)gx * blockDim.x;
  for (int64_t s0 = bx * (int64_t)blockDim.x + threadIdx.x; s0 < ns;
       s0 += kVecUnroll * stride) {
    double w[kVecUnroll];
    double2 y[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      const int64_t s = s0 + u * stride;
      if (s < ns) {
        w[u] = weights ? weights[s] : invn;
        y[u] = CPLX ? reinterpret_cast<const double2*>(yv)[s]
                    : make_double2(reinterpret_cast<const double*>(yv)[s], 0.0);
      }
    }
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      const int64_t s = s0 + u * stride;
      if (s < ns) {
        if (CPLX)
          reinterpret_cast<double2*>(vout)[s] =
              make_double2(w[u] * (y[u].x - mr), w[u] * (y[u].y - mi));
        else
          reinterpret_cast<double*>(vout)[s] = w[u] * (y[u].x - mr);
      }
    }
  }
}

template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) center_apply_kernel(
    const void* __restrict__ yv, void* vout, const double* __restrict__ weights, int64_t ns,
    const double* red, const double* scal, int nb) {
  center_apply_body<CPLX>(blockIdx.x, gridDim.x, yv, vout, weights, ns, red, scal, nb);
}

// s + e = a + b exactly (Knuth's TwoSum in FP32)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// out = sum_z part[z] (+ eps * p);  red[b] = sum conj(p) . out (if p given).
// The FP32 partials of the splits are added in split order as an unevaluated
// FP32 pair (running sum and running error of TwoSum), converted to FP64 once:
// FP64 arithmetic is a small fraction of the FP32 rate on this GPU.
// The element X'[m][n] (no parameter) is forced to 0.
template <bool CPLX>
__device__ __forceinline__ void reduce_parts_body(int bx, int gx, 
    const void* __restrict__ partv, int splits, int64_t pa, int64_t corner, void* outv,
    const void* __restrict__ pv, double eps, double* red, const double* scal) {
  if (scal && scal[SC_DONE] != 0.0) return;
  using DT = typename D<CPLX>::T;
  DT* out = reinterpret_cast<DT*>(outv);
  const DT* p = reinterpret_cast<const DT*>(pv);
  double dot = 0.0;
  const int64_t stride = (int64_t)gx * blockDim.x;
  for (int64_t e0 = bx * (int64_t)blockDim.x + threadIdx.x; e0 < pa;
       e0 += kVecUnroll * stride) {
    float2 hi[kVecUnroll], lo[kVecUnroll];
    DT pp[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      hi[u] = make_float2(0.f, 0.f);
      lo[u] = make_float2(0.f, 0.f);
      pp[u] = D<CPLX>::zero();
      if (p && e0 + u * stride < pa) pp[u] = p[e0 + u * stride];
    }
    // the partials of up to kZ splits are loaded together, then added in split order
    constexpr int kZ = 4;
    for (int z0 = 0; z0 < splits; z0 += kZ) {
      float2 v[kZ][kVecUnroll];
#pragma unroll
      for (int zz = 0; zz < kZ; ++zz)
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
          const int64_t e = e0 + u * stride;
          v[zz][u] = make_float2(0.f, 0.f);
          if (z0 + zz < splits && e < pa) {
            const int64_t o = (int64_t)(z0 + zz) * pa + e;
            if constexpr (CPLX) v[zz][u] = reinterpret_cast<const float2*>(partv)[o];
            else v[zz][u].x = reinterpret_cast<const float*>(partv)[o];
          }
        }
#pragma unroll
      for (int zz = 0; zz < kZ; ++zz)
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
          if (z0 + zz < splits) {
            float er;
            two_sum(hi[u].x, v[zz][u].x, hi[u].x, er);
            lo[u].x += er;
            if constexpr (CPLX) {
              two_sum(hi[u].y, v[zz][u].y, hi[u].y, er);
              lo[u].y += er;
            }
          }
        }
    }
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      const int64_t e = e0 + u * stride;
      if (e < pa) {
        DT a;
        if constexpr (CPLX)
          a = make_double2((double)hi[u].x + (double)lo[u].x, (double)hi[u].y + (double)lo[u].y);
        else
          a = (double)hi[u].x + (double)lo[u].x;
        if (p) a = axpy(eps, pp[u], a);
        if (e == corner) a = D<CPLX>::zero();
        out[e] = a;
        if (p) dot += cdot_re(pp[u], a);
      }
    }
  }
  if (red) {
    double b = block_sum(dot);
    if (threadIdx.x == 0) red[bx] = b;
  }
}

template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) reduce_parts_kernel(
    const void* __restrict__ partv, int splits, int64_t pa, int64_t corner, void* outv,
    const void* __restrict__ pv, double eps, double* red, const double* scal) {
  reduce_parts_body<CPLX>(blockIdx.x, gridDim.x, partv, splits, pa, corner, outv, pv, eps, red, scal);
}

// x = 0, r = p = F, rs = ||F||^2 (run after F was reduced into r)
template <bool CPLX>
__device__ __forceinline__ void cg_init_body(int bx, int gx, void* xv, void* rv, void* pv,
                                                              int64_t pa, double* red) {
  using DT = typename D<CPLX>::T;
  DT* x = reinterpret_cast<DT*>(xv);
  DT* r = reinterpret_cast<DT*>(rv);
  DT* p = reinterpret_cast<DT*>(pv);
  double nn = 0.0;
  const int64_t stride = (int64_t)gx * blockDim.x;
  for (int64_t e0 = bx * (int64_t)blockDim.x + threadIdx.x; e0 < pa;
       e0 += kVecUnroll * stride) {
    DT rr[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u)
      if (e0 + u * stride < pa) rr[u] = r[e0 + u * stride];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      const int64_t e = e0 + u * stride;
      if (e < pa) {
        x[e] = D<CPLX>::zero();
        p[e] = rr[u];
        nn += norm2(rr[u]);
      }
    }
  }
  double b = block_sum(nn);
  if (threadIdx.x == 0) red[kVecBlocks + bx] = b;
}

template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) cg_init_kernel(void* xv, void* rv, void* pv,
                                                              int64_t pa, double* red) {
  cg_init_body<CPLX>(blockIdx.x, gridDim.x, xv, rv, pv, pa, red);
}

__device__ __forceinline__ void cg_init_scalars_body(int bx, int gx, const double* red, double* scal, double rtol, int nb) {
  double rs = sum_partials(red + kVecBlocks, nb);
  if (threadIdx.x == 0) {
    scal[SC_RS0] = rs;
    scal[SC_RS1] = rs;
    scal[SC_FNORM] = sqrt(rs);
    scal[SC_ITERS] = 0.0;
    scal[SC_DONE] = (rs == 0.0) ? 1.0 : 0.0;
    if (!isfinite(rs)) {
      scal[SC_NONFINITE] = 1.0;
      scal[SC_DONE] = 1.0;
    }
  }
}

__global__ void cg_init_scalars_kernel(const double* red, double* scal, double rtol, int nb) {
  cg_init_scalars_body(blockIdx.x, gridDim.x, red, scal, rtol, nb);
}

// alpha = rs / p^H A p; x += alpha p; r -= alpha A p; red2 = ||r||^2 partials
template <bool CPLX>
__device__ __forceinline__ void cg_step_x_body(int bx, int gx, void* xv, void* rv,
                                                                const void* pv, const void* apv,
                                                                int64_t pa, double* red,
                                                                double* scal, int it, int nb) {
  if (scal[SC_DONE] != 0.0) return;
  using DT = typename D<CPLX>::T;
  DT* x = reinterpret_cast<DT*>(xv);
  DT* r = reinterpret_cast<DT*>(rv);
  const DT* p = reinterpret_cast<const DT*>(pv);
  const DT* ap = reinterpret_cast<const DT*>(apv);
  const double pap = sum_partials(red, nb);
  const double rs = scal[(it & 1) ? SC_RS1 : SC_RS0];
  const double alpha = rs / pap;
  double nn = 0.0;
  const int64_t stride = (int64_t)gx * blockDim.x;
  for (int64_t e0 = bx * (int64_t)blockDim.x + threadIdx.x; e0 < pa;
       e0 += kVecUnroll * stride) {
    DT pp[kVecUnroll], xx[kVecUnroll], aa[kVecUnroll], rr[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      const int64_t e = e0 + u * stride;
      if (e < pa) {
        pp[u] = p[e];
        xx[u] = x[e];
        aa[u] = ap[e];
        rr[u] = r[e];
      }
    }
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      const int64_t e = e0 + u * stride;
      if (e < pa) {
        x[e] = axpy(alpha, pp[u], xx[u]);
        const DT q = axpy(-alpha, aa[u], rr[u]);
        r[e] = q;
        nn += norm2(q);
      }
    }
  }
  double b = block_sum(nn);
  if (threadIdx.x == 0) red[kVecBlocks + bx] = b;
}

template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) cg_step_x_kernel(void* xv, void* rv,
                                                                const void* pv, const void* apv,
                                                                int64_t pa, double* red,
                                                                double* scal, int it, int nb) {
  cg_step_x_body<CPLX>(blockIdx.x, gridDim.x, xv, rv, pv, apv, pa, red, scal, it, nb);
}

// beta = rs_new / rs; p = r + beta p; convergence test on ||r|| <= rtol ||F||
template <bool CPLX>
__device__ __forceinline__ void cg_step_p_body(int bx, int gx, const void* rv, void* pv,
                                                                int64_t pa, const double* red,
                                                                double* scal, int it,
                                                                double rtol, int nb,
                                                                const PlaneOut& po = PlaneOut{}) {
  if (scal[SC_DONE] != 0.0) return;
  using DT = typename D<CPLX>::T;
  const DT* r = reinterpret_cast<const DT*>(rv);
  DT* p = reinterpret_cast<DT*>(pv);
  const double rs_new = sum_partials(red + kVecBlocks, nb);
  const double rs = scal[(it & 1) ? SC_RS1 : SC_RS0];
  const double fn = scal[SC_FNORM];
  const bool conv = sqrt(rs_new) <= rtol * fn;
  const bool bad = !isfinite(rs_new);
  if (!conv && !bad) {
    const double beta = rs_new / rs;
    const int64_t stride = (int64_t)gx * blockDim.x;
    for (int64_t e0 = bx * (int64_t)blockDim.x + threadIdx.x; e0 < pa;
         e0 += kVecUnroll * stride) {
      DT pp[kVecUnroll], rr[kVecUnroll];
#pragma unroll
      for (int u = 0; u < kVecUnroll; ++u) {
        const int64_t e = e0 + u * stride;
        if (e < pa) {
          pp[u] = p[e];
          rr[u] = r[e];
        }
      }
#pragma unroll
      for (int u = 0; u < kVecUnroll; ++u) {
        const int64_t e = e0 + u * stride;
        if (e < pa) {
          const DT q = axpy(beta, pp[u], rr[u]);
          p[e] = q;
          if (po.planes) {
            // the BF16 hi/lo planes of the new p for the next forward contraction
            const int j = (int)(e / po.na), i = (int)(e % po.na);
            const int64_t pl = (int64_t)po.mt * 128 * po.na64;
            uint32_t hi, lo;
            split_bf16(re(q), hi, lo);
            const int64_t k0 = bplane_index(j, i, 0, CPLX, po.na64);
            po.planes[k0] = (uint16_t)hi;
            po.planes[pl + k0] = (uint16_t)lo;
            if constexpr (CPLX) {
              split_bf16(im(q), hi, lo);
              const int64_t k1 = bplane_index(j, i, 1, CPLX, po.na64);
              po.planes[k1] = (uint16_t)hi;
              po.planes[pl + k1] = (uint16_t)lo;
            }
          }
        }
      }
    }
  }
  if (bx == 0 && threadIdx.x == 0) {
    scal[(it & 1) ? SC_RS0 : SC_RS1] = rs_new;
    scal[SC_ITERS] = (double)(it + 1);
    if (conv || bad) scal[SC_DONE] = 1.0;
    if (bad) scal[SC_NONFINITE] = 1.0;
  }
}

template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) cg_step_p_kernel(const void* rv, void* pv,
                                                                int64_t pa, const double* red,
                                                                double* scal, int it,
                                                                double rtol, int nb,
                                                                PlaneOut po) {
  cg_step_p_body<CPLX>(blockIdx.x, gridDim.x, rv, pv, pa, red, scal, it, rtol, nb, po);
}

__device__ __forceinline__ void sr_write_info(const double* scal, double* info, double rtol);

// alpha <- alpha - lr delta (FP64 master), delta in the augmented layout; info.
template <bool CPLX>
__device__ __forceinline__ void sr_update_body(int bx, int gx, double* a, double* b, double* w, int n, int m,
                                 const void* __restrict__ xv, double lr, const double* scal,
                                 double* info, int n_iter_final, double rtol) {
  using DT = typename D<CPLX>::T;
  const DT* x = reinterpret_cast<const DT*>(xv);
  const int na = n + 1;
  const int64_t tot = (int64_t)(m + 1) * na;
  for (int64_t e = bx * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gx * blockDim.x) {
    int j = (int)(e / na), i = (int)(e % na);
    double* dst;
    if (j < m && i < n) dst = w + (CPLX ? 2 : 1) * ((int64_t)j * n + i);
    else if (j < m) dst = b + (CPLX ? 2 : 1) * j;
    else if (i < n) dst = a + (CPLX ? 2 : 1) * i;
    else continue;
    if constexpr (CPLX) {
      dst[0] -= lr * x[e].x;
      dst[1] -= lr * x[e].y;
    } else {
      dst[0] -= lr * x[e];
    }
  }
  if (bx == 0 && threadIdx.x == 0) sr_write_info(scal, info, rtol);
}

// info {CG iterations, residual, ||F||, flags} from the CG scalars (one thread)
__device__ __forceinline__ void sr_write_info(const double* scal, double* info, double rtol) {
  {
    const double iters = scal[SC_ITERS];
    const double fn = scal[SC_FNORM];
    const double rs = scal[((int)iters & 1) ? SC_RS1 : SC_RS0];
    const double res = fn > 0.0 ? sqrt(rs) / fn : 0.0;
    info[NK_INFO_CG_ITERS] = iters;
    info[NK_INFO_CG_RESID] = res;
    info[NK_INFO_F_NORM] = fn;
    int flags = 0;
    if (res > rtol) flags |= 1 << NK_ERR_NOT_CONVERGED;
    if (scal[SC_NONFINITE] != 0.0 || !isfinite(res)) flags |= 1 << NK_ERR_NONFINITE;
    if (*reinterpret_cast<const int*>(scal + SC_ERR) != 0) flags |= 1 << NK_ERR_TIMEOUT;
    info[NK_INFO_FLAGS] = (double)flags;
  }
}

template <bool CPLX>
__global__ void sr_update_kernel(double* a, double* b, double* w, int n, int m,
                                 const void* __restrict__ xv, double lr, const double* scal,
                                 double* info, int n_iter_final, double rtol) {
  sr_update_body<CPLX>(blockIdx.x, gridDim.x, a, b, w, n, m, xv, lr, scal, info, n_iter_final, rtol);
}

// ------------------------------------------------------------------ symmetric RBM
// Tied parameters in the augmented layout [alpha + 1][n + 1]: (f, i < n) = Wt[f][i],
// (f, n) = bt[f], (alpha, 0) = at; the other entries of the last row stand for
// nothing and stay 0 in every CG vector (their fold lists are empty).

__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double shfl_xor(double v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ double2 shfl_xor(double2 v, int o) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// P x: out[e] = x[tie[e]] over the untied augmented layout (0 where tie < 0)
template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) symm_expand_vec_kernel(
    const void* __restrict__ xv, const int* __restrict__ tie, int64_t pa, void* outv,
    const double* scal) {
  if (scal && scal[SC_DONE] != 0.0) return;
  using DT = typename D<CPLX>::T;
  const DT* x = reinterpret_cast<const DT*>(xv);
  DT* out = reinterpret_cast<DT*>(outv);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < pa;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = tie[e];
    out[e] = k >= 0 ? x[k] : D<CPLX>::zero();
  }
}

// P^T u (+ eps p): one warp per tied element sums its untied elements (lane l
// takes list entries l, l + 32, ..., then a fixed xor tree), so the result does
// not depend on scheduling; with p, per-block partials of Re p^H out -> red[bx].
template <bool CPLX>
__global__ void __launch_bounds__(kVecThreads) symm_fold_kernel(
    const void* __restrict__ uv, const int* __restrict__ off, const int* __restrict__ idx,
    int64_t pa_t, void* outv, const void* __restrict__ pv, double eps, double* red,
    const double* scal) {
  if (scal && scal[SC_DONE] != 0.0) return;
  using DT = typename D<CPLX>::T;
  const DT* u = reinterpret_cast<const DT*>(uv);
  const DT* p = reinterpret_cast<const DT*>(pv);
  DT* out = reinterpret_cast<DT*>(outv);
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < pa_t; q += nw) {
    DT acc = D<CPLX>::zero();
    const int k1 = off[q + 1];
    for (int k = off[q] + lane; k < k1; k += 32) acc = vadd(acc, u[idx[k]]);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc = vadd(acc, shfl_xor(acc, o));
    if (lane == 0) {
      if (p) {
        acc = axpy(eps, p[q], acc);
        dot += cdot_re(p[q], acc);
      }
      out[q] = acc;
    }
  }
  if (red) {
    const double b = block_sum(dot);
    if (threadIdx.x == 0) red[blockIdx.x] = b;
  }
}

// theta_t <- theta_t - lr delta (tied layout); info
template <bool CPLX>
__global__ void symm_update_kernel(double* a, double* b, double* w, int n, int alpha,
                                   const void* __restrict__ xv, double lr,
                                   const double* scal, double* info, double rtol) {
  using DT = typename D<CPLX>::T;
  const DT* x = reinterpret_cast<const DT*>(xv);
  const int na = n + 1, c = CPLX ? 2 : 1;
  const int64_t tot = (int64_t)(alpha + 1) * na;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(e / na), i = (int)(e % na);
    double* dst;
    if (f < alpha && i < n) dst = w + c * ((int64_t)f * n + i);
    else if (f < alpha) dst = b + c * f;
    else if (i == 0) dst = a;
    else continue;
    if constexpr (CPLX) {
      dst[0] -= lr * x[e].x;
      dst[1] -= lr * x[e].y;
    } else {
      dst[0] -= lr * x[e];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sr_write_info(scal, info, rtol);
}

// untied (a, b, W) from the tied parameters: a_i = at, b_(f,g) = bt_f,
// W[(f,g)][i] = Wt[f][perm[g][i]]
__global__ void symm_params_kernel(const double* __restrict__ ta, const double* __restrict__ tb,
                                   const double* __restrict__ tw, int n, int alpha, int ng,
                                   const int* __restrict__ perm, int cplx, double* a, double* b,
                                   double* w) {
  const int m = alpha * ng, c = cplx ? 2 : 1;
  const int64_t nw = (int64_t)m * n, tot = nw + m + n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double* src;
    double* dst;
    if (e < nw) {
      const int j = (int)(e / n), i = (int)(e % n);
      src = tw + c * ((int64_t)(j / ng) * n + perm[(int64_t)(j % ng) * n + i]);
      dst = w + c * e;
    } else if (e < nw + m) {
      const int j = (int)(e - nw);
      src = tb + c * (j / ng);
      dst = b + c * j;
    } else {
      src = ta;
      dst = a + c * (e - nw - m);
    }
    dst[0] = src[0];
    if (c == 2) dst[1] = src[1];
  }
}

// grad (a, b, W order) from the augmented adjoint result
template <bool CPLX>
__global__ void scatter_grad_kernel(const void* __restrict__ gv, int n, int m, double* grad) {
  using DT = typename D<CPLX>::T;
  const DT* g = reinterpret_cast<const DT*>(gv);
  const int na = n + 1;
  const int64_t tot = (int64_t)(m + 1) * na;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int j = (int)(e / na), i = (int)(e % na);
    int64_t k;
    if (j < m && i < n) k = (int64_t)n + m + (int64_t)j * n + i;
    else if (j < m) k = n + j;
    else if (i < n) k = i;
    else continue;
    if constexpr (CPLX) {
      grad[2 * k] = g[e].x;
      grad[2 * k + 1] = g[e].y;
    } else {
      grad[k] = g[e];
    }
  }
}

// ------------------------------------------------------------------ batched kernels
// The same kernels for every problem of an SR batch: blockIdx.y selects the
// problem (its SrDesc; complex and real problems share a launch and branch on
// its field), blockIdx.x runs over the problem's own grid (the one the
// single-problem launch uses), so each problem's reductions keep their order
// and a batched step computes exactly what nk_sr_step computes for it.

__global__ void __launch_bounds__(kVecThreads) stats_mean_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_ns) return;
  if (d.cplx) stats_mean_body<true>(blockIdx.x, d.nb_ns, d.eloc, d.weights, d.ns, d.red);
  else stats_mean_body<false>(blockIdx.x, d.nb_ns, d.eloc, d.weights, d.ns, d.red);
}

__global__ void __launch_bounds__(kVecThreads) stats_dev_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_ns) return;
  if (d.cplx)
    stats_dev_body<true>(blockIdx.x, d.nb_ns, d.eloc, d.weights, d.ns, d.n_chains, d.red, d.v,
                         d.nb_ns);
  else
    stats_dev_body<false>(blockIdx.x, d.nb_ns, d.eloc, d.weights, d.ns, d.n_chains, d.red, d.v,
                          d.nb_ns);
}

__global__ void stats_finish_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  stats_finish_body(d.weights, d.ns, d.n_chains, d.red, d.nb_ns, d.info, d.scal);
}

__global__ void flags_reset_batch(const SrDesc* __restrict__ D) {
  if (threadIdx.x == 0) {
    D[blockIdx.y].scal[SC_DONE] = 0.0;
    D[blockIdx.y].scal[SC_ERR] = 0.0;
  }
}

// in_cg = 0: F into r (no shift, no inner product); 1: S p + eps p into ap
__global__ void __launch_bounds__(kVecThreads) reduce_parts_batch(const SrDesc* __restrict__ D,
                                                                  int in_cg, double eps) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_pa) return;
  char* out = in_cg ? d.ap : d.r;
  const void* p = in_cg ? d.p : nullptr;
  double* red = in_cg ? d.red : nullptr;
  const double* scal = in_cg ? d.scal : nullptr;
  const double e = in_cg ? eps : 0.0;
  if (d.cplx)
    reduce_parts_body<true>(blockIdx.x, d.nb_pa, d.part, d.splits, d.pa, d.corner, out, p, e,
                            red, scal);
  else
    reduce_parts_body<false>(blockIdx.x, d.nb_pa, d.part, d.splits, d.pa, d.corner, out, p, e,
                             red, scal);
}

__global__ void __launch_bounds__(kVecThreads) cg_init_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_pa) return;
  if (d.cplx)
    cg_init_body<true>(blockIdx.x, d.nb_pa, d.x, d.r, d.p, d.pa, d.red);
  else
    cg_init_body<false>(blockIdx.x, d.nb_pa, d.x, d.r, d.p, d.pa, d.red);
}

__global__ void cg_init_scalars_batch(const SrDesc* __restrict__ D, double rtol) {
  const SrDesc& d = D[blockIdx.y];
  cg_init_scalars_body(0, 1, d.red, d.scal, rtol, d.nb_pa);
}

__global__ void __launch_bounds__(kVecThreads) center_partial_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_ns || d.ctr_parts > 0) return;  // else the forward wrote them
  if (d.cplx)
    center_partial_body<true>(blockIdx.x, d.nb_ns, d.y, d.weights, d.ns, d.red, d.scal);
  else
    center_partial_body<false>(blockIdx.x, d.nb_ns, d.y, d.weights, d.ns, d.red, d.scal);
}

__global__ void __launch_bounds__(kVecThreads) center_apply_batch(const SrDesc* __restrict__ D) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_ns) return;
  const int parts = d.ctr_parts > 0 ? d.ctr_parts : d.nb_ns;
  if (d.cplx)
    center_apply_body<true>(blockIdx.x, d.nb_ns, d.y, d.v, d.weights, d.ns, d.red, d.scal,
                            parts);
  else
    center_apply_body<false>(blockIdx.x, d.nb_ns, d.y, d.v, d.weights, d.ns, d.red, d.scal,
                             parts);
}

__global__ void __launch_bounds__(kVecThreads) cg_step_x_batch(const SrDesc* __restrict__ D,
                                                               int it) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_pa) return;
  if (d.cplx)
    cg_step_x_body<true>(blockIdx.x, d.nb_pa, d.x, d.r, d.p, d.ap, d.pa, d.red, d.scal, it,
                       d.nb_pa);
  else
    cg_step_x_body<false>(blockIdx.x, d.nb_pa, d.x, d.r, d.p, d.ap, d.pa, d.red, d.scal, it,
                       d.nb_pa);
}

__global__ void __launch_bounds__(kVecThreads) cg_step_p_batch(const SrDesc* __restrict__ D,
                                                               int it, double rtol) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_pa) return;
  PlaneOut po;
  po.planes = reinterpret_cast<uint16_t*>(d.xbf);
  po.na = d.n + 1;
  po.mt = d.mt1;
  po.na64 = d.na64;
  if (d.cplx)
    cg_step_p_body<true>(blockIdx.x, d.nb_pa, d.r, d.p, d.pa, d.red, d.scal, it, rtol, d.nb_pa,
                         po);
  else
    cg_step_p_body<false>(blockIdx.x, d.nb_pa, d.r, d.p, d.pa, d.red, d.scal, it, rtol, d.nb_pa,
                          po);
  if (d.fwd_nseg == 2) {
    // the next forward's two halves add onto zero (y of this iteration is consumed)
    double* y = reinterpret_cast<double*>(d.y);
    const int64_t len = d.ns * (d.cplx ? 2 : 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
         e += (int64_t)d.nb_pa * blockDim.x)
      y[e] = 0.0;
  }
}

__global__ void sr_update_batch(const SrDesc* __restrict__ D, double lr, int n_cg, double rtol) {
  const SrDesc& d = D[blockIdx.y];
  if ((int)blockIdx.x >= d.nb_pa) return;
  if (d.cplx)
    sr_update_body<true>(blockIdx.x, d.nb_pa, d.a, d.b, d.w, d.n, d.m, d.x, lr, d.scal, d.info,
                       n_cg, rtol);
  else
    sr_update_body<false>(blockIdx.x, d.nb_pa, d.a, d.b, d.w, d.n, d.m, d.x, lr, d.scal, d.info,
                       n_cg, rtol);
}

// ------------------------------------------------------------------ drivers

// A symmetric RBM's tables, tied parameters and tied CG vectors (nk_sr_step_symm).
struct SymmRun {
  const int *tie, *off, *idx, *perm;
  int64_t pa_t;
  int alpha, n_perm;
  double *a, *b, *w;
  char *x, *r, *p, *ap;
};

// sy = NULL: SR in the RBM's own parameters.  sy: SR in the tied parameters;
// the untied vectors x, r, p, ap of the scratch then hold expanded and
// not-yet-folded products only.
template <bool CPLX>
static nk_status sr_step_t(nk_rbm* r, const int8_t* sigma, const void* T, const double* eloc,
                           const double* weights, int64_t ns, int n_chains, double eps,
                           double lr, int n_cg, double rtol, int prec, char* sc,
                           double* info, cudaStream_t st, const SymmRun* sy = nullptr) {
  SrLayout L(r->n, r->m, CPLX, ns);
  double* scal = (double*)(sc + L.scal);
  double* red = (double*)(sc + L.red);
  const int n = r->n, m = r->m;
  const int64_t corner = (int64_t)m * L.na + n;
  const bool tc = prec == NK_PREC_BF16X2;
  // the CG runs on these vectors (the tied ones for a symmetric RBM)
  const int64_t pa_cg = sy ? sy->pa_t : L.pa;
  char* cx = sy ? sy->x : sc + L.x;
  char* cr = sy ? sy->r : sc + L.r;
  char* cp = sy ? sy->p : sc + L.p;
  char* cap = sy ? sy->ap : sc + L.ap;
  const int nbc = sr_vec_blocks(pa_cg);
  const int nbf = sy ? (int)std::min<int64_t>(kVecBlocks, (pa_cg + 7) / 8) : 0;
  int* err = reinterpret_cast<int*>(scal + SC_ERR);
  const int splits = sr_choose_splits(L, prec, r->sr_splits);
  AdjTcArgs aa{};
  FwdTcArgs fa{};
  if (tc) {
    aa.T = T;
    aa.ns = ns;
    aa.n = n;
    aa.m = m;
    aa.cplx = CPLX;
    aa.na64 = L.na64;
    aa.splits = splits;
    aa.part = sc + L.part;
    aa.err = err;
    fa.sigma = sigma;
    fa.ns = ns;
    fa.n = n;
    fa.m = m;
    fa.cplx = CPLX;
    fa.mode = 0;
    fa.mt = L.mt1;
    fa.na64 = L.na64;
    fa.rows = m + 1;
    fa.T = T;
    fa.y = sc + L.y;
    fa.skip = scal + SC_DONE;
    fa.err = err;
    fa.sig_rows = sc + L.sigr;
  }
  {
    const int nbs0 = sr_vec_blocks(ns);
    stats_mean_kernel<CPLX><<<nbs0, kVecThreads, 0, st>>>(eloc, weights, ns, red);
    stats_dev_kernel<CPLX><<<nbs0, kVecThreads, 0, st>>>(eloc, weights, ns, n_chains, red,
                                                        sc + L.v, nbs0);
    stats_finish_kernel<<<1, 32, 0, st>>>(weights, ns, n_chains, red, nbs0, info, scal);
  }
  if (nk_status e = check_launch("nk_sr_step(stats)")) return e;
  cudaMemsetAsync(scal + SC_DONE, 0, sizeof(double), st);
  cudaMemsetAsync(scal + SC_ERR, 0, sizeof(double), st);
  // F = adjoint(w o (E - <E>)) -> r
  if (tc) {
    if (nk_status e = launch_sigma_t(sigma, ns, n, L.na64, sc + L.sigt, st)) return e;
    if (nk_status e = launch_sigma_rows(sigma, ns, n, L.na64, sc + L.sigr, st)) return e;
    aa.v = sc + L.v;
    aa.skip = nullptr;
    if (nk_status e = launch_adj_tc(aa, sc + L.sigt, st)) return e;
  } else {
    launch_adjoint_fp32<CPLX>(sigma, T, sc + L.v, ns, n, m, splits, sc + L.part, nullptr, st);
  }
  const int nbp = sr_vec_blocks(L.pa), nbs = sr_vec_blocks(ns);
  reduce_parts_kernel<CPLX><<<nbp, kVecThreads, 0, st>>>(sc + L.part, splits, L.pa, corner,
                                                         sc + L.r, nullptr, 0.0, nullptr,
                                                         nullptr);
  if (sy)
    symm_fold_kernel<CPLX><<<nbf, kVecThreads, 0, st>>>(sc + L.r, sy->off, sy->idx, pa_cg, cr,
                                                        nullptr, 0.0, nullptr, nullptr);
  cg_init_kernel<CPLX><<<nbc, kVecThreads, 0, st>>>(cx, cr, cp, pa_cg, red);
  cg_init_scalars_kernel<<<1, 32, 0, st>>>(red, scal, rtol, nbc);
  if (nk_status e = check_launch("nk_sr_step(force)")) return e;
  const int64_t sg_blocks = (ns + kSgBS - 1) / kSgBS;
  aa.v = sc + L.v;
  aa.skip = scal + SC_DONE;
  // The tensor-core forward also writes the partial sums of the centring mean
  // (one per CTA), when they fit the partials buffer: no separate partial pass.
  const int ctr_parts = tc ? fwd_centring_parts(ns, L.mt1) : 0;
  if (ctr_parts) {
    fa.mean_part = red + 2 * kVecBlocks;
    fa.mean_stride = kVecBlocks;
    fa.weights = weights;
  }
  // and for small hidden layers the adjoint centres y itself while loading it
  const bool adj_ctr = ctr_parts && adj_centres(m, CPLX);
  if (adj_ctr) {
    aa.y = sc + L.y;
    aa.mean_part = red + 2 * kVecBlocks;
    aa.mean_stride = kVecBlocks;
    aa.mean_parts = ctr_parts;
    aa.weights = weights;
  }
  // from the second CG iteration on, cg_step_p writes the planes of p itself
  PlaneOut po;
  if (tc) {
    po.planes = (uint16_t*)(sc + L.xbf);
    po.na = L.na;
    po.mt = L.mt1;
    po.na64 = L.na64;
  }
  for (int it = 0; it < n_cg; ++it) {
    if (sy)  // the untied p = P p_t for the contractions
      symm_expand_vec_kernel<CPLX><<<nbp, kVecThreads, 0, st>>>(cp, sy->tie, L.pa, sc + L.p,
                                                                scal);
    if (tc) {
      if (it == 0 || sy) {
        if (nk_status e = launch_bplanes_from_f64(sc + L.p, m + 1, n + 1, L.na, CPLX, L.mt1,
                                                  L.na64, sc + L.xbf, scal + SC_DONE, st))
          return e;
      }
      if (nk_status e = launch_fwd_tc(fa, sc + L.xbf, st)) return e;
    } else {
      to_f32_kernel<CPLX><<<nbp, kVecThreads, 0, st>>>(sc + L.p, sc + L.xf, L.pa, scal);
      forward_fp32_kernel<CPLX><<<(unsigned)sg_blocks, kSgThreads, 0, st>>>(
          sigma, ns, n, m, sc + L.xf, T, sc + L.y, scal);
    }
    if (ctr_parts == 0)
      center_partial_kernel<CPLX><<<nbs, kVecThreads, 0, st>>>(sc + L.y, weights, ns, red, scal);
    if (!adj_ctr)
      center_apply_kernel<CPLX><<<nbs, kVecThreads, 0, st>>>(sc + L.y, sc + L.v, weights, ns,
                                                             red, scal, ctr_parts ? ctr_parts : nbs);
    if (tc) {
      if (nk_status e = launch_adj_tc(aa, sc + L.sigt, st)) return e;
    } else {
      launch_adjoint_fp32<CPLX>(sigma, T, sc + L.v, ns, n, m, splits, sc + L.part, scal, st);
    }
    if (sy) {  // S_t p_t + eps p_t = P^T (S P p_t) + eps p_t
      reduce_parts_kernel<CPLX><<<nbp, kVecThreads, 0, st>>>(
          sc + L.part, splits, L.pa, corner, sc + L.ap, nullptr, 0.0, nullptr, scal);
      symm_fold_kernel<CPLX><<<nbf, kVecThreads, 0, st>>>(sc + L.ap, sy->off, sy->idx, pa_cg,
                                                          cap, cp, eps, red, scal);
    } else {
      reduce_parts_kernel<CPLX><<<nbp, kVecThreads, 0, st>>>(
          sc + L.part, splits, L.pa, corner, sc + L.ap, sc + L.p, eps, red, scal);
    }
    cg_step_x_kernel<CPLX><<<nbc, kVecThreads, 0, st>>>(cx, cr, cp, cap, pa_cg, red, scal, it,
                                                        sy ? nbf : nbc);
    cg_step_p_kernel<CPLX><<<nbc, kVecThreads, 0, st>>>(cr, cp, pa_cg, red, scal, it, rtol, nbc,
                                                        sy ? PlaneOut{} : po);
    if (nk_status e = check_launch("nk_sr_step(cg)")) return e;
  }
  if (sy) {
    symm_update_kernel<CPLX><<<nbc, kVecThreads, 0, st>>>(sy->a, sy->b, sy->w, n, sy->alpha, cx,
                                                          lr, scal, info, rtol);
    symm_params_kernel<<<nbp, kVecThreads, 0, st>>>(sy->a, sy->b, sy->w, n, sy->alpha,
                                                    sy->n_perm, sy->perm, CPLX, r->a, r->b, r->w);
  } else {
    sr_update_kernel<CPLX><<<nbp, kVecThreads, 0, st>>>(r->a, r->b, r->w, n, m, sc + L.x, lr,
                                                        scal, info, n_cg, rtol);
  }
  if (nk_status e = check_launch("nk_sr_step(update)")) return e;
  return launch_prepare(r, st);
}

nk_status run_sr_step(nk_rbm* r, const int8_t* sigma, const void* t, const double* eloc,
                      const double* weights, int64_t ns, int n_chains, double diag_shift,
                      double lr, int n_cg, double cg_rtol, int prec, void* scratch,
                      size_t scratch_bytes, double* info, cudaStream_t st) {
  size_t need = sr_scratch_bytes(r->n, r->m, r->is_complex, ns);
  if (scratch_bytes < need)
    return fail(NK_ERR_SHAPE, "nk_sr_step: scratch of %zu B, need %zu B", scratch_bytes, need);
  if (r->is_complex)
    return sr_step_t<true>(r, sigma, t, eloc, weights, ns, n_chains, diag_shift, lr, n_cg, cg_rtol,
                           prec, (char*)scratch, info, st);
  return sr_step_t<false>(r, sigma, t, eloc, weights, ns, n_chains, diag_shift, lr, n_cg, cg_rtol,
                          prec, (char*)scratch, info, st);
}

// ------------------------------------------------------------------ symmetric RBM (host)

SymmTables::SymmTables(int n_, int alpha_, int n_perm_) : n(n_), alpha(alpha_), n_perm(n_perm_) {
  const int64_t m = (int64_t)alpha * n_perm;
  pa = (m + 1) * (n + 1);
  pa_t = (int64_t)(alpha + 1) * (n + 1);
  size_t o = 0;
  auto take = [&](int64_t count) {
    size_t at = o;
    o += (size_t)round_up(count * (int64_t)sizeof(int32_t), 256);
    return at;
  };
  perm = take((int64_t)n_perm * n);
  tie = take(pa);
  off = take(pa_t + 1);
  idx = take(std::max<int64_t>(pa - 1, 1));
  total = o;
}

// tie: untied augmented element (j, i) -> tied element; the fold lists are the
// untied elements of each tied one in ascending order (a counting sort).
nk_status symm_build_tables(const int32_t* perm, int n, int alpha, int n_perm,
                            std::vector<int32_t>* out) {
  const SymmTables T(n, alpha, n_perm);
  std::vector<char> seen((size_t)n);
  for (int g = 0; g < n_perm; ++g) {
    std::fill(seen.begin(), seen.end(), 0);
    for (int i = 0; i < n; ++i) {
      const int32_t k = perm[(int64_t)g * n + i];
      if (k < 0 || k >= n || seen[k])
        return fail(NK_ERR_INVALID_ARG, "nk_symm_upload: row %d of perm is not a permutation", g);
      seen[k] = 1;
    }
  }
  out->assign(T.total / sizeof(int32_t), 0);
  int32_t* base = out->data();
  int32_t* P = base + T.perm / 4;
  int32_t* tie = base + T.tie / 4;
  int32_t* off = base + T.off / 4;
  int32_t* idx = base + T.idx / 4;
  std::copy(perm, perm + (int64_t)n_perm * n, P);
  const int na = n + 1, m = alpha * n_perm;
  for (int j = 0; j <= m; ++j)
    for (int i = 0; i <= n; ++i) {
      int64_t t;
      if (j < m && i < n) t = (int64_t)(j / n_perm) * na + perm[(int64_t)(j % n_perm) * n + i];
      else if (j < m) t = (int64_t)(j / n_perm) * na + n;
      else if (i < n) t = (int64_t)alpha * na;
      else t = -1;
      tie[(int64_t)j * na + i] = (int32_t)t;
    }
  std::vector<int64_t> cnt((size_t)T.pa_t + 1, 0);
  for (int64_t e = 0; e < T.pa; ++e)
    if (tie[e] >= 0) ++cnt[(size_t)tie[e] + 1];
  for (int64_t q = 0; q < T.pa_t; ++q) cnt[(size_t)q + 1] += cnt[(size_t)q];
  for (int64_t q = 0; q <= T.pa_t; ++q) off[q] = (int32_t)cnt[(size_t)q];
  for (int64_t e = 0; e < T.pa; ++e)
    if (tie[e] >= 0) idx[cnt[(size_t)tie[e]]++] = (int32_t)e;
  return NK_OK;
}

static size_t symm_vec_bytes(int n, int alpha, int cplx) {
  return (size_t)round_up((int64_t)(alpha + 1) * (n + 1) * (cplx ? 16 : 8), 256);
}

size_t sr_symm_scratch_bytes(int n, int alpha, int n_perm, int cplx, int64_t ns) {
  return sr_scratch_bytes(n, alpha * n_perm, cplx, ns) + 4 * symm_vec_bytes(n, alpha, cplx);
}

static SymmRun symm_run(const nk_rbm_symm* s, char* vec) {
  const SymmTables T(s->n, s->alpha, s->n_perm);
  const char* tb = (const char*)s->tables;
  SymmRun y;
  y.perm = (const int*)(tb + T.perm);
  y.tie = (const int*)(tb + T.tie);
  y.off = (const int*)(tb + T.off);
  y.idx = (const int*)(tb + T.idx);
  y.pa_t = T.pa_t;
  y.alpha = s->alpha;
  y.n_perm = s->n_perm;
  y.a = s->a;
  y.b = s->b;
  y.w = s->w;
  y.x = y.r = y.p = y.ap = nullptr;
  if (vec) {
    const size_t vb = symm_vec_bytes(s->n, s->alpha, s->is_complex);
    y.x = vec;
    y.r = vec + vb;
    y.p = vec + 2 * vb;
    y.ap = vec + 3 * vb;
  }
  return y;
}

nk_status run_symm_expand(const nk_rbm_symm* s, nk_rbm* r, cudaStream_t st) {
  const SymmRun y = symm_run(s, nullptr);
  const int64_t tot = (int64_t)r->m * r->n + r->m + r->n;
  const int blocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (tot + 1023) / 1024));
  symm_params_kernel<<<blocks, kVecThreads, 0, st>>>(s->a, s->b, s->w, s->n, s->alpha, s->n_perm,
                                                     y.perm, s->is_complex, r->a, r->b, r->w);
  if (nk_status e = check_launch("nk_symm_expand")) return e;
  return launch_prepare(r, st);
}

nk_status run_sr_step_symm(nk_rbm_symm* s, nk_rbm* r, const int8_t* sigma, const void* t,
                           const double* eloc, const double* weights, int64_t ns,
                           int n_chains, double diag_shift, double lr, int n_cg,
                           double cg_rtol, int prec, void* scratch, size_t scratch_bytes,
                           double* info, cudaStream_t st) {
  const size_t base = sr_scratch_bytes(r->n, r->m, r->is_complex, ns);
  const size_t need = sr_symm_scratch_bytes(s->n, s->alpha, s->n_perm, s->is_complex, ns);
  if (scratch_bytes < need)
    return fail(NK_ERR_SHAPE, "nk_sr_step_symm: scratch of %zu B, need %zu B", scratch_bytes,
                need);
  const SymmRun y = symm_run(s, (char*)scratch + base);
  if (r->is_complex)
    return sr_step_t<true>(r, sigma, t, eloc, weights, ns, n_chains, diag_shift, lr, n_cg,
                           cg_rtol, prec, (char*)scratch, info, st, &y);
  return sr_step_t<false>(r, sigma, t, eloc, weights, ns, n_chains, diag_shift, lr, n_cg,
                          cg_rtol, prec, (char*)scratch, info, st, &y);
}

// ------------------------------------------------------------------ SR batches

// Split count of item i of a batch: the RBM's own setting, else a batch-wide
// default that spreads about two waves of adjoint CTAs over all problems.
static int batch_item_splits(const nk_sr_batch_item* items, int n_inst, int i, int prec) {
  const nk_rbm* r = items[i].rbm;
  SrLayout L(r->n, r->m, r->is_complex, items[i].ns);
  if (r->sr_splits > 0) return sr_choose_splits(L, prec, r->sr_splits);
  int64_t tiles = 0;
  for (int k = 0; k < n_inst; ++k) {
    const int hj = items[k].rbm->is_complex ? 64 : 128;
    tiles += (items[k].rbm->m + 1 + hj - 1) / hj;
  }
  // about four CTAs per SM over the whole batch: the instances' CTAs differ in
  // work (sites padded to 64 or 128, 1-7 hidden tiles), and finer pieces end the
  // launch with less idle time (64 uneven 1D instances: 34.5 -> 32.6 ms per
  // iteration against two per SM; eight per SM: 33.4)
  const int s = (int)std::max<int64_t>(1, (4 * 152) / std::max<int64_t>(tiles, 1));
  return sr_choose_splits(L, prec, s);
}

// Problems in descriptor order: complex ones first, then real ones (items order
// within each field).
static std::vector<int> batch_order(const nk_sr_batch_item* items, int n_inst) {
  std::vector<int> order;
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < n_inst; ++i)
      if ((items[i].rbm->is_complex != 0) == (pass == 0)) order.push_back(i);
  return order;
}

nk_status sr_batch_check(const nk_sr_batch_item* items, int n_inst, int prec) {
  if (n_inst < 1 || !items) return fail(NK_ERR_INVALID_ARG, "SR batch: no items");
  if (prec != NK_PREC_BF16X2)
    return fail(NK_ERR_UNSUPPORTED, "SR batch: only the tensor-core precision NK_PREC_BF16X2");
  for (int i = 0; i < n_inst; ++i) {
    const nk_sr_batch_item& it = items[i];
    const nk_rbm* r = it.rbm;
    if (!r || !r->ws || !r->a || !r->b || !r->w)
      return fail(NK_ERR_INVALID_ARG, "SR batch: item %d has no RBM or workspace", i);
    if (it.ns < 1 || !it.sigma || !it.t || !it.eloc || !it.scratch || !it.info_out)
      return fail(NK_ERR_INVALID_ARG, "SR batch: item %d: NULL pointer or ns < 1", i);
    if (it.n_chains < 0 || (it.n_chains > 0 && it.ns % it.n_chains))
      return fail(NK_ERR_SHAPE, "SR batch: item %d: ns not a multiple of n_chains", i);
    if (((uintptr_t)it.scratch) & 255)
      return fail(NK_ERR_INVALID_ARG, "SR batch: item %d: scratch not 256-byte aligned", i);
    if (it.scratch_bytes < sr_scratch_bytes(r->n, r->m, r->is_complex, it.ns))
      return fail(NK_ERR_SHAPE, "SR batch: item %d: scratch too small", i);
    if (!tc_supported_shape(r->n, r->m))
      return fail(NK_ERR_UNSUPPORTED, "SR batch: item %d: n + 1 > 448", i);
  }
  return NK_OK;
}

size_t sr_batch_desc_bytes(int n_inst) { return (size_t)std::max(n_inst, 0) * sizeof(SrDesc); }

nk_status sr_batch_describe(const nk_sr_batch_item* items, int n_inst, int prec, void* host,
                            size_t bytes) {
  if (nk_status e = sr_batch_check(items, n_inst, prec)) return e;
  if (!host || bytes < sr_batch_desc_bytes(n_inst))
    return fail(NK_ERR_SHAPE, "SR batch: descriptor buffer of %zu B, need %zu B", bytes,
                sr_batch_desc_bytes(n_inst));
  const std::vector<int> order = batch_order(items, n_inst);
  SrDesc* out = reinterpret_cast<SrDesc*>(host);
  for (int z = 0; z < n_inst; ++z) {
    const nk_sr_batch_item& it = items[order[z]];
    nk_rbm* r = it.rbm;
    const int cplx = r->is_complex ? 1 : 0;
    SrLayout L(r->n, r->m, cplx, it.ns);
    WsLayout W(r->n, r->m, cplx);
    SrDesc d;
    memset(&d, 0, sizeof(d));
    char* sc = (char*)it.scratch;
    if (!tc_make_map(&d.fwd_map, sc + L.xbf, 2LL * L.mt1 * 128, L.na64, L.na64, 128))
      return NK_ERR_CUDA;
    if (!tc_make_map(&d.adj_map, sc + L.sigt, L.na64, L.ns8, L.ns8, L.na64 / 2))
      return NK_ERR_CUDA;
    if (!tc_make_map(&d.sig_map, sc + L.sigr, it.ns, L.na64, L.na64, 128)) return NK_ERR_CUDA;
    d.fwd_nseg = fwd_tc_nseg(it.ns, L.mt1, 0, true);
    d.ctr_parts = fwd_centring_parts(it.ns, L.mt1);
    d.splits = batch_item_splits(items, n_inst, order[z], prec);
    d.nb_pa = sr_vec_blocks(L.pa);
    d.nb_ns = sr_vec_blocks(it.ns);
    d.cplx = cplx;
    d.n = r->n;
    d.m = r->m;
    d.n_chains = it.n_chains;
    d.na64 = L.na64;
    d.mt1 = L.mt1;
    d.mp = W.mp;
    d.wmt = W.mt;
    d.wna64 = W.na64;
    d.ns = it.ns;
    d.pa = L.pa;
    d.corner = (int64_t)r->m * L.na + r->n;
    d.ns8 = L.ns8;
    d.sigma = it.sigma;
    d.T = it.t;
    d.eloc = it.eloc;
    d.weights = it.weights;
    d.a = r->a;
    d.b = r->b;
    d.w = r->w;
    d.ws = (char*)r->ws;
    d.ws_a32 = W.a32;
    d.ws_b32 = W.b32;
    d.ws_wt = W.wt;
    d.ws_tab = W.tab;
    d.ws_xw = W.xw;
    d.ws_wbf = W.wbf;
    d.x = sc + L.x;
    d.r = sc + L.r;
    d.p = sc + L.p;
    d.ap = sc + L.ap;
    d.part = sc + L.part;
    d.y = sc + L.y;
    d.v = sc + L.v;
    d.sigt = sc + L.sigt;
    d.sigr = sc + L.sigr;
    d.xbf = sc + L.xbf;
    d.red = (double*)(sc + L.red);
    d.scal = (double*)(sc + L.scal);
    d.done = d.scal + SC_DONE;
    d.info = it.info_out;
    memcpy(&out[z], &d, sizeof(d));
  }
  return NK_OK;
}

// one sub-batch: problems [z0, z0 + G) of the descriptor order (up to kBatchMax)
static nk_status sr_batch_group(const nk_sr_batch_item* items, int n_inst,
                                const std::vector<int>& order, int z0, int G,
                                const SrDesc* D, double eps, double lr, int n_cg, double rtol,
                                int prec, cudaStream_t st) {
  const SrDesc* Dg = D + z0;
  FwdBatch fb{};
  AdjBatch ab{};
  int max_fwd = 1, max_adj = 1, max_sp = 1, max_na64 = 64;
  int64_t max_ns8 = 8, max_xp = 1, max_wp = 1, max_work = 1, max_minb = 1, max_rows = 1;
  for (int z = 0; z < G; ++z) {
    const nk_sr_batch_item& it = items[order[z0 + z]];
    const nk_rbm* r = it.rbm;
    const int cplx = r->is_complex ? 1 : 0;
    const int HJ = cplx ? 64 : 128;
    SrLayout L(r->n, r->m, cplx, it.ns);
    WsLayout W(r->n, r->m, cplx);
    char* sc = (char*)it.scratch;
    double* scal = (double*)(sc + L.scal);
    const int splits = batch_item_splits(items, n_inst, order[z0 + z], prec);
    FwdTcArgs& fa = fb.a[z];
    fa.sigma = it.sigma;
    fa.ns = it.ns;
    fa.n = r->n;
    fa.m = r->m;
    fa.cplx = cplx;
    fa.mode = 0;
    fa.mt = L.mt1;
    fa.na64 = L.na64;
    fa.rows = r->m + 1;
    fa.T = it.t;
    fa.y = sc + L.y;
    fa.skip = scal + SC_DONE;
    fa.err = reinterpret_cast<int*>(scal + SC_ERR);
    fa.nseg = fwd_tc_nseg(it.ns, L.mt1, 0, true);
    if (fwd_centring_parts(it.ns, L.mt1)) {
      fa.mean_part = (double*)(sc + L.red) + 2 * kVecBlocks;
      fa.mean_stride = kVecBlocks;
      fa.weights = it.weights;
    }
    fb.map[z] = &Dg[z].fwd_map;
    fb.smap[z] = &Dg[z].sig_map;
    fb.tiles[z] = (int)((it.ns + 127) / 128);
    AdjTcArgs& aa = ab.a[z];
    aa.T = it.t;
    aa.v = sc + L.v;
    aa.ns = it.ns;
    aa.n = r->n;
    aa.m = r->m;
    aa.cplx = cplx;
    aa.na64 = L.na64;
    aa.splits = splits;
    aa.part = sc + L.part;
    aa.skip = nullptr;
    aa.err = reinterpret_cast<int*>(scal + SC_ERR);
    ab.map[z] = &Dg[z].adj_map;
    ab.chunk[z] = round_up(std::max<int64_t>((it.ns + splits - 1) / splits, 1), 64);
    ab.tiles[z] = (r->m + 1 + HJ - 1) / HJ;
    ab.splits[z] = splits;
    max_fwd = std::max(max_fwd, fb.tiles[z] * fa.nseg);
    max_rows = std::max<int64_t>(max_rows, it.ns * (L.na64 / 8));
    max_adj = std::max(max_adj, ab.tiles[z]);
    max_sp = std::max(max_sp, splits);
    max_na64 = std::max(max_na64, L.na64);
    max_ns8 = std::max<int64_t>(max_ns8, L.ns8);
    max_xp = std::max<int64_t>(max_xp, (int64_t)L.mt1 * 128 * L.na64);
    max_wp = std::max<int64_t>(max_wp, (int64_t)W.mt * 128 * W.na64);
    max_work = std::max<int64_t>(max_work, (int64_t)W.mp * (r->n + 1));
    max_minb = std::max<int64_t>(max_minb, (std::max(W.mp, r->n) + 255) / 256);
  }
  int max_nbp = 1, max_nbs = 1;
  for (int z = 0; z < G; ++z) {
    const nk_sr_batch_item& it = items[order[z0 + z]];
    SrLayout L(it.rbm->n, it.rbm->m, it.rbm->is_complex ? 1 : 0, it.ns);
    max_nbp = std::max(max_nbp, sr_vec_blocks(L.pa));
    max_nbs = std::max(max_nbs, sr_vec_blocks(it.ns));
  }
  const dim3 vg(max_nbp, G), vs(max_nbs, G), one(1, G);
  bool all_fused = true;  // every forward of the group writes its centring partials
  for (int z = 0; z < G; ++z) all_fused = all_fused && fb.a[z].mean_part != nullptr;
  stats_mean_batch<<<vs, kVecThreads, 0, st>>>(Dg);
  stats_dev_batch<<<vs, kVecThreads, 0, st>>>(Dg);
  stats_finish_batch<<<one, 32, 0, st>>>(Dg);
  flags_reset_batch<<<one, 32, 0, st>>>(Dg);
  if (nk_status e = check_launch("nk_sr_step_batch(stats)")) return e;
  if (nk_status e = launch_sigma_t_batch(Dg, G, max_ns8, max_na64, st)) return e;
  if (nk_status e = launch_sigma_rows_batch(Dg, G, max_rows, st)) return e;
  if (nk_status e = launch_adj_tc_batch(ab, G, max_adj, max_sp, max_na64, st)) return e;
  reduce_parts_batch<<<vg, kVecThreads, 0, st>>>(Dg, 0, 0.0);
  cg_init_batch<<<vg, kVecThreads, 0, st>>>(Dg);
  cg_init_scalars_batch<<<one, 32, 0, st>>>(Dg, rtol);
  if (nk_status e = check_launch("nk_sr_step_batch(force)")) return e;
  // the adjoints centre the forwards' outputs themselves when every problem of
  // the group qualifies (otherwise the centring launch runs for all of them)
  bool all_adj_ctr = all_fused;
  for (int z = 0; z < G; ++z) {
    const nk_rbm* r = items[order[z0 + z]].rbm;
    all_adj_ctr = all_adj_ctr && adj_centres(r->m, r->is_complex ? 1 : 0);
  }
  for (int z = 0; z < G; ++z) {
    ab.a[z].skip = fb.a[z].skip;
    if (all_adj_ctr) {
      const nk_sr_batch_item& it = items[order[z0 + z]];
      SrLayout L(it.rbm->n, it.rbm->m, it.rbm->is_complex ? 1 : 0, it.ns);
      ab.a[z].y = (char*)it.scratch + L.y;
      ab.a[z].mean_part = fb.a[z].mean_part;
      ab.a[z].mean_stride = kVecBlocks;
      ab.a[z].mean_parts = fwd_centring_parts(it.ns, L.mt1);
      ab.a[z].weights = it.weights;
    }
  }
  for (int it = 0; it < n_cg; ++it) {
    // from the second CG iteration on, cg_step_p_batch writes the planes of p itself
    if (it == 0) {
      if (nk_status e = launch_bplanes_p_batch(Dg, G, max_xp, st)) return e;
    }
    if (nk_status e = launch_fwd_tc_batch(fb, G, max_fwd, max_na64, st)) return e;
    if (!all_fused) center_partial_batch<<<vs, kVecThreads, 0, st>>>(Dg);
    if (!all_adj_ctr) center_apply_batch<<<vs, kVecThreads, 0, st>>>(Dg);
    if (nk_status e = launch_adj_tc_batch(ab, G, max_adj, max_sp, max_na64, st)) return e;
    reduce_parts_batch<<<vg, kVecThreads, 0, st>>>(Dg, 1, eps);
    cg_step_x_batch<<<vg, kVecThreads, 0, st>>>(Dg, it);
    cg_step_p_batch<<<vg, kVecThreads, 0, st>>>(Dg, it, rtol);
    if (nk_status e = check_launch("nk_sr_step_batch(cg)")) return e;
  }
  sr_update_batch<<<vg, kVecThreads, 0, st>>>(Dg, lr, n_cg, rtol);
  if (nk_status e = check_launch("nk_sr_step_batch(update)")) return e;
  if (nk_status e = launch_prepare_batch(Dg, G, max_work, max_minb, st)) return e;
  return launch_bplanes_rbm_batch(Dg, G, max_wp, st);
}

nk_status run_sr_step_batch(const nk_sr_batch_item* items, int n_inst, const void* desc_dev,
                            double eps, double lr, int n_cg, double rtol, int prec,
                            cudaStream_t st) {
  if (nk_status e = sr_batch_check(items, n_inst, prec)) return e;
  if (!desc_dev || (((uintptr_t)desc_dev) & 255))
    return fail(NK_ERR_INVALID_ARG, "nk_sr_step_batch: descriptors NULL or not 256-byte aligned");
  const std::vector<int> order = batch_order(items, n_inst);
  const SrDesc* D = reinterpret_cast<const SrDesc*>(desc_dev);
  for (int z = 0; z < n_inst; z += kBatchMax) {
    const int G = std::min(kBatchMax, n_inst - z);
    if (nk_status e = sr_batch_group(items, n_inst, order, z, G, D, eps, lr, n_cg, rtol, prec, st))
      return e;
  }
  return NK_OK;
}

// ------------------------------------------------------------------ autotuner

template <bool CPLX>
static nk_status time_adjoint(const nk_rbm* r, const int8_t* sigma, const void* T, int64_t ns,
                              int prec, char* sc, const SrLayout& L, int splits,
                              cudaStream_t st, float* ms) {
  const int64_t corner = (int64_t)r->m * L.na + r->n;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_sr_tune: cannot create events");
  AdjTcArgs aa{};
  aa.T = T;
  aa.v = sc + L.v;
  aa.ns = ns;
  aa.n = r->n;
  aa.m = r->m;
  aa.cplx = CPLX;
  aa.na64 = L.na64;
  aa.splits = splits;
  aa.part = sc + L.part;
  nk_status e = NK_OK;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == NK_OK; ++rep) {
    cudaEventRecord(e0, st);
    if (prec == NK_PREC_BF16X2)
      e = launch_adj_tc(aa, sc + L.sigt, st);
    else
      launch_adjoint_fp32<CPLX>(sigma, T, sc + L.v, ns, r->n, r->m, splits, sc + L.part, nullptr,
                                st);
    reduce_parts_kernel<CPLX><<<sr_vec_blocks(L.pa), kVecThreads, 0, st>>>(
        sc + L.part, splits, L.pa, corner, sc + L.ap, nullptr, 0.0, nullptr, nullptr);
    cudaEventRecord(e1, st);
    if (e == NK_OK) e = check_launch("nk_sr_tune");
    if (cudaEventSynchronize(e1) != cudaSuccess) e = fail(NK_ERR_CUDA, "nk_sr_tune: sync");
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) best = std::min(best, t);  // first repetition is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return e;
}

nk_status run_sr_tune(nk_rbm* r, const int8_t* sigma, const void* t, int64_t ns, int prec,
                      void* scratch, size_t scratch_bytes, cudaStream_t st) {
  SrLayout L(r->n, r->m, r->is_complex, ns);
  if (scratch_bytes < L.total)
    return fail(NK_ERR_SHAPE, "nk_sr_tune: scratch of %zu B, need %zu B", scratch_bytes, L.total);
  char* sc = (char*)scratch;
  // any finite v: only the timing matters
  if (cudaMemsetAsync(sc + L.v, 0, (size_t)ns * (r->is_complex ? 16 : 8), st) != cudaSuccess)
    return fail(NK_ERR_CUDA, "nk_sr_tune: memset");
  if (prec == NK_PREC_BF16X2) {
    if (nk_status e = launch_sigma_t(sigma, ns, r->n, L.na64, sc + L.sigt, st)) return e;
  }
  const int h = prec == NK_PREC_BF16X2 ? L.splits_tc : L.splits_fp32;
  // candidates: the heuristic, half of it, and the split counts that fill
  // one to four whole waves of adjoint CTAs (one per SM)
  const int hj = tc_hidden_per_tile(r->is_complex);
  const int tiles = prec == NK_PREC_BF16X2 ? (r->m + 1 + hj - 1) / hj
                                           : ceil_div(L.na, 64) * ceil_div(L.ma, 64);
  int cand[6] = {h, h / 2};
  for (int k = 1; k <= 4; ++k) cand[1 + k] = (k * 152) / tiles;
  int best_s = sr_choose_splits(L, prec, h);
  float best_t = 1e30f;
  int tried[6];
  int n_tried = 0;
  for (int k = 0; k < 6; ++k) {
    const int sp = sr_choose_splits(L, prec, std::max(1, cand[k]));
    bool seen = false;
    for (int u = 0; u < n_tried; ++u) seen = seen || tried[u] == sp;
    if (seen) continue;
    tried[n_tried++] = sp;
    float ms = 0.f;
    nk_status e = r->is_complex
                      ? time_adjoint<true>(r, sigma, t, ns, prec, sc, L, sp, st, &ms)
                      : time_adjoint<false>(r, sigma, t, ns, prec, sc, L, sp, st, &ms);
    if (e) return e;
    if (ms < best_t) {
      best_t = ms;
      best_s = sp;
    }
  }
  r->sr_splits = best_s;
  return NK_OK;
}

// ------------------------------------------------------------------ K8 backward
// grad_k = sum_s conj(O_sk) g_s (analytic RBM log-derivatives, Sec. 2.2.5) over
// chunks of at most kBackChunk samples: per chunk, T = tanh(theta) is
// recomputed from sigma (the theta contraction of ln psi with a tanh epilogue
// and no ln cosh), the adjoint contraction writes its split-K partials, the
// partials are reduced over splits (fixed order) and the chunk's sum is added
// to an FP64 accumulator in chunk order.  Scratch holds one chunk's T and the
// adjoint's buffers for one chunk: it does not grow with ns beyond kBackChunk.

constexpr int64_t kBackChunk = 16384;

static int64_t backward_chunk(int64_t ns) {
  return std::min<int64_t>(std::max<int64_t>(ns, 1), kBackChunk);
}

size_t backward_scratch_bytes(int n, int m, int cplx, int64_t ns) {
  const int64_t c = backward_chunk(ns);
  SrLayout L(n, m, cplx, c);
  const size_t f = cplx ? 8 : 4;
  return L.total + (size_t)round_up(c * m * f, 256) +
         (size_t)round_up(L.pa * (cplx ? 16 : 8), 256);
}

template <bool CPLX>
__global__ void copy_g_kernel(const double* g, void* v, int64_t ns) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns;
       s += (int64_t)gridDim.x * blockDim.x) {
    if (CPLX) reinterpret_cast<double2*>(v)[s] = make_double2(g[2 * s], g[2 * s + 1]);
    else reinterpret_cast<double*>(v)[s] = g[2 * s];
  }
}

// acc = x (first chunk) or acc + x
template <bool CPLX>
__global__ void accumulate_kernel(void* accv, const void* xv, int64_t pa, int first) {
  using DT = typename D<CPLX>::T;
  DT* acc = reinterpret_cast<DT*>(accv);
  const DT* x = reinterpret_cast<const DT*>(xv);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < pa;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (first) {
      acc[e] = x[e];
    } else if constexpr (CPLX) {
      acc[e] = make_double2(acc[e].x + x[e].x, acc[e].y + x[e].y);
    } else {
      acc[e] += x[e];
    }
  }
}

template <bool CPLX>
static nk_status backward_t(const nk_rbm* r, const int8_t* sigma, int64_t ns, const double* g,
                            double* grad, int prec, char* sc, cudaStream_t st) {
  const int64_t chunk = backward_chunk(ns);
  SrLayout L(r->n, r->m, CPLX, chunk);
  const size_t f = CPLX ? 8 : 4;
  char* T = sc + L.total;
  char* acc = T + round_up(chunk * r->m * f, 256);
  const bool tc = prec == NK_PREC_BF16X2;
  const int splits = sr_choose_splits(L, prec, r->sr_splits);
  const int64_t corner = (int64_t)r->m * L.na + r->n;
  const int64_t nchunks = (ns + chunk - 1) / chunk;
  for (int64_t k = 0; k < nchunks; ++k) {
    const int64_t c0 = k * chunk, cn = std::min<int64_t>(chunk, ns - c0);
    const int8_t* sg = sigma + c0 * r->n;
    const int sp = (int)std::max<int64_t>(1, std::min<int64_t>(splits, (cn + 63) / 64));
    nk_status e = tc ? launch_logpsi_bf16(r, sg, cn, nullptr, nullptr, st, T)
                     : launch_logpsi_fp32(r, sg, cn, nullptr, nullptr, st, T);
    if (e) return e;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((cn + 255) / 256, 1024));
    copy_g_kernel<CPLX><<<(unsigned)blocks, 256, 0, st>>>(g + 2 * c0, sc + L.v, cn);
    if (tc) {
      if ((e = launch_sigma_t(sg, cn, r->n, L.na64, sc + L.sigt, st))) return e;
      AdjTcArgs aa{};
      aa.T = T;
      aa.v = sc + L.v;
      aa.ns = cn;
      aa.n = r->n;
      aa.m = r->m;
      aa.cplx = CPLX;
      aa.na64 = L.na64;
      aa.splits = sp;
      aa.part = sc + L.part;
      if ((e = launch_adj_tc(aa, sc + L.sigt, st))) return e;
    } else {
      launch_adjoint_fp32<CPLX>(sg, T, sc + L.v, cn, r->n, r->m, sp, sc + L.part, nullptr, st);
    }
    reduce_parts_kernel<CPLX><<<sr_vec_blocks(L.pa), kVecThreads, 0, st>>>(
        sc + L.part, sp, L.pa, corner, sc + L.x, nullptr, 0.0, nullptr, nullptr);
    if (nchunks > 1)
      accumulate_kernel<CPLX><<<sr_vec_blocks(L.pa), kVecThreads, 0, st>>>(acc, sc + L.x, L.pa,
                                                                           k == 0 ? 1 : 0);
  }
  scatter_grad_kernel<CPLX><<<sr_vec_blocks(L.pa), kVecThreads, 0, st>>>(
      nchunks > 1 ? acc : sc + L.x, r->n, r->m, grad);
  return check_launch("nk_rbm_logpsi_backward");
}

nk_status run_backward(const nk_rbm* r, const int8_t* sigma, int64_t ns, const double* g,
                       double* grad, int prec, void* scratch, size_t scratch_bytes,
                       cudaStream_t st) {
  size_t need = backward_scratch_bytes(r->n, r->m, r->is_complex, ns);
  if (scratch_bytes < need)
    return fail(NK_ERR_SHAPE, "nk_rbm_logpsi_backward: scratch of %zu B, need %zu B",
                scratch_bytes, need);
  return r->is_complex ? backward_t<true>(r, sigma, ns, g, grad, prec, (char*)scratch, st)
                       : backward_t<false>(r, sigma, ns, g, grad, prec, (char*)scratch, st);
}

}  // namespace nk
