// Multi-layer feed-forward network with ln cosh activations (Sec. 2.2.2: FFNN
// machines of dense layers y = W x + b and Lncosh activations with a sum
// output; the one-layer network is the RBM without visible bias):
//   x_0 = sigma,  h_l = W_l x_(l-1) + b_l,  x_l = ln cosh(h_l),  ln psi = sum_j x_(L, j),
// and its backward grad_k = sum_s conj(O_sk) g_s (the convention of the RBM
// backward) by the holomorphic chain rule:
//   e_L = conj(tanh h_L) g,  e_(l-1) = conj(tanh h_(l-1)) (e_l conj(W_l)),
//   grad W_l = e_l^T conj(x_(l-1)),  grad b_l = sum_s e_l.
// Every contraction runs on the CUDA cores in FP32 (64 x 64 output tiles, 16-deep
// K chunks, a 4 x 4 register block per thread) reading the FP64 master
// parameters directly; ln psi and the gradients are summed in FP64 (the weight
// gradients over sample splits in a fixed order).  The backward recomputes the
// forward into its scratch, so it needs nothing from an earlier call.
#include "common.cuh"
#include "internal.h"

namespace nk {

namespace {

constexpr int kFT = 64;       // output tile (rows and columns)
constexpr int kFK = 16;       // K chunk
constexpr int kFThreads = 256;
constexpr int kFMaxLayers = 8;

template <bool CPLX>
struct FT;
template <>
struct FT<true> {
  using F = float2;
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
};
template <>
struct FT<false> {
  using F = float;
  static __device__ __forceinline__ float zero() { return 0.f; }
};

__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cconj(float a) { return a; }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float cmul(float a, float b) { return a * b; }

template <bool CPLX>
__device__ __forceinline__ typename FT<CPLX>::F from_master(const double* p, int64_t k) {
  if constexpr (CPLX) return make_float2((float)p[2 * k], (float)p[2 * k + 1]);
  else return (float)p[k];
}

template <bool CPLX>
__device__ __forceinline__ typename FT<CPLX>::F lncosh_t(typename FT<CPLX>::F h) {
  if constexpr (CPLX) {
    cf l = lncosh_c(cf{h.x, h.y});
    return make_float2(l.x, l.y);
  } else {
    return lncosh_f(h);
  }
}

template <bool CPLX>
__device__ __forceinline__ typename FT<CPLX>::F tanh_t(typename FT<CPLX>::F h) {
  if constexpr (CPLX) {
    cf t = tanh_c(cf{h.x, h.y});
    return make_float2(t.x, t.y);
  } else {
    return tanh_f(h);
  }
}

// C[r][c] = sum_{k in [kb, ke)} A(r, k) B(c, k) for one 64 x 64 tile.  The
// loaders return an operand element (zero outside the problem); ROW_FAST_A / _B
// choose which index consecutive threads step through when a tile is staged
// (the one contiguous in memory).  Epi(r, c, acc) receives every element of the
// tile that lies inside R x C.
template <bool CPLX, bool ROW_FAST_A, bool ROW_FAST_B, class LA, class LB, class Epi>
__device__ __forceinline__ void gemm_tile(int64_t R, int64_t C, int64_t kb, int64_t ke,
                                          int64_t r0, int64_t c0, const LA& la, const LB& lb,
                                          const Epi& epi) {
  using F = typename FT<CPLX>::F;
  __shared__ __align__(16) F As[kFK][kFT];
  __shared__ __align__(16) F Bs[kFK][kFT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  F acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = FT<CPLX>::zero();
  for (int64_t k0 = kb; k0 < ke; k0 += kFK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * kFThreads;
      const int ra = ROW_FAST_A ? (e & 63) : (e >> 4), ka = ROW_FAST_A ? (e >> 6) : (e & 15);
      const int rb = ROW_FAST_B ? (e & 63) : (e >> 4), kb2 = ROW_FAST_B ? (e >> 6) : (e & 15);
      const int64_t k_a = k0 + ka, k_b = k0 + kb2;
      As[ka][ra] = (r0 + ra < R && k_a < ke) ? la(r0 + ra, k_a) : FT<CPLX>::zero();
      Bs[kb2][rb] = (c0 + rb < C && k_b < ke) ? lb(c0 + rb, k_b) : FT<CPLX>::zero();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kFK; ++kk) {
      F a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = As[kk][ty * 4 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if constexpr (CPLX) {
            acc[p][q].x = fmaf(a[p].x, b[q].x, fmaf(-a[p].y, b[q].y, acc[p][q].x));
            acc[p][q].y = fmaf(a[p].x, b[q].y, fmaf(a[p].y, b[q].x, acc[p][q].y));
          } else {
            acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
          }
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t r = r0 + ty * 4 + p, c = c0 + tx + 16 * q;
      if (r < R && c < C) epi(r, c, acc[p][q]);
    }
}

// ---------------------------------------------------------------- forward

// h_l = x_(l-1) W_l^T + b_l for a tile of samples x outputs; stores h_l and
// x_l = ln cosh(h_l).  Layer 1 reads sigma (int8).
template <bool CPLX, bool FIRST>
__global__ void __launch_bounds__(kFThreads) ffnn_fwd_kernel(const int8_t* __restrict__ sigma,
                                                             const void* __restrict__ xin,
                                                             int64_t ns, int win, int wout,
                                                             const double* __restrict__ Wm,
                                                             const double* __restrict__ bm,
                                                             void* hout, void* xout) {
  using F = typename FT<CPLX>::F;
  const F* X = reinterpret_cast<const F*>(xin);
  F* H = reinterpret_cast<F*>(hout);
  F* Y = reinterpret_cast<F*>(xout);
  auto la = [&](int64_t s, int64_t i) -> F {
    if constexpr (FIRST) {
      F v = FT<CPLX>::zero();
      if constexpr (CPLX) v.x = (float)sigma[s * win + i]; else v = (float)sigma[s * win + i];
      return v;
    } else {
      return X[s * win + i];
    }
  };
  auto lb = [&](int64_t j, int64_t i) -> F { return from_master<CPLX>(Wm, j * win + i); };
  auto epi = [&](int64_t s, int64_t j, F acc) {
    const F b = from_master<CPLX>(bm, j);
    F h;
    if constexpr (CPLX) h = make_float2(acc.x + b.x, acc.y + b.y); else h = acc + b;
    H[s * wout + j] = h;
    Y[s * wout + j] = lncosh_t<CPLX>(h);
  };
  gemm_tile<CPLX, false, false>(ns, wout, 0, win, (int64_t)blockIdx.y * kFT,
                                (int64_t)blockIdx.x * kFT, la, lb, epi);
}

// ln psi_s = sum_j x_(L, s, j), FP64, one warp per sample (fixed order)
template <bool CPLX>
__global__ void ffnn_rowsum_kernel(const void* __restrict__ xl, int64_t ns, int w,
                                   double* __restrict__ logpsi) {
  using F = typename FT<CPLX>::F;
  const F* X = reinterpret_cast<const F*>(xl);
  const int lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (s >= ns) return;
  double r = 0.0, i = 0.0;
  for (int j = lane; j < w; j += 32) {
    const F v = X[s * w + j];
    if constexpr (CPLX) {
      r += (double)v.x;
      i += (double)v.y;
    } else {
      r += (double)v;
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    r += __shfl_xor_sync(0xffffffffu, r, off);
    i += __shfl_xor_sync(0xffffffffu, i, off);
  }
  if (lane == 0) {
    logpsi[2 * s] = r;
    logpsi[2 * s + 1] = i;
  }
}

// ---------------------------------------------------------------- backward

// e_L = conj(tanh h_L) g
template <bool CPLX>
__global__ void ffnn_top_kernel(const void* __restrict__ hl, const double* __restrict__ g,
                                int64_t ns, int w, void* eout) {
  using F = typename FT<CPLX>::F;
  const F* H = reinterpret_cast<const F*>(hl);
  F* E = reinterpret_cast<F*>(eout);
  const int64_t tot = ns * w;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < tot;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = x / w;
    const F t = cconj(tanh_t<CPLX>(H[x]));
    if constexpr (CPLX) E[x] = cmul(t, make_float2((float)g[2 * s], (float)g[2 * s + 1]));
    else E[x] = t * (float)g[2 * s];
  }
}

// e_(l-1)[s][i] = conj(tanh h_(l-1)[s][i]) sum_j e_l[s][j] conj(W_l[j][i])
template <bool CPLX>
__global__ void __launch_bounds__(kFThreads) ffnn_bwd_kernel(const void* __restrict__ ein,
                                                             const void* __restrict__ hprev,
                                                             int64_t ns, int wl, int wprev,
                                                             const double* __restrict__ Wm,
                                                             void* eout) {
  using F = typename FT<CPLX>::F;
  const F* E = reinterpret_cast<const F*>(ein);
  const F* H = reinterpret_cast<const F*>(hprev);
  F* Eo = reinterpret_cast<F*>(eout);
  auto la = [&](int64_t s, int64_t j) -> F { return E[s * wl + j]; };
  auto lb = [&](int64_t i, int64_t j) -> F { return cconj(from_master<CPLX>(Wm, j * wprev + i)); };
  auto epi = [&](int64_t s, int64_t i, F acc) {
    Eo[s * wprev + i] = cmul(cconj(tanh_t<CPLX>(H[s * wprev + i])), acc);
  };
  gemm_tile<CPLX, false, true>(ns, wprev, 0, wl, (int64_t)blockIdx.y * kFT,
                               (int64_t)blockIdx.x * kFT, la, lb, epi);
}

// partial[z][j][i] = sum_{s in split z} e_l[s][j] conj(x'_(l-1)[s][i]),
// x' = [x | 1] (i = wprev is the bias column); layer 1 reads sigma
template <bool CPLX, bool FIRST>
__global__ void __launch_bounds__(kFThreads) ffnn_wgrad_kernel(const void* __restrict__ ein,
                                                               const int8_t* __restrict__ sigma,
                                                               const void* __restrict__ xprev,
                                                               int64_t ns, int wl, int wprev,
                                                               int64_t chunk, void* partv) {
  using F = typename FT<CPLX>::F;
  const F* E = reinterpret_cast<const F*>(ein);
  const F* X = reinterpret_cast<const F*>(xprev);
  F* part = reinterpret_cast<F*>(partv) + (int64_t)blockIdx.z * wl * (wprev + 1);
  auto la = [&](int64_t j, int64_t s) -> F { return E[s * wl + j]; };
  auto lb = [&](int64_t i, int64_t s) -> F {
    F v = FT<CPLX>::zero();
    if (i == wprev) {
      if constexpr (CPLX) v.x = 1.f; else v = 1.f;
    } else if constexpr (FIRST) {
      if constexpr (CPLX) v.x = (float)sigma[s * wprev + i]; else v = (float)sigma[s * wprev + i];
    } else {
      v = cconj(X[s * wprev + i]);
    }
    return v;
  };
  auto epi = [&](int64_t j, int64_t i, F acc) { part[j * (wprev + 1) + i] = acc; };
  const int64_t kb = (int64_t)blockIdx.z * chunk, ke = std::min<int64_t>(ns, kb + chunk);
  gemm_tile<CPLX, true, true>(wl, wprev + 1, kb, ke, (int64_t)blockIdx.y * kFT,
                              (int64_t)blockIdx.x * kFT, la, lb, epi);
}

// grad (this layer's W then b, flat, FP64) = fixed-order sum over the splits
template <bool CPLX>
__global__ void ffnn_wreduce_kernel(const void* __restrict__ partv, int splits, int wl, int wprev,
                                    double* __restrict__ grad) {
  using F = typename FT<CPLX>::F;
  const F* part = reinterpret_cast<const F*>(partv);
  const int64_t per = (int64_t)wl * (wprev + 1);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < per;
       x += (int64_t)gridDim.x * blockDim.x) {
    double r = 0.0, im = 0.0;
    for (int z = 0; z < splits; ++z) {
      const F v = part[z * per + x];
      if constexpr (CPLX) {
        r += (double)v.x;
        im += (double)v.y;
      } else {
        r += (double)v;
      }
    }
    const int64_t j = x / (wprev + 1), i = x % (wprev + 1);
    const int64_t k = i < wprev ? j * wprev + i : (int64_t)wl * wprev + j;
    if constexpr (CPLX) {
      grad[2 * k] = r;
      grad[2 * k + 1] = im;
    } else {
      grad[k] = r;
    }
  }
}

struct FfnnLayout {
  int L, cplx;
  int w[kFMaxLayers + 1];
  int64_t ns;
  int splits;
  size_t h[kFMaxLayers], x[kFMaxLayers], e0, e1, part, total;
  int64_t off[kFMaxLayers];  // flat parameter offset of each layer (in parameters)
  int64_t chunk;
  FfnnLayout(const nk_ffnn* f, int64_t ns_) {
    L = f->n_layers;
    cplx = f->is_complex ? 1 : 0;
    ns = std::max<int64_t>(ns_, 1);
    for (int l = 0; l <= L; ++l) w[l] = f->widths[l];
    const size_t fs = cplx ? 8 : 4;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t o = 0;
    int wmax = 0;
    int64_t pmax = 0, po = 0;
    for (int l = 1; l <= L; ++l) {
      h[l - 1] = o;
      o += up((size_t)ns * w[l] * fs);
      x[l - 1] = o;
      o += up((size_t)ns * w[l] * fs);
      wmax = std::max(wmax, w[l]);
      pmax = std::max<int64_t>(pmax, (int64_t)w[l] * (w[l - 1] + 1));
      off[l - 1] = po;
      po += (int64_t)w[l] * (w[l - 1] + 1);
    }
    splits = (int)std::min<int64_t>(16, std::max<int64_t>(1, ns / 1024));
    chunk = ((ns + splits - 1) / splits + kFK - 1) / kFK * kFK;
    e0 = o;
    o += up((size_t)ns * wmax * fs);
    e1 = o;
    o += up((size_t)ns * wmax * fs);
    part = o;
    o += up((size_t)splits * pmax * fs);
    total = o;
  }
};

dim3 tiles(int64_t rows, int64_t cols, int z = 1) {
  return dim3((unsigned)((cols + kFT - 1) / kFT), (unsigned)((rows + kFT - 1) / kFT), (unsigned)z);
}

template <bool CPLX>
nk_status forward_t(const nk_ffnn* f, const FfnnLayout& Lo, const int8_t* sigma, int64_t ns,
                    double* logpsi, char* sc, cudaStream_t st) {
  const int64_t fs = CPLX ? 2 : 1;  // doubles per parameter
  for (int l = 1; l <= Lo.L; ++l) {
    const double* Wm = f->params + fs * Lo.off[l - 1];
    const double* bm = Wm + fs * (int64_t)Lo.w[l] * Lo.w[l - 1];
    if (l == 1)
      ffnn_fwd_kernel<CPLX, true><<<tiles(ns, Lo.w[1]), kFThreads, 0, st>>>(
          sigma, nullptr, ns, Lo.w[0], Lo.w[1], Wm, bm, sc + Lo.h[0], sc + Lo.x[0]);
    else
      ffnn_fwd_kernel<CPLX, false><<<tiles(ns, Lo.w[l]), kFThreads, 0, st>>>(
          sigma, sc + Lo.x[l - 2], ns, Lo.w[l - 1], Lo.w[l], Wm, bm, sc + Lo.h[l - 1],
          sc + Lo.x[l - 1]);
  }
  if (logpsi)
    ffnn_rowsum_kernel<CPLX><<<(unsigned)((ns + 7) / 8), 256, 0, st>>>(sc + Lo.x[Lo.L - 1], ns,
                                                                      Lo.w[Lo.L], logpsi);
  return check_launch("nk_ffnn forward");
}

template <bool CPLX>
nk_status backward_t(const nk_ffnn* f, const FfnnLayout& Lo, const int8_t* sigma, int64_t ns,
                     const double* g, double* grad, char* sc, cudaStream_t st) {
  if (nk_status e = forward_t<CPLX>(f, Lo, sigma, ns, nullptr, sc, st)) return e;
  const int64_t fs = CPLX ? 2 : 1;
  const int L = Lo.L;
  char* ecur = sc + Lo.e0;
  char* enext = sc + Lo.e1;
  const int64_t tot = ns * Lo.w[L];
  ffnn_top_kernel<CPLX><<<(unsigned)std::min<int64_t>(1024, (tot + 255) / 256), 256, 0, st>>>(
      sc + Lo.h[L - 1], g, ns, Lo.w[L], ecur);
  for (int l = L; l >= 1; --l) {
    const double* Wm = f->params + fs * Lo.off[l - 1];
    const int wl = Lo.w[l], wp = Lo.w[l - 1];
    if (l == 1)
      ffnn_wgrad_kernel<CPLX, true><<<tiles(wl, wp + 1, Lo.splits), kFThreads, 0, st>>>(
          ecur, sigma, nullptr, ns, wl, wp, Lo.chunk, sc + Lo.part);
    else
      ffnn_wgrad_kernel<CPLX, false><<<tiles(wl, wp + 1, Lo.splits), kFThreads, 0, st>>>(
          ecur, sigma, sc + Lo.x[l - 2], ns, wl, wp, Lo.chunk, sc + Lo.part);
    const int64_t per = (int64_t)wl * (wp + 1);
    ffnn_wreduce_kernel<CPLX><<<(unsigned)std::min<int64_t>(1024, (per + 255) / 256), 256, 0, st>>>(
        sc + Lo.part, Lo.splits, wl, wp, grad + fs * Lo.off[l - 1]);
    if (l > 1) {
      ffnn_bwd_kernel<CPLX><<<tiles(ns, wp), kFThreads, 0, st>>>(ecur, sc + Lo.h[l - 2], ns, wl,
                                                                 wp, Wm, enext);
      std::swap(ecur, enext);
    }
  }
  return check_launch("nk_ffnn backward");
}

}  // namespace

nk_status check_ffnn(const nk_ffnn* f, const char* who) {
  if (!f || !f->widths || !f->params) return fail(NK_ERR_INVALID_ARG, "%s: NULL network", who);
  if (f->n_layers < 1 || f->n_layers > kFMaxLayers)
    return fail(NK_ERR_SHAPE, "%s: n_layers = %d outside [1, %d]", who, f->n_layers, kFMaxLayers);
  for (int l = 0; l <= f->n_layers; ++l)
    if (f->widths[l] < 1 || f->widths[l] > (1 << 20))
      return fail(NK_ERR_SHAPE, "%s: width %d of layer %d", who, f->widths[l], l);
  return NK_OK;
}

size_t ffnn_scratch_bytes(const nk_ffnn* f, int64_t ns) { return FfnnLayout(f, ns).total; }

nk_status run_ffnn_logpsi(const nk_ffnn* f, const int8_t* sigma, int64_t ns, double* logpsi,
                          void* scratch, size_t bytes, cudaStream_t st) {
  FfnnLayout Lo(f, ns);
  if (bytes < Lo.total)
    return fail(NK_ERR_SHAPE, "nk_ffnn_logpsi: scratch of %zu B, need %zu B", bytes, Lo.total);
  return f->is_complex ? forward_t<true>(f, Lo, sigma, ns, logpsi, (char*)scratch, st)
                       : forward_t<false>(f, Lo, sigma, ns, logpsi, (char*)scratch, st);
}

nk_status run_ffnn_backward(const nk_ffnn* f, const int8_t* sigma, int64_t ns, const double* g,
                            double* grad, void* scratch, size_t bytes, cudaStream_t st) {
  FfnnLayout Lo(f, ns);
  if (bytes < Lo.total)
    return fail(NK_ERR_SHAPE, "nk_ffnn_backward: scratch of %zu B, need %zu B", bytes, Lo.total);
  return f->is_complex ? backward_t<true>(f, Lo, sigma, ns, g, grad, (char*)scratch, st)
                       : backward_t<false>(f, Lo, sigma, ns, g, grad, (char*)scratch, st);
}

}  // namespace nk
